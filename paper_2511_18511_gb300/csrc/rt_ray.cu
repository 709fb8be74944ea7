// rt_ray.cu — kernels of the ToF path: field packing, shooting-method linking
// with the fused travel time, travel time at fixed angles, the adjoint scatter
// and the explicit system-matrix rows.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cfloat>
#include <climits>
#include <cstdint>
#include <type_traits>

#include <cub/device/device_scan.cuh>
#include <math_constants.h>

#include "rt_internal.h"
#include "rt_trace.cuh"
#include "rt_link.cuh"
#include "rt_bspline.cuh"

namespace rt {

constexpr int kBlock = 128;

static int grid_for(int n) { return (n + kBlock - 1) / kBlock; }

size_t node_bytes(int prec, int interp) {
    if (interp == RT_BSPLINE) return prec == RT_FP64 ? sizeof(CellBS<double>) : sizeof(CellBS<float>);
    return prec == RT_FP64 ? sizeof(CellCoef<double>) : sizeof(CellCoef<float>);
}

// Field layout and register cache of each sampler (template argument I =
// enum rt_interpolator), and the resident blocks per SM the persistent kernels
// are compiled for.
template <typename T, int I> struct Samp;
template <typename T> struct Samp<T, RT_BILINEAR> {
    using Field = CellCoef<T>;
    using CellT = Cell<T>;
};
template <typename T> struct Samp<T, RT_BSPLINE> {
    using Field = CellBS<T>;
    using CellT = CellS<T>;
};
template <typename T, int I> struct Occ { static constexpr int blocks = LinkOcc<T>::blocks; };
template <> struct Occ<float, RT_BSPLINE> { static constexpr int blocks = 4; };

template <typename T, int I>
__device__ __forceinline__ typename Samp<T, I>::CellT make_cell(const Geom& G, const typename Samp<T, I>::Field* F) {
    typename Samp<T, I>::CellT C;
    C.F = F;
    C.nx = G.nx;
    C.ny = G.ny;
    C.pi = INT_MIN;
    C.pj = INT_MIN;
    return C;
}

// ---------------------------------------------------------------- A1: field pack

// Nodal values at node (i, j): c (mm/us), h*dc/dx and h*dc/dy by central
// differences inside and one-sided differences at the edges (paper Sec. 3.3.1:
// the gradient is interpolated from grid values), and s = 1/c.
__device__ __forceinline__ void node_vals(const double* __restrict__ c_mps, int nx, int ny, int i, int j,
                                          double v[4]) {
    const size_t k = (size_t)j * nx + i;
    const double c = 1e-3 * c_mps[k];
    const double cxm = 1e-3 * c_mps[i > 0 ? k - 1 : k], cxp = 1e-3 * c_mps[i < nx - 1 ? k + 1 : k];
    const double cym = 1e-3 * c_mps[j > 0 ? k - nx : k], cyp = 1e-3 * c_mps[j < ny - 1 ? k + nx : k];
    v[0] = c;
    v[1] = (i > 0 && i < nx - 1) ? 0.5 * (cxp - cxm) : (cxp - cxm);
    v[2] = (j > 0 && j < ny - 1) ? 0.5 * (cyp - cym) : (cyp - cym);
    v[3] = 1.0 / c;
}

// A1: per-cell bilinear coefficients of the four nodal fields, computed in FP64
// and stored in the marching precision; flags c <= 0 or NaN.
template <typename T>
__global__ void k_pack(const double* __restrict__ c_mps, int nx, int ny, CellCoef<T>* F, int* bad) {
    const int ncx = nx - 1, n = ncx * (ny - 1);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int j = k / ncx, i = k - j * ncx;
        double v00[4], v10[4], v01[4], v11[4];
        node_vals(c_mps, nx, ny, i, j, v00);
        node_vals(c_mps, nx, ny, i + 1, j, v10);
        node_vals(c_mps, nx, ny, i, j + 1, v01);
        node_vals(c_mps, nx, ny, i + 1, j + 1, v11);
        const double cs[4] = {v00[0], v10[0], v01[0], v11[0]};
        for (int q = 0; q < 4; ++q)
            if (!(cs[q] > 0.0) || !isfinite(cs[q])) atomicOr(bad, 1);
        typename Vec4T<T>::type f[4];
        for (int q = 0; q < 4; ++q) {
            f[q].x = (T)v00[q];
            f[q].y = (T)(v10[q] - v00[q]);
            f[q].z = (T)(v01[q] - v00[q]);
            f[q].w = (T)((v11[q] - v10[q]) - (v01[q] - v00[q]));
        }
        CellCoef<T> o;
        o.c = f[0];
        o.gx = f[1];
        o.gy = f[2];
        o.s = f[3];
        F[k] = o;
    }
}

__global__ void k_tx_phi(const double* __restrict__ tx, int n_tx, double R, double* __restrict__ phi) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tx) return;
    const double x = tx[2 * t], y = tx[2 * t + 1];
    phi[t] = on_ring(x, y, R) ? atan2(y, x) : nan("");
}

cudaError_t launch_tx_phi(const Geom& G, double* phi, cudaStream_t s) {
    k_tx_phi<<<(G.n_tx + 127) / 128, 128, 0, s>>>(G.tx, G.n_tx, G.R, phi);
    return cudaGetLastError();
}

cudaError_t launch_pack(const rt_grid& g, const double* c_mps, void* field, int* dflag, int prec,
                        cudaStream_t s) {
    const int n = (g.nx - 1) * (g.ny - 1);
    const int blocks = (n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16;
    cudaError_t e = cudaMemsetAsync(dflag, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (prec == RT_FP64)
        k_pack<double><<<blocks, 256, 0, s>>>(c_mps, g.nx, g.ny, (CellCoef<double>*)field, dflag);
    else
        k_pack<float><<<blocks, 256, 0, s>>>(c_mps, g.nx, g.ny, (CellCoef<float>*)field, dflag);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- A4: linking

// ---------------------------------------------------------------- fan start

// Cold-start prediction from a fan of K rays per emitter at evenly spaced
// angles over the inward fan (an option; fan_rays = 0 keeps the paper's
// straight-line start, Sec. 3.4.1). psi = interception angle counter-clockwise
// from the emitter, NaN when the ray has no interception.
__global__ void k_fan_mark(Geom G, const double* __restrict__ theta, int* need) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G.n_pairs) return;
    int e, r;
    pair_of(G, k, e, r);
    if (e >= 0 && e < G.n_tx && isnan(theta[k])) need[e] = 1;
}

// Thread order: the ray of fan index k of emitter e runs on thread
// e + n_tx * rank(k), where rank orders the fan indices from the middle of the
// fan (toward the centre, the longest rays) outward. A warp then marches the
// same relative angle from consecutive emitters: nearly parallel rays of nearly
// equal length through nearby cells, and the launch ends with the short rays
// near the tangents.
// G carries the fan's tracing step; margin (ds/R of the linking step) fixes
// the fan's launch angles, which the linking predictions assume.
template <typename T, int I>
__global__ void __launch_bounds__(kBlock) k_fan(Geom G, const typename Samp<T, I>::Field* __restrict__ F, int K,
                                                double margin, const int* __restrict__ need, double* fan,
                                                unsigned long long* counters) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    const int rank = id / G.n_tx, e = id - rank * G.n_tx;
    const int half = K / 2;
    const int k = (rank & 1) ? half - (rank + 1) / 2 : half + rank / 2;
    long long steps = 0;
    if (id < G.n_tx * K && need[e] && !*G.bad_field) {
        const double xe = G.tx[2 * e], ye = G.tx[2 * e + 1];
        const double phi_e = atan2(ye, xe);
        const double a_min = phi_e + 0.5 * kPi + margin, a_max = phi_e + 1.5 * kPi - margin;
        const double step = (a_max - a_min) / (K - 1);
        auto C = make_cell<T, I>(G, F);
        NoSink ns;
        const TraceOut o = trace_ray<T>(C, G, xe, ye, fan_theta(a_min, step, k), xe, ye, ns);
        fan[(size_t)e * K + k] = (o.flags & 3) ? nan("") : mod_2pi(atan2(o.hy, o.hx) - phi_e);
        steps = o.steps;
    }
    // every thread of the block reaches this point
    __syncwarp();
    unsigned long long v = (unsigned long long)steps;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&counters[7], v);
}

// Persistent linking kernel: each lane takes pairs from the queue, advances
// its own trace up to kLinkSteps RK4 steps per loop iteration, and updates the
// linking state when a trace ends, so lanes never wait for other lanes' pairs
// (a lane whose trace ends early in an iteration idles for the rest of it).
// The iteration's bookkeeping (queue fetch, reconvergence of the warp) cost a
// lone lane about 85 ns per step at one step per iteration: 537 against 363 ns
// per RK4 step for the plain traced-ray kernel; at 16 steps it is 428 ns.
// Resident blocks per SM the link kernel is compiled for. The recording
// variant, which keeps a run accumulator per lane, runs 4 blocks (128
// registers): 53.0 against 54.5 ms at 5 on the cold breast workload. The plain
// FP32 link stays at 6 (80 registers): at 5 its cold link was no faster and
// its warm start (one trace per pair, throughput-bound) slower.
template <typename T, int I, bool REC> struct LinkBlocks { static constexpr int v = Occ<T, I>::blocks; };
template <typename T, int I> struct LinkBlocks<T, I, true> { static constexpr int v = 4; };

// RK4 steps per loop iteration of k_link (measured on the breast workload:
// 1 -> 60.6 ms, 4 -> 55.1, 8 -> 54.5, 16 -> 53.6 for the recording link)
constexpr int kLinkSteps = 16;

template <typename T, int I, bool REC, bool ROUNDS = false>
__global__ void __launch_bounds__(kLinkBlock, LinkBlocks<T, I, REC>::v) k_link(Geom G, const typename Samp<T, I>::Field* __restrict__ F,
                                                     double tol, int max_iter, double* theta, double* tof,
                                                     double* hit, int32_t* status, int32_t* iters,
                                                     unsigned long long* counters, int* queue, int fan_rays,
                                                     const double* __restrict__ fan, RowRec rec, LinkRound rd,
                                                     int lanes) {
    __shared__ LinkState sh[kLinkBlock];
    // per-block tallies (status counts, RK4 steps): updated once per trace, so
    // they live in shared memory rather than in the step loop's registers
    __shared__ unsigned long long tally[5];
    if (threadIdx.x < 5) tally[threadIdx.x] = 0;
    __syncthreads();
    const int n_in = (ROUNDS && rd.aside_in) ? *rd.n_in : 0;
    LinkState& L = sh[threadIdx.x];
    auto C = make_cell<T, I>(G, F);
    TraceState<T> ts;
    typename std::conditional<REC, RecSink<T>, NoSink>::type ns;
    if constexpr (REC) {
        ns.cap = rec.cap;
        ns.nx = G.nx;
        ns.ny = G.ny;
        ns.begin(rec.runs);
    }
    bool active = false;
    // Only the first `lanes` lanes of each warp take pairs (all 32 unless the
    // problem has fewer pairs than the grid has lanes): a warp of few rays
    // steps at a lower latency than a full one. A round that resumes set-aside
    // pairs learns their number only here, so it spreads them itself.
    if (ROUNDS && rd.aside_in) {
        const long long warps = (long long)gridDim.x * (kLinkBlock / 32);
        lanes = (int)min(32LL, max(1LL, ((long long)n_in + warps - 1) / warps));
    }
    if ((threadIdx.x & 31) >= lanes) goto done;
    for (;;) {
        if (ROUNDS && !active && rd.aside_in) {
            // resume a pair set aside by the previous round (R12: refined first)
            const int slot = fetch_pair(queue);
            if (slot >= n_in) break;
            L = rd.aside_in[slot];
            if (rd.sub && L.fan_k0 >= -1 && L.n_eval == 2) subfan_apply(L, rd.sub + (size_t)slot * rd.sub_m, rd.sub_m, G.R);
            if constexpr (REC) ns.begin(rec.runs + (size_t)L.k * rec.cap);
            trace_begin(ts, G, L.xe, L.ye, L.next);
            active = true;
        }
        if (!active) {
            const int qslot = fetch_pair(queue);
            if (qslot >= G.n_pairs) break;
            const int k = queue_pair(G, qslot);
            LinkCtx X;
            if (!setup_pair(G, k, X)) {
                theta[k] = nan("");
                if (tof) tof[k] = nan("");
                if (hit) { hit[2 * k] = nan(""); hit[2 * k + 1] = nan(""); }
                if (iters) iters[k] = 0;
                if (status) status[k] = RT_RAY_BADINPUT;
                atomicAdd(&tally[3], 1ull);
                continue;
            }
            L.xe = X.xe; L.ye = X.ye; L.xr = X.xr; L.yr = X.yr;
            L.phi_e = X.phi_e; L.psi_r = X.psi_r; L.th_lo = X.th_lo; L.th_hi = X.th_hi;
            const double margin = fmax(G.ds / G.R, 1e-9);
            L.a_min = X.th_lo + margin;
            L.a_max = X.th_hi - margin;
            const double tin = theta[k];
            double th0 = isnan(tin) ? atan2(X.yr - X.ye, X.xr - X.xe) : tin;
            th0 = X.th_lo + mod_2pi(th0 - X.th_lo);
            th0 = fmin(fmax(th0, L.a_min), L.a_max);
            L.th0 = th0;
            L.next = th0;
            L.k = k;
            L.n_eval = 0;
            L.phase = 0;
            L.psi_at_lo = 0.0;
            L.best_d2 = CUDART_INF;
            L.fan_k0 = -2;
            if (fan_rays >= 2 && isnan(tin)) {
                int e, r;
                pair_of(G, k, e, r);
                fan_start(G, L, fan + (size_t)e * fan_rays, fan_rays);
            }
            if constexpr (REC) ns.begin(rec.runs + (size_t)k * rec.cap);
            trace_begin(ts, G, L.xe, L.ye, L.next);
            active = true;
        }
        bool ended = false;
#pragma unroll 1
        for (int u = 0; u < kLinkSteps; ++u)
            if (trace_step(C, G, ts, ns)) {
                ended = true;
                break;
            }
        if (ended) {
            const TraceOut o = trace_end(C, G, ts, L.xe, L.ye, L.xr, L.yr, ns);
            atomicAdd(&tally[4], (unsigned long long)o.steps);
            if (link_update(G, L, o, tol, max_iter, fan_rays >= 2 ? fan : nullptr, fan_rays)) {
                const int k = L.k;
                const int st = (L.best_d2 <= tol * tol) ? RT_RAY_OK
                               : (L.best_d2 == DBL_MAX ? RT_RAY_STEPCAP : RT_RAY_MAXITER);
                theta[k] = L.best_th;
                if (tof) tof[k] = L.best_T;
                if (hit) { hit[2 * k] = L.best_hx; hit[2 * k + 1] = L.best_hy; }
                if (iters) iters[k] = L.n_eval;
                if (status) status[k] = st;
                if constexpr (REC) {
                    // the slot holds the last trace: the linked ray when it reached tol
                    const bool last_is_best = st == RT_RAY_OK && ns.n <= rec.cap &&
                                              L.best_th == L.next && o.flags == 0;
                    rec.len[k] = last_is_best ? ns.n : -1;
                }
                atomicAdd(&tally[st == RT_RAY_OK ? 0 : (st == RT_RAY_MAXITER ? 1 : 2)], 1ull);
                active = false;
            } else if (ROUNDS && rd.stop_after && L.n_eval >= rd.stop_after) {
                rd.aside_out[atomicAdd(rd.n_out, 1)] = L;   // next angle already chosen
                active = false;
            } else {
                if constexpr (REC) ns.begin(rec.runs + (size_t)L.k * rec.cap);
                trace_begin(ts, G, L.xe, L.ye, L.next);
            }
        }
    }
done:
    __syncthreads();
    if (counters && threadIdx.x == 0) {
        if (tally[0]) atomicAdd(&counters[RT_RAY_OK], tally[0]);
        if (tally[1]) atomicAdd(&counters[RT_RAY_MAXITER], tally[1]);
        if (tally[2]) atomicAdd(&counters[RT_RAY_STEPCAP], tally[2]);
        if (tally[3]) atomicAdd(&counters[RT_RAY_BADINPUT], tally[3]);
        atomicAdd(&counters[7], tally[4]);
    }
}

// Blocks of a persistent launch on the current device: resident blocks per
// SM x SMs (cached per device and kernel slot).
template <typename K>
static int persistent_blocks(K kernel, int slot) {
    static std::atomic<int> cache[64][16];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int v = cache[dev][slot].load(std::memory_order_relaxed);
    if (!v) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kLinkBlock, 0);
        v = sms * (per_sm > 0 ? per_sm : 1);
        cache[dev][slot].store(v, std::memory_order_relaxed);
    }
    return v;
}

template <typename T, int I>
static void fan_impl(const Geom& G, const void* field, int fan_rays, double margin, double* fan,
                     const int* fan_need, unsigned long long* counters, cudaStream_t s) {
    const int nf = G.n_tx * fan_rays;
    k_fan<T, I><<<grid_for(nf), kBlock, 0, s>>>(G, (const typename Samp<T, I>::Field*)field, fan_rays, margin,
                                                fan_need, fan, counters);
}

Geom with_step(const Geom& G, double ds) {
    Geom F = G;
    F.ds = ds;
    F.dsf = (float)ds;
    F.Hf = (float)(ds / G.h);
    F.max_steps = (long long)std::ceil(8.0 * G.R / ds);
    F.max_steps_i = (int)F.max_steps;
    return F;
}

cudaError_t launch_fan(const Geom& G, double fan_ds, const void* field, int prec, int fan_rays, const double* theta,
                       double* fan, int* fan_need, unsigned long long* counters, cudaStream_t s) {
    if (G.n_pairs == 0 || fan_rays < 2) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(fan_need, 0, sizeof(int) * (size_t)G.n_tx, s);
    if (e != cudaSuccess) return e;
    k_fan_mark<<<grid_for(G.n_pairs), kBlock, 0, s>>>(G, theta, fan_need);
    const Geom F = fan_ds > 0.0 ? with_step(G, fan_ds) : G;
    const double margin = fmax(G.ds / G.R, 1e-9);
    const bool bs = G.interp == RT_BSPLINE;
    if (prec == RT_FP64) {
        if (bs) fan_impl<double, RT_BSPLINE>(F, field, fan_rays, margin, fan, fan_need, counters, s);
        else fan_impl<double, RT_BILINEAR>(F, field, fan_rays, margin, fan, fan_need, counters, s);
    } else {
        if (bs) fan_impl<float, RT_BSPLINE>(F, field, fan_rays, margin, fan, fan_need, counters, s);
        else fan_impl<float, RT_BILINEAR>(F, field, fan_rays, margin, fan, fan_need, counters, s);
    }
    return cudaGetLastError();
}

template <typename T, int I, bool REC = false, bool ROUNDS = false>
static void link_impl(const Geom& G, const void* field, double tol, int max_iter, double* theta, double* tof,
                      double* hit, int32_t* status, int32_t* iters, unsigned long long* counters, int* queue,
                      int fan_rays, double* fan, int slot, cudaStream_t s, const RowRec& rec = RowRec{},
                      const LinkRound& rd = LinkRound{}) {
    // With fewer pairs than the persistent grid has lanes, the pairs are
    // spread over all of its warps, ceil(pairs / warps) lanes each, rather
    // than packed 32 to a warp on a few SMs (the linking is per pair, so the
    // results do not depend on the lanes that run them).
    const int pb = persistent_blocks(k_link<T, I, REC, ROUNDS>, slot);
    const long long warps = (long long)pb * (kLinkBlock / 32);
    const long long pairs = G.n_pairs;   // an upper bound of the pairs a rounds launch resumes
    const int lanes = (int)std::min<long long>(32, std::max<long long>(1, (pairs + warps - 1) / warps));
    const long long per_block = (long long)lanes * (kLinkBlock / 32);
    const int nb = (int)std::min<long long>(pb, (pairs + per_block - 1) / per_block);
    k_link<T, I, REC, ROUNDS><<<nb, kLinkBlock, 0, s>>>(G, (const typename Samp<T, I>::Field*)field, tol, max_iter,
                                                        theta, tof, hit, status, iters, counters, queue, fan_rays,
                                                        fan, rec, rd, lanes);
}

size_t link_state_bytes() { return sizeof(LinkState); }

// R12 sub-fan rays of the pairs set aside after their second trace: item
// (slot, q) traces ray q of pair slot at the fan's step (Gf) and stores its
// misfit (NaN when it does not reach the ring, or for a pair that was not
// fan-started).
template <typename T, int I>
__global__ void __launch_bounds__(kBlock) k_subfan(Geom Gf, const typename Samp<T, I>::Field* __restrict__ F,
                                                   const LinkState* __restrict__ aside, const int* n_aside, int M,
                                                   double* sub, unsigned long long* counters) {
    const long long items = (long long)(*n_aside) * M;
    long long steps = 0;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const int slot = (int)(it / M), q = (int)(it - (long long)slot * M) + 1;
        const LinkState& L = aside[slot];
        double v = nan("");
        if (L.fan_k0 >= -1 && L.n_eval == 2) {
            auto C = make_cell<T, I>(Gf, F);
            NoSink ns;
            const TraceOut o = trace_ray<T>(C, Gf, L.xe, L.ye, subfan_theta(L, q, M), L.xe, L.ye, ns);
            if (!(o.flags & 3)) v = Gf.R * (mod_2pi(atan2(o.hy, o.hx) - L.phi_e) - L.psi_r);
            steps += o.steps;
        }
        sub[(size_t)slot * M + (q - 1)] = v;
    }
    __syncwarp();
    unsigned long long v = (unsigned long long)steps;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&counters[7], v);
}

template <typename T, int I, bool REC>
static cudaError_t link_rounds(const Geom& G, const void* field, double tol, int max_iter, double* theta,
                               double* tof, double* hit, int32_t* status, int32_t* iters,
                               unsigned long long* counters, int fan_rays, double fan_ds, double* fan, int slot,
                               const LinkWork& W, cudaStream_t s, const RowRec& rec) {
    // counters: queues of the two rounds, then the set-aside count. The first
    // round runs every pair's first two traces in one persistent launch (the
    // second traces fill the first ones' drain) and sets aside the pairs the
    // second trace left unlinked; after their sub-fan the second round resumes
    // them, spread over all warps.
    cudaError_t e = cudaMemsetAsync(W.ctr, 0, 3 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    LinkRound r1{2, W.aside, W.ctr + 2, nullptr, nullptr, nullptr, 0};
    link_impl<T, I, REC, true>(G, field, tol, max_iter, theta, tof, hit, status, iters, counters, W.ctr, fan_rays,
                               fan, slot, s, rec, r1);
    const Geom Gf = with_step(G, fan_ds > 0 ? fan_ds : G.ds);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_subfan<T, I><<<(unsigned)(sms > 0 ? sms * 8 : 1216), kBlock, 0, s>>>(
        Gf, (const typename Samp<T, I>::Field*)field, W.aside, W.ctr + 2, W.subfan, W.sub, counters);
    LinkRound r2{0, nullptr, nullptr, W.aside, W.ctr + 2, W.sub, W.subfan};
    link_impl<T, I, REC, true>(G, field, tol, max_iter, theta, tof, hit, status, iters, counters, W.ctr + 1,
                               fan_rays, fan, slot, s, rec, r2);
    return cudaGetLastError();
}

cudaError_t launch_link(const Geom& G, const void* field, int prec, double tol, int max_iter,
                        double* theta, double* tof, double* hit, int32_t* status, int32_t* iters,
                        unsigned long long* counters, int* queue, int fan_rays, double fan_ds, double* fan,
                        int* fan_need, cudaStream_t s, const RowRec* rec, const LinkWork* W) {
    if (G.n_pairs == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (fan_rays >= 2) {
        e = launch_fan(G, fan_ds, field, prec, fan_rays, theta, fan, fan_need, counters, s);
        if (e != cudaSuccess) return e;
    }
    if (W && W->subfan > 0) {   // R12 rounds: FP32-compensated, bilinear (checked by the caller)
        if (rec)
            return link_rounds<float, RT_BILINEAR, true>(G, field, tol, max_iter, theta, tof, hit, status, iters,
                                                         counters, fan_rays, fan_ds, fan, 12, *W, s, *rec);
        return link_rounds<float, RT_BILINEAR, false>(G, field, tol, max_iter, theta, tof, hit, status, iters,
                                                      counters, fan_rays, fan_ds, fan, 13, *W, s, RowRec{});
    }
    if (rec) {   // recording: FP32-compensated, bilinear (checked by the caller)
        link_impl<float, RT_BILINEAR, true>(G, field, tol, max_iter, theta, tof, hit, status, iters, counters, queue,
                                            fan_rays, fan, 11, s, *rec);
        return cudaGetLastError();
    }
    const bool bs = G.interp == RT_BSPLINE;
    if (prec == RT_FP64) {
        if (bs) link_impl<double, RT_BSPLINE>(G, field, tol, max_iter, theta, tof, hit, status, iters, counters, queue,
                                              fan_rays, fan, 9, s);
        else link_impl<double, RT_BILINEAR>(G, field, tol, max_iter, theta, tof, hit, status, iters, counters, queue,
                                            fan_rays, fan, 3, s);
    } else {
        if (bs) link_impl<float, RT_BSPLINE>(G, field, tol, max_iter, theta, tof, hit, status, iters, counters, queue,
                                             fan_rays, fan, 10, s);
        else link_impl<float, RT_BILINEAR>(G, field, tol, max_iter, theta, tof, hit, status, iters, counters, queue,
                                           fan_rays, fan, 4, s);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- A5: ToF at fixed angles

template <typename T, int I>
__global__ void __launch_bounds__(kBlock) k_tof(Geom G, const typename Samp<T, I>::Field* __restrict__ F,
                                                const double* theta, double* tof, double* hit) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G.n_pairs) return;
    LinkCtx L;
    if (!setup_pair(G, k, L)) {
        tof[k] = nan("");
        if (hit) { hit[2 * k] = nan(""); hit[2 * k + 1] = nan(""); }
        return;
    }
    auto C = make_cell<T, I>(G, F);
    NoSink ns;
    TraceOut o = trace_ray<T>(C, G, L.xe, L.ye, theta[k], L.xr, L.yr, ns);
    tof[k] = o.T;
    if (hit) { hit[2 * k] = o.hx; hit[2 * k + 1] = o.hy; }
}

cudaError_t launch_tof(const Geom& G, const void* field, int prec, const double* theta, double* tof,
                       double* hit, cudaStream_t s) {
    if (G.n_pairs == 0) return cudaSuccess;
    const int nb = grid_for(G.n_pairs);
    const bool bs = G.interp == RT_BSPLINE;
    if (prec == RT_FP64) {
        if (bs) k_tof<double, RT_BSPLINE><<<nb, kBlock, 0, s>>>(G, (const CellBS<double>*)field, theta, tof, hit);
        else k_tof<double, RT_BILINEAR><<<nb, kBlock, 0, s>>>(G, (const CellCoef<double>*)field, theta, tof, hit);
    } else {
        if (bs) k_tof<float, RT_BSPLINE><<<nb, kBlock, 0, s>>>(G, (const CellBS<float>*)field, theta, tof, hit);
        else k_tof<float, RT_BILINEAR><<<nb, kBlock, 0, s>>>(G, (const CellCoef<float>*)field, theta, tof, hit);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- A6: adjoint scatter

template <typename T, int I> struct AdjOf { using type = AdjSink<T>; };
template <typename T> struct AdjOf<T, RT_BSPLINE> { using type = AdjSinkBSp<T>; };

// Adjoint scatter: one thread per pair retraces the ray at its angle and
// scatters its weights, in the work-queue order (longest chords first,
// consecutive emitters at one ring offset, so a warp's rays have equal chords
// and run through nearby cells). A plain launch whose blocks retire as they
// finish measured faster than a persistent one with a work queue (26.1 vs
// 27.9 ms on the breast workload; 52.6 vs 61.0 ms with the B-spline).
template <typename T, int I>
__global__ void __launch_bounds__(kBlock, Occ<T, I>::blocks)
    k_adjoint(Geom G, const typename Samp<T, I>::Field* __restrict__ F, const double* theta, const double* g_tof,
                 const double* tof_ref, double* g) {
    const int slot = blockIdx.x * kBlock + threadIdx.x;
    if (slot >= G.n_pairs) return;
    const int k = queue_pair(G, slot);
    const double w = g_tof[k] - (tof_ref ? tof_ref[k] : 0.0);
    if (w == 0.0 || !isfinite(w)) return;
    LinkCtx X;
    if (!setup_pair(G, k, X)) return;
    auto C = make_cell<T, I>(G, F);
    typename AdjOf<T, I>::type sink;
    sink.g = g; sink.nx = G.nx; sink.ny = G.ny;
    sink.init();
    sink.w = (T)w;
    trace_ray<T>(C, G, X.xe, X.ye, theta[k], X.xr, X.yr, sink);
}

// g_c = -1000 * (L^T w) / c_mps^2 : s = 1000/c_mps (us/mm)
__global__ void k_adjoint_finish(double* g, const double* __restrict__ c_mps, int n) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double c = c_mps[k];
        g[k] = -1000.0 * g[k] / (c * c);
    }
}

// Adjoint from recorded rows: a warp per pair (in the work-queue order). The
// warp stages kRowSeg consecutive runs of its row in shared memory with
// coalesced loads (16-byte loads where every row starts on a 16-byte
// boundary), then lane l takes runs l, l + 32, ...: neighbouring lanes hold
// neighbouring cells of the ray, so the FP64 atomics of one instruction share
// sectors. Each weight is w * (FP32 run weight) in FP32, widened to FP64, as
// AdjSink::flush forms it. Pairs without a row are left to
// k_adjoint_unrecorded.
constexpr int kRowSeg = 128;                   // runs per warp segment (2560 bytes)

template <typename T>
__global__ void __launch_bounds__(kBlock) k_adjoint_rows(Geom G, const double* g_tof, const double* tof_ref,
                                                         double* g, RowRec rec, int vec) {
    __shared__ float4 seg_buf[kBlock / 32][kRowSeg * 20 / 16];
    const long long wid = (blockIdx.x * (long long)kBlock + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= G.n_pairs) return;
    const int k = queue_pair(G, (int)wid);
    const int n = rec.len[k];
    if (n <= 0) return;
    const double wd = g_tof[k] - (tof_ref ? tof_ref[k] : 0.0);
    if (wd == 0.0 || !isfinite(wd)) return;
    const T w = (T)wd;
    const rt_run* row = rec.runs + (size_t)k * rec.cap;
    const int nx = G.nx;
    float4* buf = seg_buf[threadIdx.x >> 5];
    const float* bw = reinterpret_cast<const float*>(buf);
    for (int base = 0; base < n; base += kRowSeg) {
        const int cnt = min(kRowSeg, n - base);
        __syncwarp();
        if (vec) {
            // the row's capacity is a multiple of 4 runs (80 bytes), so the
            // rounded-up segment stays inside the row
            const float4* src = reinterpret_cast<const float4*>(row + base);
            const int nv = (cnt * 20 + 15) >> 4;
            for (int q = lane; q < nv; q += 32) buf[q] = src[q];
        } else {
            const float* src = reinterpret_cast<const float*>(row + base);
            float* dst = reinterpret_cast<float*>(buf);
            for (int q = lane; q < cnt * 5; q += 32) dst[q] = src[q];
        }
        __syncwarp();
        for (int r = lane; r < cnt; r += 32) {
            // 5-word runs at a lane stride of 5 words: distinct banks
            double* p = g + __float_as_int(bw[r * 5]);
            atomicAdd(p, to_double(w * (T)bw[r * 5 + 1]));
            atomicAdd(p + 1, to_double(w * (T)bw[r * 5 + 2]));
            atomicAdd(p + nx, to_double(w * (T)bw[r * 5 + 3]));
            atomicAdd(p + nx + 1, to_double(w * (T)bw[r * 5 + 4]));
        }
    }
}

// The pairs whose row was not recorded (len < 0: a row longer than the
// capacity, or a pair the link did not finish on its reported ray), traced
// again at their angle, a thread per pair.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_adjoint_unrecorded(Geom G,
                                                               const typename Samp<T, RT_BILINEAR>::Field* __restrict__ F,
                                                               const double* theta, const double* g_tof,
                                                               const double* tof_ref, double* g, const int32_t* len) {
    const long long k = blockIdx.x * (long long)kBlock + threadIdx.x;
    if (k >= G.n_pairs || len[k] >= 0) return;
    const double wd = g_tof[k] - (tof_ref ? tof_ref[k] : 0.0);
    if (wd == 0.0 || !isfinite(wd)) return;
    LinkCtx X;
    if (!setup_pair(G, (int)k, X)) return;
    auto C = make_cell<T, RT_BILINEAR>(G, F);
    AdjSink<T> sink;
    sink.g = g; sink.nx = G.nx; sink.ny = G.ny;
    sink.init();
    sink.w = (T)wd;
    trace_ray<T>(C, G, X.xe, X.ye, theta[k], X.xr, X.yr, sink);
}

cudaError_t launch_adjoint_rows(const Geom& G, const void* field, const double* theta, const double* g_tof,
                                const double* tof_ref, const double* c_mps, const RowRec& rec, double* g_c,
                                cudaStream_t s) {
    const int n = G.nx * G.ny;
    cudaError_t e = cudaMemsetAsync(g_c, 0, sizeof(double) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    if (G.n_pairs > 0) {
        const long long threads = (long long)G.n_pairs * 32;
        const int vec = ((reinterpret_cast<uintptr_t>(rec.runs) & 15) == 0 && (rec.cap & 3) == 0) ? 1 : 0;
        k_adjoint_rows<float><<<(unsigned)((threads + kBlock - 1) / kBlock), kBlock, 0, s>>>(G, g_tof, tof_ref, g_c,
                                                                                          rec, vec);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_adjoint_unrecorded<float><<<(unsigned)((G.n_pairs + kBlock - 1) / kBlock), kBlock, 0, s>>>(
            G, (const typename Samp<float, RT_BILINEAR>::Field*)field, theta, g_tof, tof_ref, g_c, rec.len);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int blocks = (n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8;
    k_adjoint_finish<<<blocks, 256, 0, s>>>(g_c, c_mps, n);
    return cudaGetLastError();
}

template <typename T, int I>
static void adjoint_impl(const Geom& G, const void* field, const double* theta, const double* g_tof,
                         const double* tof_ref, double* g_c, cudaStream_t s) {
    k_adjoint<T, I><<<grid_for(G.n_pairs), kBlock, 0, s>>>(G, (const typename Samp<T, I>::Field*)field, theta,
                                                             g_tof, tof_ref, g_c);
}

cudaError_t launch_adjoint(const Geom& G, const void* field, int prec, const double* theta,
                           const double* g_tof, const double* tof_ref, const double* c_mps,
                           double* g_c, cudaStream_t s) {
    const int n = G.nx * G.ny;
    cudaError_t e = cudaMemsetAsync(g_c, 0, sizeof(double) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    if (G.n_pairs > 0) {
        const bool bs = G.interp == RT_BSPLINE;
        if (prec == RT_FP64) {
            if (bs) adjoint_impl<double, RT_BSPLINE>(G, field, theta, g_tof, tof_ref, g_c, s);
            else adjoint_impl<double, RT_BILINEAR>(G, field, theta, g_tof, tof_ref, g_c, s);
        } else {
            if (bs) adjoint_impl<float, RT_BSPLINE>(G, field, theta, g_tof, tof_ref, g_c, s);
            else adjoint_impl<float, RT_BILINEAR>(G, field, theta, g_tof, tof_ref, g_c, s);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // B-spline: the scatter ran over the slowness coefficients; P^-T maps it to the nodes
    if (G.interp == RT_BSPLINE) {
        e = launch_bs_filter(g_c, G.nx, G.ny, 1, true, s);
        if (e != cudaSuccess) return e;
    }
    const int blocks = (n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8;
    k_adjoint_finish<<<blocks, 256, 0, s>>>(g_c, c_mps, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- A5b: system-matrix rows

// Counting pass: 4 entries per cell visit. Filling pass: writes them.
template <typename T>
struct RowSink {
    int nx, ny;
    int32_t* col;
    double* val;
    int64_t pos;       // next write position (fill) / count
    int64_t end;       // fill: end of this row (writes never pass it)
    bool fill;
    CellAcc<T> acc;
    __device__ __forceinline__ void flush() {
        if (acc.ai == INT_MIN) return;
        if (fill && pos + 4 <= end) {
            double w00, w10, w01, w11;
            acc.node_weights(w00, w10, w01, w11);
            const int i = min(max(acc.ai, 0), nx - 2), j = min(max(acc.aj, 0), ny - 2);
            const int32_t n0 = j * nx + i;
            col[pos] = n0;          val[pos] = w00;
            col[pos + 1] = n0 + 1;  val[pos + 1] = w10;
            col[pos + 2] = n0 + nx; val[pos + 2] = w01;
            col[pos + 3] = n0 + nx + 1; val[pos + 3] = w11;
        }
        pos += 4;
    }
    __device__ __forceinline__ void add(int ci, int cj, T tx, T ty, T a) {
        if (ci != acc.ai || cj != acc.aj) {
            flush();
            acc.reset();
            acc.ai = ci;
            acc.aj = cj;
        }
        acc.W += a;
        acc.Wx += a * tx;
        acc.Wy += a * ty;
        acc.Wxy += a * tx * ty;
    }
    __device__ __forceinline__ void finish() { flush(); }
};

template <typename T, int I> struct RowsOf { using type = RowSink<T>; };
template <typename T> struct RowsOf<T, RT_BSPLINE> { using type = RowSinkBSp<T>; };

template <typename T, int I>
__global__ void __launch_bounds__(kBlock) k_rows(Geom G, const typename Samp<T, I>::Field* __restrict__ F,
                                                 const double* theta, int64_t* row_ptr, int32_t* col,
                                                 double* val, bool fill) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G.n_pairs) return;
    LinkCtx L;
    typename RowsOf<T, I>::type sink;
    sink.nx = G.nx; sink.ny = G.ny; sink.col = col; sink.val = val; sink.fill = fill;
    sink.pos = fill ? row_ptr[k] : 0;
    sink.end = fill ? row_ptr[k + 1] : 0;
    sink.acc.reset();
    if (setup_pair(G, k, L)) {
        auto C = make_cell<T, I>(G, F);
        trace_ray<T>(C, G, L.xe, L.ye, theta[k], L.xr, L.yr, sink);
    }
    if (!fill) row_ptr[k + 1] = sink.pos;
}

cudaError_t launch_rows(const Geom& G, const void* field, int prec, const double* theta, int64_t* row_ptr,
                        int32_t* col, double* val, bool fill, cudaStream_t s) {
    if (G.n_pairs == 0) return cudaSuccess;
    const int nb = grid_for(G.n_pairs);
    const bool bs = G.interp == RT_BSPLINE;
    if (prec == RT_FP64) {
        if (bs) k_rows<double, RT_BSPLINE><<<nb, kBlock, 0, s>>>(G, (const CellBS<double>*)field, theta, row_ptr, col,
                                                                 val, fill);
        else k_rows<double, RT_BILINEAR><<<nb, kBlock, 0, s>>>(G, (const CellCoef<double>*)field, theta, row_ptr, col,
                                                               val, fill);
    } else {
        if (bs) k_rows<float, RT_BSPLINE><<<nb, kBlock, 0, s>>>(G, (const CellBS<float>*)field, theta, row_ptr, col,
                                                                val, fill);
        else k_rows<float, RT_BILINEAR><<<nb, kBlock, 0, s>>>(G, (const CellCoef<float>*)field, theta, row_ptr, col,
                                                              val, fill);
    }
    return cudaGetLastError();
}

// In-place inclusive scan of row_ptr[1..n] (row_ptr[0] = 0 set by the caller).
// With tmp == nullptr only reports the workspace size.
cudaError_t launch_scan(int64_t* row_ptr, int n, void* tmp, size_t* tmp_bytes, cudaStream_t s) {
    return cub::DeviceScan::InclusiveSum(tmp, *tmp_bytes, row_ptr + 1, row_ptr + 1, n, s);
}

}  // namespace rt
