// rt_ray.cu — kernels of the ToF path: field packing, shooting-method linking
// with the fused travel time, travel time at fixed angles, the adjoint scatter
// and the explicit system-matrix rows.
#include <cfloat>
#include <climits>
#include <cstdint>

#include <cub/device/device_scan.cuh>
#include <math_constants.h>

#include "rt_internal.h"
#include "rt_trace.cuh"

namespace rt {

constexpr double kPi = 3.141592653589793;
constexpr int kBlock = 128;

static int grid_for(int n) { return (n + kBlock - 1) / kBlock; }

size_t node_bytes(int prec) { return prec == RT_FP64 ? sizeof(CellCoef<double>) : sizeof(CellCoef<float>); }

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

__device__ __forceinline__ double mod_2pi(double a) { return a - 2.0 * kPi * floor(a / (2.0 * kPi)); }

struct LinkCtx {
    double xe, ye, xr, yr, phi_e, psi_r, th_lo, th_hi;
};

__device__ __forceinline__ bool on_ring(double x, double y, double R) {
    return fabs(sqrt(x * x + y * y) - R) <= 1e-9 * R;
}

// Resolves pair k; false if the pair or its transducers are invalid.
__device__ __forceinline__ bool setup_pair(const Geom& G, int k, LinkCtx& L) {
    int e, r;
    pair_of(G, k, e, r);
    if (*G.bad_field || e < 0 || e >= G.n_tx || r < 0 || r >= G.n_tx || e == r) return false;
    L.xe = G.tx[2 * e]; L.ye = G.tx[2 * e + 1];
    L.xr = G.tx[2 * r]; L.yr = G.tx[2 * r + 1];
    if (!on_ring(L.xe, L.ye, G.R) || !on_ring(L.xr, L.yr, G.R)) return false;
    L.phi_e = atan2(L.ye, L.xe);
    L.psi_r = mod_2pi(atan2(L.yr, L.xr) - L.phi_e);
    L.th_lo = L.phi_e + 0.5 * kPi;
    L.th_hi = L.phi_e + 1.5 * kPi;
    return true;
}

// Per-lane linking state of the persistent kernel, kept in shared memory so
// that only the trace state occupies registers in the marching loop.
struct LinkState {
    double xe, ye, xr, yr, phi_e, psi_r, th_lo, th_hi;
    double a_min, a_max;
    double th0, m0, mp;              // first angle, its misfit, the probe's misfit
    double best_th, best_T, best_hx, best_hy, best_dist;
    double ta, fa, tb, fb;           // bracket
    double prev_th, prev_m, cur_th, cur_m;
    double psi_at_lo, next;
    int k, n_eval, phase, last, e0_flagged;
};

__device__ __forceinline__ void br_insert(LinkState& L, double t, double m) {
    if (!(t > fmin(L.ta, L.tb) && t < fmax(L.ta, L.tb))) return;
    if (m < 0) {
        L.ta = t; L.fa = m;
        if (L.last == -1) L.fb *= 0.5;
        L.last = -1;
    } else {
        L.tb = t; L.fb = m;
        if (L.last == 1) L.fa *= 0.5;
        L.last = 1;
    }
}

// Misfit of an ended trace (same rule as evaluate()).
__device__ __forceinline__ void misfit_of(const Geom& G, const LinkState& L, const TraceOut& o, double theta,
                                          double& m, double& dist) {
    const double dx = o.hx - L.xr, dy = o.hy - L.yr;
    dist = sqrt(dx * dx + dy * dy);
    double psi;
    if (o.flags & 3) {
        psi = (theta - L.th_lo < L.th_hi - theta) ? L.psi_at_lo : 2.0 * kPi - L.psi_at_lo;
        dist = DBL_MAX;
    } else {
        psi = mod_2pi(atan2(o.hy, o.hx) - L.phi_e);
    }
    m = G.R * (psi - L.psi_r);
}

// Next angle inside the bracket: the secant of (prev, cur) if it falls inside,
// else the Regula-Falsi point of the bracket.
__device__ __forceinline__ double next_angle(const LinkState& L, double cand) {
    if (!(isfinite(cand) && cand > fmin(L.ta, L.tb) && cand < fmax(L.ta, L.tb)))
        cand = (L.ta * L.fb - L.tb * L.fa) / (L.fb - L.fa);
    return cand;
}

// Linking update after the trace of L.next ended (the same decisions as
// link_pair). Returns true when the pair is finished.
__device__ bool link_update(const Geom& G, LinkState& L, const TraceOut& o, double tol, int max_iter) {
    const double theta = L.next;
    double m, dist;
    misfit_of(G, L, o, theta, m, dist);
    ++L.n_eval;
    if (dist < L.best_dist) {
        L.best_th = theta; L.best_T = o.T; L.best_hx = o.hx; L.best_hy = o.hy; L.best_dist = dist;
    }
    if (dist <= tol) return true;
    if (L.phase == 0) {
        L.m0 = m;
        L.e0_flagged = (o.flags & 3) != 0;
        if (L.n_eval >= max_iter) return true;
        L.phase = 1;
        L.next = L.a_min;   // orientation probe next to the fan's lower end
        return false;
    }
    if (L.phase == 1) {
        const bool ccw = (m / G.R + L.psi_r) < kPi;
        L.psi_at_lo = ccw ? 0.0 : 2.0 * kPi;
        if (L.e0_flagged) {
            const double psi0 = (L.th0 - L.th_lo < L.th_hi - L.th0) ? L.psi_at_lo : 2.0 * kPi - L.psi_at_lo;
            L.m0 = G.R * (psi0 - L.psi_r);
        }
        const double mp = (o.flags & 3) ? G.R * (L.psi_at_lo - L.psi_r) : m;
        L.ta = ccw ? L.th_lo : L.th_hi; L.fa = -G.R * L.psi_r;
        L.tb = ccw ? L.th_hi : L.th_lo; L.fb = G.R * (2.0 * kPi - L.psi_r);
        L.last = 0;
        br_insert(L, theta, mp);
        br_insert(L, L.th0, L.m0);
        L.last = 0;
        L.prev_th = L.cur_th = L.th0;
        L.prev_m = L.cur_m = L.m0;
        if (L.n_eval >= max_iter) return true;
        L.phase = 2;
        L.next = next_angle(L, L.th0 - L.m0 / (ccw ? 2.0 * G.R : -2.0 * G.R));
        return false;
    }
    br_insert(L, theta, m);
    L.prev_th = L.cur_th; L.prev_m = L.cur_m;
    L.cur_th = theta; L.cur_m = m;
    if (L.n_eval >= max_iter) return true;
    const double den = L.cur_m - L.prev_m;
    const double cand = (den != 0.0) ? L.cur_th - L.cur_m * (L.cur_th - L.prev_th) / den : nan("");
    L.next = next_angle(L, cand);
    return false;
}

// ---------------------------------------------------------------- fan start

// Cold-start prediction from a fan of K rays per emitter at evenly spaced
// angles over the inward fan (an option; fan_rays = 0 keeps the paper's
// straight-line start, Sec. 3.4.1). psi = interception angle counter-clockwise
// from the emitter, NaN when the ray has no interception.
__device__ __forceinline__ double fan_theta(double a_min, double step, int k) { return a_min + k * step; }

__global__ void k_fan_mark(Geom G, const double* __restrict__ theta, int* need) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G.n_pairs) return;
    int e, r;
    pair_of(G, k, e, r);
    if (e >= 0 && e < G.n_tx && isnan(theta[k])) need[e] = 1;
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_fan(Geom G, const CellCoef<T>* __restrict__ F, int K,
                                                const int* __restrict__ need, double* fan,
                                                unsigned long long* counters) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    const int e = id / K, k = id - e * K;
    long long steps = 0;
    if (id < G.n_tx * K && need[e] && !*G.bad_field) {
        const double xe = G.tx[2 * e], ye = G.tx[2 * e + 1];
        const double phi_e = atan2(ye, xe);
        const double margin = fmax(G.ds / G.R, 1e-9);
        const double a_min = phi_e + 0.5 * kPi + margin, a_max = phi_e + 1.5 * kPi - margin;
        const double step = (a_max - a_min) / (K - 1);
        Cell<T> C;
        C.F = F; C.nx = G.nx; C.ny = G.ny; C.pi = INT_MIN; C.pj = INT_MIN;
        NoSink ns;
        const TraceOut o = trace_ray<T>(C, G, xe, ye, fan_theta(a_min, step, k), xe, ye, ns);
        fan[id] = (o.flags & 3) ? nan("") : mod_2pi(atan2(o.hy, o.hx) - phi_e);
        steps = o.steps;
    }
    // every thread of the block reaches this point
    __syncwarp();
    unsigned long long v = (unsigned long long)steps;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&counters[7], v);
}

// Fan start of a cold pair (the rule of the CPU reference, written so that the
// per-ray scan issues no FP64 instruction): the interval of the sequence (fan
// end, rays 0..K-1, fan end) where psi crosses psi_r whose middle lies closest
// to the straight-line angle in fan-index units; first angle from the inverse
// cubic of the four rays around it (when monotone and inside), else linear.
// psi values are non-negative, so "psi < psi_r" is the signed compare of their
// IEEE bit patterns; NaN (no interception) has the largest patterns.
__device__ void fan_start(const Geom& G, LinkState& L, const double* __restrict__ psi, int K) {
    const bool ccw = isnan(psi[0]) ? true : (psi[0] < kPi);
    L.psi_at_lo = ccw ? 0.0 : 2.0 * kPi;
    const double psi_hi_end = 2.0 * kPi - L.psi_at_lo;
    const double step = (L.a_max - L.a_min) / (K - 1);
    double th_s = atan2(L.yr - L.ye, L.xr - L.xe);
    th_s = L.th_lo + mod_2pi(th_s - L.th_lo);
    const double u_s = (th_s - L.a_min) / step;
    const long long* pb = reinterpret_cast<const long long*>(psi);
    const long long b_r = __double_as_longlong(L.psi_r);
    const long long b_lo = __double_as_longlong(L.psi_at_lo), b_hi = __double_as_longlong(psi_hi_end);
    const long long b_nan = 0x7ff0000000000000ll;
    bool neg_prev = b_lo < b_r;
    int jsel = K + 1;
    double best_gap = CUDART_INF;
    for (int j = 1; j <= K + 1; ++j) {
        long long b;
        if (j <= K) {
            const int k = j - 1;
            b = pb[k];
            if (b > b_nan) b = (k < K / 2) ? b_lo : b_hi;
        } else {
            b = b_hi;
        }
        const bool neg = b < b_r;
        if (neg != neg_prev) {
            const double gap = fabs((j - 1.5) - u_s);
            if (gap < best_gap) { best_gap = gap; jsel = j; }
        }
        neg_prev = neg;
    }
    const double R = G.R;
    double t0, t1, p0, p1;
    {
        const int ja = jsel - 1, jb = jsel;
        if (ja == 0) { t0 = L.th_lo; p0 = L.psi_at_lo; }
        else { const int k = ja - 1; t0 = fan_theta(L.a_min, step, k); p0 = psi[k]; if (isnan(p0)) p0 = (k < K / 2) ? L.psi_at_lo : psi_hi_end; }
        if (jb == K + 1) { t1 = L.th_hi; p1 = psi_hi_end; }
        else { const int k = jb - 1; t1 = fan_theta(L.a_min, step, k); p1 = psi[k]; if (isnan(p1)) p1 = (k < K / 2) ? L.psi_at_lo : psi_hi_end; }
    }
    const double m0 = R * (p0 - L.psi_r), m1 = R * (p1 - L.psi_r);
    if (m0 < 0) { L.ta = t0; L.fa = m0; L.tb = t1; L.fb = m1; }
    else { L.ta = t1; L.fa = m1; L.tb = t0; L.fb = m0; }
    L.last = 0;
    double th0 = t0 - m0 * (t1 - t0) / (m1 - m0);
    const int k0 = jsel - 2;
    if (k0 >= 1 && k0 + 2 <= K - 1) {
        double tt[4], mm[4];
        bool ok = true;
        for (int q = 0; q < 4; ++q) {
            const int k = k0 - 1 + q;
            const double pk = psi[k];
            if (isnan(pk)) ok = false;
            tt[q] = fan_theta(L.a_min, step, k);
            mm[q] = R * (pk - L.psi_r);
        }
        for (int q = 0; q < 3 && ok; ++q)
            if (!((mm[q + 1] - mm[q]) * (mm[2] - mm[1]) > 0)) ok = false;
        if (ok) {
            double v = 0.0;
            for (int a = 0; a < 4; ++a) {
                double l = 1.0;
                for (int b = 0; b < 4; ++b)
                    if (b != a) l *= (0.0 - mm[b]) / (mm[a] - mm[b]);
                v += l * tt[a];
            }
            if (v > fmin(t0, t1) && v < fmax(t0, t1)) th0 = v;
        }
    }
    if (!(th0 > fmin(L.ta, L.tb) && th0 < fmax(L.ta, L.tb))) th0 = 0.5 * (L.ta + L.tb);
    const bool first = fabs(m0) <= fabs(m1);
    L.cur_th = L.prev_th = first ? t0 : t1;
    L.cur_m = L.prev_m = first ? m0 : m1;
    L.th0 = th0;
    L.next = th0;
    L.phase = 2;
}

// Work order of the persistent kernel. For the all-pairs list, queue slot q
// serves ring offsets o = r - e (mod N) from the longest chord (o = N/2) down to
// the shortest (o = 1, N-1), N emitters per offset, so the launch's tail is
// made of the shortest rays; the pair's own index k is returned. Explicit pair
// lists are served in their order.
__device__ __forceinline__ int queue_pair(const Geom& G, int q) {
    if (G.pairs) return q;
    const int N = G.n_tx;
    const int t = q / N, e = q - t * N;
    const int h = (N + 1) / 2;
    const int o = (t & 1) ? h - (t + 1) / 2 : h + t / 2;
    const int r = (e + o) % N;
    return e * (N - 1) + r - (r > e);
}

// Warp-aggregated fetch of the next pair index from the work queue.
__device__ __forceinline__ int fetch_pair(int* queue) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(queue, __popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}

constexpr int kLinkBlock = 128;
// Resident blocks per SM asked of the compiler: FP32 at <= 85 registers
// (6 blocks, 24 warps), FP64 unconstrained.
template <typename T> struct LinkOcc { static constexpr int blocks = 1; };
template <> struct LinkOcc<float> { static constexpr int blocks = 6; };

// Persistent linking kernel: each lane takes pairs from the queue, advances
// its own trace one RK4 step per loop iteration, and updates the linking
// state when a trace ends, so lanes never wait for other lanes' pairs.
template <typename T>
__global__ void __launch_bounds__(kLinkBlock, LinkOcc<T>::blocks) k_link(Geom G, const typename NodeT<T>::type* __restrict__ F,
                                                     double tol, int max_iter, double* theta, double* tof,
                                                     double* hit, int32_t* status, int32_t* iters,
                                                     unsigned long long* counters, int* queue, int fan_rays,
                                                     const double* __restrict__ fan) {
    __shared__ LinkState sh[kLinkBlock];
    LinkState& L = sh[threadIdx.x];
    Cell<T> C;
    C.F = F; C.nx = G.nx; C.ny = G.ny; C.pi = INT_MIN; C.pj = INT_MIN;
    TraceState<T> ts;
    NoSink ns;
    long long steps = 0;
    unsigned n_ok = 0, n_max = 0, n_cap = 0, n_bad = 0;
    bool active = false;
    for (;;) {
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
                ++n_bad;
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
            L.best_dist = CUDART_INF;
            if (fan_rays >= 2 && isnan(tin)) {
                int e, r;
                pair_of(G, k, e, r);
                fan_start(G, L, fan + (size_t)e * fan_rays, fan_rays);
            }
            trace_begin(ts, G, L.xe, L.ye, L.next);
            active = true;
        }
        if (trace_step(C, G, ts, ns)) {
            const TraceOut o = trace_end(C, G, ts, L.xe, L.ye, L.xr, L.yr, ns);
            steps += o.steps;
            if (link_update(G, L, o, tol, max_iter)) {
                const int k = L.k;
                const int st = (L.best_dist <= tol) ? RT_RAY_OK
                               : (L.best_dist == DBL_MAX ? RT_RAY_STEPCAP : RT_RAY_MAXITER);
                theta[k] = L.best_th;
                if (tof) tof[k] = L.best_T;
                if (hit) { hit[2 * k] = L.best_hx; hit[2 * k + 1] = L.best_hy; }
                if (iters) iters[k] = L.n_eval;
                if (status) status[k] = st;
                n_ok += st == RT_RAY_OK;
                n_max += st == RT_RAY_MAXITER;
                n_cap += st == RT_RAY_STEPCAP;
                active = false;
            } else {
                trace_begin(ts, G, L.xe, L.ye, L.next);
            }
        }
    }
    if (counters) {
        __syncwarp();
        unsigned long long v[5] = {n_ok, n_max, n_cap, n_bad, (unsigned long long)steps};
#pragma unroll
        for (int q = 0; q < 5; ++q)
            for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
        if ((threadIdx.x & 31) == 0) {
            if (v[0]) atomicAdd(&counters[RT_RAY_OK], v[0]);
            if (v[1]) atomicAdd(&counters[RT_RAY_MAXITER], v[1]);
            if (v[2]) atomicAdd(&counters[RT_RAY_STEPCAP], v[2]);
            if (v[3]) atomicAdd(&counters[RT_RAY_BADINPUT], v[3]);
            atomicAdd(&counters[7], v[4]);
        }
    }
}

// Blocks of a persistent launch: resident blocks per SM x SMs (cached per slot).
template <typename K>
static int persistent_blocks(K kernel, int slot) {
    static int cache[8] = {0};
    if (!cache[slot]) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kLinkBlock, 0);
        cache[slot] = sms * (per_sm > 0 ? per_sm : 1);
    }
    return cache[slot];
}

cudaError_t launch_link(const Geom& G, const void* field, int prec, double tol, int max_iter,
                        double* theta, double* tof, double* hit, int32_t* status, int32_t* iters,
                        unsigned long long* counters, int* queue, int fan_rays, double* fan,
                        int* fan_need, cudaStream_t s) {
    if (G.n_pairs == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (fan_rays >= 2) {
        e = cudaMemsetAsync(fan_need, 0, sizeof(int) * (size_t)G.n_tx, s);
        if (e != cudaSuccess) return e;
        k_fan_mark<<<grid_for(G.n_pairs), kBlock, 0, s>>>(G, theta, fan_need);
        const int nf = G.n_tx * fan_rays;
        if (prec == RT_FP64)
            k_fan<double><<<grid_for(nf), kBlock, 0, s>>>(G, (const CellCoef<double>*)field, fan_rays, fan_need, fan,
                                                          counters);
        else
            k_fan<float><<<grid_for(nf), kBlock, 0, s>>>(G, (const CellCoef<float>*)field, fan_rays, fan_need, fan,
                                                         counters);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (prec == RT_FP64) {
        const int nb = min(persistent_blocks(k_link<double>, 3), (G.n_pairs + kLinkBlock - 1) / kLinkBlock);
        k_link<double><<<nb, kLinkBlock, 0, s>>>(G, (const CellCoef<double>*)field, tol, max_iter, theta, tof, hit,
                                                 status, iters, counters, queue, fan_rays, fan);
    } else {
        const int nb = min(persistent_blocks(k_link<float>, 4), (G.n_pairs + kLinkBlock - 1) / kLinkBlock);
        k_link<float><<<nb, kLinkBlock, 0, s>>>(G, (const CellCoef<float>*)field, tol, max_iter, theta, tof, hit,
                                                status, iters, counters, queue, fan_rays, fan);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- A5: ToF at fixed angles

template <typename T>
__global__ void __launch_bounds__(kBlock) k_tof(Geom G, const typename NodeT<T>::type* __restrict__ F,
                                                const double* theta, double* tof, double* hit) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G.n_pairs) return;
    LinkCtx L;
    if (!setup_pair(G, k, L)) {
        tof[k] = nan("");
        if (hit) { hit[2 * k] = nan(""); hit[2 * k + 1] = nan(""); }
        return;
    }
    Cell<T> C;
    C.F = F; C.nx = G.nx; C.ny = G.ny; C.pi = INT_MIN; C.pj = INT_MIN;
    NoSink ns;
    TraceOut o = trace_ray<T>(C, G, L.xe, L.ye, theta[k], L.xr, L.yr, ns);
    tof[k] = o.T;
    if (hit) { hit[2 * k] = o.hx; hit[2 * k + 1] = o.hy; }
}

cudaError_t launch_tof(const Geom& G, const void* field, int prec, const double* theta, double* tof,
                       double* hit, cudaStream_t s) {
    if (G.n_pairs == 0) return cudaSuccess;
    if (prec == RT_FP64)
        k_tof<double><<<grid_for(G.n_pairs), kBlock, 0, s>>>(G, (const CellCoef<double>*)field, theta, tof, hit);
    else
        k_tof<float><<<grid_for(G.n_pairs), kBlock, 0, s>>>(G, (const CellCoef<float>*)field, theta, tof, hit);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- A6: adjoint scatter

// Scatters w * alpha_m * phi_j(x_m) into g (FP64 atomics), one flush of the
// four nodes per run of consecutive points in one cell. The node weights are
// formed in the marching precision and widened exactly to FP64 for the atomic.
template <typename T>
struct AdjSink {
    double* g;
    T w;
    int nx, ny;
    CellAcc<T> acc;
    __device__ __forceinline__ void flush() {
        if (acc.ai == INT_MIN) return;
        const T w11 = acc.Wxy, w10 = acc.Wx - acc.Wxy, w01 = acc.Wy - acc.Wxy;
        const T w00 = (acc.W - acc.Wx) - w01;
        const int i = min(max(acc.ai, 0), nx - 2), j = min(max(acc.aj, 0), ny - 2);
        double* p = g + (size_t)j * nx + i;
        atomicAdd(p, to_double(w * w00));
        atomicAdd(p + 1, to_double(w * w10));
        atomicAdd(p + nx, to_double(w * w01));
        atomicAdd(p + nx + 1, to_double(w * w11));
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
    __device__ __forceinline__ void finish() {
        flush();
        acc.reset();
    }
};

struct PairEnds {
    double xe, ye, xr, yr;
};

// Persistent adjoint: each lane takes pairs from the queue (longest chords
// first), retraces the ray at its angle and scatters its weights.
template <typename T>
__global__ void __launch_bounds__(kLinkBlock, LinkOcc<T>::blocks)
    k_adjoint(Geom G, const CellCoef<T>* __restrict__ F, const double* theta, const double* g_tof,
              const double* tof_ref, double* g, int* queue) {
    __shared__ PairEnds sh[kLinkBlock];
    PairEnds& E = sh[threadIdx.x];
    Cell<T> C;
    C.F = F; C.nx = G.nx; C.ny = G.ny; C.pi = INT_MIN; C.pj = INT_MIN;
    TraceState<T> ts;
    AdjSink<T> sink;
    sink.g = g; sink.nx = G.nx; sink.ny = G.ny;
    sink.acc.reset();
    bool active = false;
    for (;;) {
        if (!active) {
            const int qslot = fetch_pair(queue);
            if (qslot >= G.n_pairs) break;
            const int k = queue_pair(G, qslot);
            const double w = g_tof[k] - (tof_ref ? tof_ref[k] : 0.0);
            if (w == 0.0 || !isfinite(w)) continue;
            LinkCtx X;
            if (!setup_pair(G, k, X)) continue;
            E.xe = X.xe; E.ye = X.ye; E.xr = X.xr; E.yr = X.yr;
            sink.w = (T)w;
            trace_begin(ts, G, X.xe, X.ye, theta[k]);
            active = true;
        }
        if (trace_step(C, G, ts, sink)) {
            trace_end(C, G, ts, E.xe, E.ye, E.xr, E.yr, sink);
            active = false;
        }
    }
}

// g_c = -1000 * (L^T w) / c_mps^2 : s = 1000/c_mps (us/mm)
__global__ void k_adjoint_finish(double* g, const double* __restrict__ c_mps, int n) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double c = c_mps[k];
        g[k] = -1000.0 * g[k] / (c * c);
    }
}

cudaError_t launch_adjoint(const Geom& G, const void* field, int prec, const double* theta,
                           const double* g_tof, const double* tof_ref, const double* c_mps,
                           double* g_c, int* queue, cudaStream_t s) {
    const int n = G.nx * G.ny;
    cudaError_t e = cudaMemsetAsync(g_c, 0, sizeof(double) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    if (G.n_pairs > 0) {
        e = cudaMemsetAsync(queue, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
        if (prec == RT_FP64) {
            const int nb = min(persistent_blocks(k_adjoint<double>, 1), (G.n_pairs + kLinkBlock - 1) / kLinkBlock);
            k_adjoint<double><<<nb, kLinkBlock, 0, s>>>(G, (const CellCoef<double>*)field, theta, g_tof, tof_ref,
                                                        g_c, queue);
        } else {
            const int nb = min(persistent_blocks(k_adjoint<float>, 2), (G.n_pairs + kLinkBlock - 1) / kLinkBlock);
            k_adjoint<float><<<nb, kLinkBlock, 0, s>>>(G, (const CellCoef<float>*)field, theta, g_tof, tof_ref,
                                                       g_c, queue);
        }
        e = cudaGetLastError();
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

template <typename T>
__global__ void __launch_bounds__(kBlock) k_rows(Geom G, const typename NodeT<T>::type* __restrict__ F,
                                                 const double* theta, int64_t* row_ptr, int32_t* col,
                                                 double* val, bool fill) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G.n_pairs) return;
    LinkCtx L;
    RowSink<T> sink;
    sink.nx = G.nx; sink.ny = G.ny; sink.col = col; sink.val = val; sink.fill = fill;
    sink.pos = fill ? row_ptr[k] : 0;
    sink.end = fill ? row_ptr[k + 1] : 0;
    sink.acc.reset();
    if (setup_pair(G, k, L)) {
        Cell<T> C;
        C.F = F; C.nx = G.nx; C.ny = G.ny; C.pi = INT_MIN; C.pj = INT_MIN;
        trace_ray<T>(C, G, L.xe, L.ye, theta[k], L.xr, L.yr, sink);
    }
    if (!fill) row_ptr[k + 1] = sink.pos;
}

cudaError_t launch_rows(const Geom& G, const void* field, int prec, const double* theta, int64_t* row_ptr,
                        int32_t* col, double* val, bool fill, cudaStream_t s) {
    if (G.n_pairs == 0) return cudaSuccess;
    if (prec == RT_FP64)
        k_rows<double><<<grid_for(G.n_pairs), kBlock, 0, s>>>(G, (const CellCoef<double>*)field, theta, row_ptr, col, val,
                                                              fill);
    else
        k_rows<float><<<grid_for(G.n_pairs), kBlock, 0, s>>>(G, (const CellCoef<float>*)field, theta, row_ptr, col,
                                                             val, fill);
    return cudaGetLastError();
}

// In-place inclusive scan of row_ptr[1..n] (row_ptr[0] = 0 set by the caller).
// With tmp == nullptr only reports the workspace size.
cudaError_t launch_scan(int64_t* row_ptr, int n, void* tmp, size_t* tmp_bytes, cudaStream_t s) {
    return cub::DeviceScan::InclusiveSum(tmp, *tmp_bytes, row_ptr + 1, row_ptr + 1, n, s);
}

}  // namespace rt
