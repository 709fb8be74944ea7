// rt_batch.cu — many ToF problems (uneven grids and rings) in one persistent
// launch: every pair of every instance is linked and, when the instance has
// measured travel times, retraced right away by the same lane with the
// adjoint weight w = T - T_ref (the gradient of 0.5*||T - T_ref||^2), so the
// forward and the adjoint share one launch and one tail.
#include <algorithm>
#include <climits>
#include <atomic>
#include <cstring>
#include <string>
#include <vector>

#include "rt_internal.h"
#include "rt_link.cuh"
#include "rt_trace.cuh"

namespace rt {

struct InstDesc {
    Geom G;
    const void* field;
    const double* fan;      // [n_tx * fan_rays] or null
    double* theta;
    double* tof;
    double* hit;
    int32_t* status;
    int32_t* iters;
    const double* tof_ref;  // null: no adjoint for this instance
    double* g;              // adjoint accumulator (then finished in place)
    const double* c_mps;    // sound speed, for the final chain rule
    long long pair_base;    // first global queue slot of this instance
};

// Adjoint sink that a lane switches on only for its adjoint retrace, so
// linking and adjoint lanes share one instruction stream. Only the running
// cell accumulation lives in registers; the target, weight and grid size sit
// in the lane's shared linking state and are read when a cell is flushed.
template <typename T>
struct GatedAdjSink {
    bool on;
    LinkState* L;
    CellAcc<T> acc;
    __device__ __forceinline__ void flush() {
        if (acc.ai == INT_MIN) return;
        const T w = (T)L->adj_w;
        const int nx = L->adj_nx, ny = L->adj_ny;
        const T w11 = acc.Wxy, w10 = acc.Wx - acc.Wxy, w01 = acc.Wy - acc.Wxy;
        const T w00 = (acc.W - acc.Wx) - w01;
        const int i = min(max(acc.ai, 0), nx - 2), j = min(max(acc.aj, 0), ny - 2);
        double* p = L->adj_g + (size_t)j * nx + i;
        atomicAdd(p, to_double(w * w00));
        atomicAdd(p + 1, to_double(w * w10));
        atomicAdd(p + nx, to_double(w * w01));
        atomicAdd(p + nx + 1, to_double(w * w11));
    }
    __device__ __forceinline__ void add(int ci, int cj, T tx, T ty, T a) {
        if (!on) return;
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
        if (!on) return;
        flush();
        acc.reset();
    }
};

// All instance descriptors travel as one kernel parameter (read through the
// constant cache, so the geometry costs no registers); 64 instances per launch.
constexpr int kMaxBatch = 64;
struct BatchParams {
    int n_inst;
    InstDesc d[kMaxBatch];
};

__device__ __forceinline__ int find_inst(const BatchParams& P, long long q) {
    int lo = 0, hi = P.n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.d[mid].pair_base <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// MINB: resident blocks per SM the kernel is compiled for (it caps the
// registers per thread at 64K / (BLOCK * MINB); fewer registers, more warps).
// STEPS: RK4 steps a lane takes between work-queue checks (its trace may end
// earlier; the lane then idles to the end of the iteration). The queue check
// and the warp's reconvergence cost a lone lane about a quarter of a step, so
// batching steps shortens the launch's tail of few active lanes.
template <typename T, int BLOCK, int STEPS, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB)
    k_batch(const __grid_constant__ BatchParams P, long long total, double tol, int max_iter, int fan_rays,
            unsigned long long* counters, unsigned long long* queue) {
    extern __shared__ unsigned char smem[];
    LinkState& L = reinterpret_cast<LinkState*>(smem)[threadIdx.x];
    Cell<T> C;
    C.F = nullptr; C.nx = 3; C.ny = 3; C.pi = INT_MIN; C.pj = INT_MIN;
    TraceState<T> ts;
    GatedAdjSink<T> sink;
    sink.on = false;
    sink.L = &L;
    sink.acc.reset();
    long long steps = 0;
    unsigned n_ok = 0, n_max = 0, n_cap = 0, n_bad = 0;
    bool active = false;
    int inst = -1;
    for (;;) {
        if (!active) {
            // warp-aggregated fetch of the next global slot
            const unsigned mask = __activemask();
            const int lane = threadIdx.x & 31;
            const int leader = __ffs(mask) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(queue, (unsigned long long)__popc(mask));
            base = __shfl_sync(mask, base, leader);
            const long long q = (long long)base + __popc(mask & ((1u << lane) - 1u));
            if (q >= total) break;
            inst = find_inst(P, q);
            const InstDesc& d = P.d[inst];
            const Geom& G = d.G;
            const int k = queue_pair(G, (int)(q - d.pair_base));
            if (C.F != d.field) {
                C.F = static_cast<const CellCoef<T>*>(d.field);
                C.nx = G.nx;
                C.ny = G.ny;
                C.pi = INT_MIN;
                C.pj = INT_MIN;
            }
            LinkCtx X;
            if (!setup_pair(G, k, X)) {
                d.theta[k] = nan("");
                d.tof[k] = nan("");
                if (d.hit) { d.hit[2 * k] = nan(""); d.hit[2 * k + 1] = nan(""); }
                if (d.iters) d.iters[k] = 0;
                if (d.status) d.status[k] = RT_RAY_BADINPUT;
                ++n_bad;
                continue;
            }
            L.xe = X.xe; L.ye = X.ye; L.xr = X.xr; L.yr = X.yr;
            L.phi_e = X.phi_e; L.psi_r = X.psi_r; L.th_lo = X.th_lo; L.th_hi = X.th_hi;
            const double margin = fmax(G.ds / G.R, 1e-9);
            L.a_min = X.th_lo + margin;
            L.a_max = X.th_hi - margin;
            const double tin = d.theta[k];
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
            if (fan_rays >= 2 && d.fan && isnan(tin)) {
                int e, r;
                pair_of(G, k, e, r);
                fan_start(G, L, d.fan + (size_t)e * fan_rays, fan_rays);
            }
            sink.on = false;
            trace_begin(ts, G, L.xe, L.ye, L.next);
            active = true;
        }
        const InstDesc& d = P.d[inst];
        const Geom& G = d.G;
        bool ended = false;
#pragma unroll 1
        for (int u = 0; u < STEPS; ++u)
            if (trace_step(C, G, ts, sink)) {
                ended = true;
                break;
            }
        if (!ended) continue;
        const TraceOut o = trace_end(C, G, ts, L.xe, L.ye, L.xr, L.yr, sink);
        steps += o.steps;
        if (sink.on) {                    // adjoint retrace done
            sink.on = false;
            active = false;
            continue;
        }
        if (link_update(G, L, o, tol, max_iter, fan_rays >= 2 ? d.fan : nullptr, fan_rays)) {
            const int k = L.k;
            const int st = (L.best_d2 <= tol * tol) ? RT_RAY_OK
                           : (L.best_d2 == DBL_MAX ? RT_RAY_STEPCAP : RT_RAY_MAXITER);
            d.theta[k] = L.best_th;
            d.tof[k] = L.best_T;
            if (d.hit) { d.hit[2 * k] = L.best_hx; d.hit[2 * k + 1] = L.best_hy; }
            if (d.iters) d.iters[k] = L.n_eval;
            if (d.status) d.status[k] = st;
            n_ok += st == RT_RAY_OK;
            n_max += st == RT_RAY_MAXITER;
            n_cap += st == RT_RAY_STEPCAP;
            const double w = d.tof_ref ? L.best_T - d.tof_ref[k] : 0.0;
            if (d.tof_ref && w != 0.0 && isfinite(w)) {
                sink.on = true;
                L.adj_g = d.g;
                L.adj_w = w;
                L.adj_nx = G.nx;
                L.adj_ny = G.ny;
                sink.acc.reset();
                trace_begin(ts, G, L.xe, L.ye, L.best_th);
            } else {
                active = false;
            }
        } else {
            trace_begin(ts, G, L.xe, L.ye, L.next);
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

// g_c = -1000 g / c^2 for every instance with an adjoint (blockIdx.y = instance).
__global__ void k_batch_finish(const __grid_constant__ BatchParams P) {
    const InstDesc& d = P.d[blockIdx.y];
    if (!d.tof_ref || !d.g) return;
    const int n = d.G.nx * d.G.ny;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double c = d.c_mps[k];
        d.g[k] = -1000.0 * d.g[k] / (c * c);
    }
}

}  // namespace rt

namespace {

using rt::InstDesc;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T, int BLOCK, int STEPS, int MINB>
cudaError_t launch_batch_kernel(const rt::BatchParams& D, long long total, double tol, int max_iter,
                                int fan_rays, unsigned long long* counters, unsigned long long* queue,
                                cudaStream_t s) {
    static std::atomic<int> cache[64];   // resident blocks of this variant, per device
    const size_t smem = sizeof(rt::LinkState) * BLOCK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int blocks = cache[dev].load(std::memory_order_relaxed);
    if (!blocks) {
        e = cudaFuncSetAttribute(rt::k_batch<T, BLOCK, STEPS, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rt::k_batch<T, BLOCK, STEPS, MINB>, BLOCK, smem);
        blocks = sms * (per_sm > 0 ? per_sm : 1);
        cache[dev].store(blocks, std::memory_order_relaxed);
    }
    const long long need = (total + BLOCK - 1) / BLOCK;
    const int nb = (int)(need < blocks ? need : blocks);
    if (nb <= 0) return cudaSuccess;
    rt::k_batch<T, BLOCK, STEPS, MINB><<<nb, BLOCK, smem, s>>>(D, total, tol, max_iter, fan_rays, counters, queue);
    return cudaGetLastError();
}

cudaError_t dispatch_batch(int prec, int block, int steps, int bpsm, const rt::BatchParams& D, long long total,
                           double tol, int max_iter, int fan_rays, unsigned long long* counters,
                           unsigned long long* queue, cudaStream_t s, bool* ok) {
    *ok = true;
    if (prec == RT_FP64) {
        if (block == 128 && steps == 16 && bpsm == 1)
            return launch_batch_kernel<double, 128, 16, 1>(D, total, tol, max_iter, fan_rays, counters, queue, s);
    } else {
#define RT_BATCH_CASE(B, U, M)                                                                                      \
    if (block == B && steps == U && bpsm == M)                                                                      \
        return launch_batch_kernel<float, B, U, M>(D, total, tol, max_iter, fan_rays, counters, queue, s);
        RT_BATCH_CASE(64, 16, 8) RT_BATCH_CASE(64, 16, 12) RT_BATCH_CASE(128, 16, 4) RT_BATCH_CASE(128, 16, 5)
        RT_BATCH_CASE(128, 16, 6) RT_BATCH_CASE(128, 1, 5) RT_BATCH_CASE(256, 16, 2) RT_BATCH_CASE(256, 16, 3)
#undef RT_BATCH_CASE
    }
    *ok = false;
    return cudaSuccess;
}

}  // namespace

extern "C" int rt_batch_run(rt_ctx* ctx, int32_t n_inst, const rt_instance* inst, const rt_options* opt,
                            void* stream) {
    if (!ctx) return RT_EINVAL;
    ctx->err.clear();
    cudaStream_t s = (cudaStream_t)stream;
    if (n_inst < 1 || !inst || !opt) return rt::set_error(ctx, RT_EINVAL, "need n_inst >= 1, instances and options");
    if (n_inst > rt::kMaxBatch) return rt::set_error(ctx, RT_EINVAL, "at most 64 instances per call");
    if (opt->precision != RT_FP64 && opt->precision != RT_FP32_COMP)
        return rt::set_error(ctx, RT_EINVAL, "unknown precision");
    if (!(opt->ds_mm > 0) || !(opt->tol_mm > 0) || opt->max_iter < 2)
        return rt::set_error(ctx, RT_EINVAL, "ds_mm and tol_mm must be > 0, max_iter >= 2");
    if (opt->integrator != RT_RK4 && opt->integrator != RT_HEUN) return rt::set_error(ctx, RT_EINVAL, "unknown integrator");
    if (opt->interpolator != RT_BILINEAR)
        return rt::set_error(ctx, RT_EINVAL, "rt_batch_run samples bilinearly (interpolator RT_BILINEAR)");
    if (opt->fan_rays == 1 || opt->fan_rays < 0 || opt->fan_rays > 65536)
        return rt::set_error(ctx, RT_EINVAL, "fan_rays must be 0 or in [2, 65536]");
    if (opt->subfan_rays != 0) return rt::set_error(ctx, RT_EINVAL, "rt_batch_run links in one launch: subfan_rays must be 0");
    const int block = opt->block_threads ? opt->block_threads : 128;
    const int steps = opt->step_unroll ? opt->step_unroll : 16;
    const int bpsm = opt->blocks_per_sm ? opt->blocks_per_sm
                                        : (opt->precision == RT_FP64 ? 1 : 512 / block);
    const size_t nb = rt::node_bytes(opt->precision);
    // per-instance geometry and workspace offsets; longest rings first
    std::vector<InstDesc> D((size_t)n_inst);
    std::vector<int> order((size_t)n_inst);
    for (int i = 0; i < n_inst; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return inst[a].prob.ring_radius_mm > inst[b].prob.ring_radius_mm;
    });
    size_t off = 0;
    std::vector<size_t> f_off(n_inst), fan_off(n_inst), need_off(n_inst), flag_off(n_inst);
    long long total = 0;
    for (int slot = 0; slot < n_inst; ++slot) {
        const int i = order[(size_t)slot];
        const rt_instance& I = inst[i];
        InstDesc& d = D[(size_t)slot];
        std::memset(&d, 0, sizeof(d));
        int rc = rt::make_geom(ctx, &I.prob, opt, &d.G);
        if (rc) return rt::set_error(ctx, rc, "instance " + std::to_string(i) + ": " + ctx->err);
        if (I.prob.n_pairs > 0 && (!I.theta_io || !I.tof_us))
            return rt::set_error(ctx, RT_EINVAL, "instance " + std::to_string(i) + ": theta_io and tof_us required");
        if (I.tof_ref && !I.g_c)
            return rt::set_error(ctx, RT_EINVAL, "instance " + std::to_string(i) + ": g_c required with tof_ref");
        f_off[slot] = off;
        off = align256(off + nb * (size_t)(I.prob.grid.nx - 1) * (size_t)(I.prob.grid.ny - 1));
        fan_off[slot] = off;
        off = align256(off + (opt->fan_rays >= 2 ? sizeof(double) * (size_t)I.prob.n_tx * opt->fan_rays : 0));
        need_off[slot] = off;
        off = align256(off + sizeof(int) * (size_t)I.prob.n_tx);
        flag_off[slot] = off;
        off = align256(off + sizeof(int));
        d.pair_base = total;
        total += I.prob.n_pairs;
    }
    // workspace (never allocated while the stream is being captured)
    if (ctx->batch_ws_bytes < off) {
        if (rt::stream_capturing(s))
            return rt::set_error(ctx, RT_EINVAL, "batch workspace too small during stream capture: run once first");
        if (cudaSetDevice(ctx->device) != cudaSuccess) return rt::set_error(ctx, RT_ECUDA, "cudaSetDevice");
        if (ctx->batch_ws) cudaFree(ctx->batch_ws);
        ctx->batch_ws = nullptr;
        ctx->batch_ws_bytes = 0;
        if (cudaMalloc(&ctx->batch_ws, off) != cudaSuccess) return rt::set_error(ctx, RT_ENOMEM, "batch workspace");
        ctx->batch_ws_bytes = off;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return rt::set_error(ctx, RT_ECUDA, "cudaSetDevice");
    unsigned char* ws = static_cast<unsigned char*>(ctx->batch_ws);
    cudaError_t e = cudaMemsetAsync(ctx->counters, 0, 8 * sizeof(unsigned long long), s);
    for (int slot = 0; slot < n_inst && e == cudaSuccess; ++slot) {
        const rt_instance& I = inst[order[(size_t)slot]];
        InstDesc& d = D[(size_t)slot];
        int* flag = reinterpret_cast<int*>(ws + flag_off[slot]);
        d.field = ws + f_off[slot];
        d.G.bad_field = flag;
        e = rt::launch_pack(I.prob.grid, I.prob.c_mps, ws + f_off[slot], flag, opt->precision, s);
        if (e != cudaSuccess) break;
        if (opt->fan_rays >= 2 && I.prob.n_pairs > 0) {
            d.fan = reinterpret_cast<const double*>(ws + fan_off[slot]);
            e = rt::launch_fan(d.G, opt->fan_ds_mm, d.field, opt->precision, opt->fan_rays, I.theta_io,
                               reinterpret_cast<double*>(ws + fan_off[slot]), reinterpret_cast<int*>(ws + need_off[slot]),
                               ctx->counters, s);
            if (e != cudaSuccess) break;
        }
        d.theta = I.theta_io;
        d.tof = I.tof_us;
        d.hit = I.hit_xy_mm;
        d.status = I.status;
        d.iters = I.iters;
        d.tof_ref = I.tof_ref;
        d.g = I.tof_ref ? I.g_c : nullptr;
        d.c_mps = I.prob.c_mps;
        if (I.tof_ref)
            e = cudaMemsetAsync(I.g_c, 0, sizeof(double) * (size_t)I.prob.grid.nx * I.prob.grid.ny, s);
    }
    if (e != cudaSuccess) return rt::set_error(ctx, RT_ECUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
    rt::BatchParams params{};   // the kernel parameter, copied at launch
    params.n_inst = n_inst;
    std::memcpy(params.d, D.data(), sizeof(InstDesc) * (size_t)n_inst);
    e = cudaMemsetAsync(ctx->queue, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return rt::set_error(ctx, RT_ECUDA, std::string("queue reset: ") + cudaGetErrorString(e));
    bool ok = true;
    e = dispatch_batch(opt->precision, block, steps, bpsm, params, total, opt->tol_mm, opt->max_iter, opt->fan_rays,
                       ctx->counters, reinterpret_cast<unsigned long long*>(ctx->queue), s, &ok);
    if (!ok)
        return rt::set_error(ctx, RT_EINVAL, "unsupported block_threads / step_unroll / blocks_per_sm combination");
    if (e != cudaSuccess) return rt::set_error(ctx, RT_ECUDA, std::string("batch kernel: ") + cudaGetErrorString(e));
    rt::k_batch_finish<<<dim3(64, (unsigned)n_inst), 256, 0, s>>>(params);
    e = cudaGetLastError();
    if (e != cudaSuccess) return rt::set_error(ctx, RT_ECUDA, std::string("batch finish: ") + cudaGetErrorString(e));
    ctx->last_stream = s;
    return RT_OK;
}
