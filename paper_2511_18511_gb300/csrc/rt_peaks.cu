// rt_peaks.cu — microbenchmarks of the hardware rates the library's kernels
// are measured against: the FP32 and FP64 fused multiply-add rates (the ray
// march and the SIMT contraction are bound by them) and the L2 bandwidth for
// random 16-byte gathers and for coalesced 16-byte reads of an L2-resident
// buffer (the naive ray march gathers the 2 x 2 stencil of every sample; the
// Born contraction streams its pre-swizzled operand tiles). The caller times
// each launch with events on `stream` and divides the work stated in
// include/rt.h by the time.
#include <cstdint>

#include <cuda_runtime.h>

#include "rt_internal.h"
#include "rt_tc.cuh"

namespace rt {
namespace {

constexpr int kPeakThreads = 256;

// 8 independent chains of x = x * m + k per thread and loop trip, unrolled 8
// times: 64 FMAs between two loop tests. The result of every chain reaches
// memory, so nothing is eliminated.
template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(int iters, T m, T k, T* __restrict__ sink) {
    T x0 = (T)threadIdx.x, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int it = 0; it < iters; it += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            x0 = fma(x0, m, k); x1 = fma(x1, m, k); x2 = fma(x2, m, k); x3 = fma(x3, m, k);
            x4 = fma(x4, m, k); x5 = fma(x5, m, k); x6 = fma(x6, m, k); x7 = fma(x7, m, k);
        }
    }
    sink[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

// iters x 8 independent random float4 loads per thread from buf[0, n_vec)
// (n_vec a power of two); the index of each load comes from its own linear
// congruential sequence, so the loads of one trip do not depend on each other.
__global__ void __launch_bounds__(kPeakThreads) k_peak_gather(const float4* __restrict__ buf, uint32_t mask,
                                                              int iters, float* __restrict__ sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t h[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) h[u] = tid * 2654435761u + (uint32_t)u * 40503u + 12345u;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int it = 0; it < iters; ++it) {
        float4 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            h[u] = h[u] * 1664525u + 1013904223u;
            v[u] = buf[(h[u] >> 4) & mask];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            s.x += v[u].x; s.y += v[u].y; s.z += v[u].z; s.w += v[u].w;
        }
    }
    sink[tid] = (s.x + s.y) + (s.z + s.w);
}

// `passes` coalesced sweeps over buf[0, n_vec) by the whole grid (float4 per
// thread and trip, grid-stride).
__global__ void __launch_bounds__(kPeakThreads) k_peak_read(const float4* __restrict__ buf, int64_t n_vec,
                                                            int passes, float* __restrict__ sink) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int p = 0; p < passes; ++p) {
        int64_t i = tid;
        for (; i + 3 * stride < n_vec; i += 4 * stride) {
            const float4 a = buf[i], b = buf[i + stride], c = buf[i + 2 * stride], d = buf[i + 3 * stride];
            s.x += (a.x + b.x) + (c.x + d.x); s.y += (a.y + b.y) + (c.y + d.y);
            s.z += (a.z + b.z) + (c.z + d.z); s.w += (a.w + b.w) + (c.w + d.w);
        }
        for (; i < n_vec; i += stride) {
            const float4 a = buf[i];
            s.x += a.x; s.y += a.y; s.z += a.z; s.w += a.w;
        }
    }
    sink[tid] = (s.x + s.y) + (s.z + s.w);
}

// Self-test of the bounded wait the tensor-core kernels use: one block inits
// an mbarrier expecting one arrival; with `arrive` thread 0 arrives, otherwise
// nothing does; thread 0 then waits on the phase with mbar_wait_for. err
// receives 0 when the phase completed, kSelfTestCode when the wait gave up.
constexpr int kSelfTestCode = 199;

__global__ void k_wait_selftest(unsigned long long limit_ns, int arrive, int* err) {
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    const uint32_t b = tc::smem_u32(&bar);
    abort_flag = 0;
    tc::mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *err = 0;
    if (arrive) tc::mbar_arrive(b);
    tc::mbar_wait_for(b, 0, &abort_flag, err, kSelfTestCode, limit_ns);
}

}  // namespace
}  // namespace rt

extern "C" {

int rt_wait_selftest(int64_t limit_ns, int32_t arrive, int32_t* err, void* stream) {
    if (!err || limit_ns < 1000 || limit_ns > 2000000000ll) return RT_EINVAL;
    rt::k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>((unsigned long long)limit_ns, arrive ? 1 : 0, err);
    return cudaGetLastError() == cudaSuccess ? RT_OK : RT_ECUDA;
}

int rt_peak_fma(int32_t dtype, int32_t blocks, int32_t iters, void* sink, void* stream) {
    if (blocks < 1 || iters < 8 || (iters & 7) || !sink || (dtype != 0 && dtype != 1)) return RT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == 0)
        rt::k_peak_fma<float><<<blocks, rt::kPeakThreads, 0, s>>>(iters, 0.999999f, 1e-7f, (float*)sink);
    else
        rt::k_peak_fma<double><<<blocks, rt::kPeakThreads, 0, s>>>(iters, 0.999999999, 1e-13, (double*)sink);
    return cudaGetLastError() == cudaSuccess ? RT_OK : RT_ECUDA;
}

int rt_peak_gather(const void* buf, int64_t n_vec, int32_t blocks, int32_t iters, float* sink, void* stream) {
    if (!buf || !sink || blocks < 1 || iters < 1 || n_vec < 1 || n_vec > (int64_t(1) << 28) ||
        (n_vec & (n_vec - 1)))
        return RT_EINVAL;
    rt::k_peak_gather<<<blocks, rt::kPeakThreads, 0, (cudaStream_t)stream>>>(
        (const float4*)buf, (uint32_t)(n_vec - 1), iters, sink);
    return cudaGetLastError() == cudaSuccess ? RT_OK : RT_ECUDA;
}

int rt_peak_read(const void* buf, int64_t n_vec, int32_t blocks, int32_t passes, float* sink, void* stream) {
    if (!buf || !sink || blocks < 1 || passes < 1 || n_vec < 1) return RT_EINVAL;
    rt::k_peak_read<<<blocks, rt::kPeakThreads, 0, (cudaStream_t)stream>>>((const float4*)buf, n_vec, passes, sink);
    return cudaGetLastError() == cudaSuccess ? RT_OK : RT_ECUDA;
}

}  // extern "C"
