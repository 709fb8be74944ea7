// rt_noalloc.cu — travel times at fixed angles without any device allocation.
//
// The regular calls keep their packed field in workspace that an rt_ctx
// allocates with cudaMalloc. Some callers cannot allocate device memory at
// the point where they need travel times: a host that owns all device memory
// through its own pool and forbids other allocators, code that must not
// allocate once it has entered a real-time loop, or a plugin whose host
// hands it only input and output buffers. For them this file keeps the
// packed field in a fixed, file-scope device array instead. Every GPU that
// loads the library holds that array until the process exits.
#include <atomic>
#include <cstdio>

#include "rt_internal.h"
#include "rt_trace.cuh"

namespace {

// Capacity of the static scratch: the packed field (64 bytes per cell in
// FP32, 128 in FP64) plus one 256-byte slot for the bad-input flag.
constexpr size_t kScratchBytes = 16u << 20;   // 16 MiB
constexpr size_t kFlagBytes = 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes + kFlagBytes];

constexpr int kMaxDevices = 64;
// Device address of g_scratch per device, found with that device current.
// Host threads that make their first call on a device at the same time may
// both look it up; they find the same address, and the atomic store makes
// that benign.
std::atomic<void*> g_scratch_ptr[kMaxDevices];

int scratch_on(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return RT_EINVAL;
    void* p = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return RT_ECUDA;
        g_scratch_ptr[dev].store(p, std::memory_order_release);
    }
    *out = static_cast<unsigned char*>(p);
    return RT_OK;
}

}  // namespace

extern "C" int rt_tof_forward_noalloc(const rt_problem* prob, const rt_options* opt, const double* theta,
                                      double* tof_us, double* hit_xy_mm, void* stream) {
    if (!prob || !opt) return RT_EINVAL;
    if (opt->precision != RT_FP64 && opt->precision != RT_FP32_COMP) return RT_EINVAL;
    if (opt->integrator != RT_RK4 && opt->integrator != RT_HEUN) return RT_EINVAL;
    if (opt->interpolator != RT_BILINEAR) return RT_EINVAL;
    if (!(opt->ds_mm > 0)) return RT_EINVAL;
    if (prob->n_pairs > 0 && (!theta || !tof_us)) return RT_EINVAL;
    rt::Geom G;
    int rc = rt::make_geom(nullptr, prob, opt, &G);
    if (rc) return rc;
    const size_t need = rt::node_bytes(opt->precision) * (size_t)(prob->grid.nx - 1) * (size_t)(prob->grid.ny - 1);
    if (need > kScratchBytes) return RT_ENOMEM;   // grid larger than the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RT_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (s) {
        // the scratch address is the current device's: the stream must be on it
        int sdev = -1;
        if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) return RT_ECUDA;
        if (sdev != dev) return RT_EINVAL;
    }
    unsigned char* base = nullptr;
    rc = scratch_on(dev, &base);
    if (rc) return rc;
    void* field = base;
    int* flag = reinterpret_cast<int*>(base + kScratchBytes);
    // launch_pack clears the flag before packing
    if (rt::launch_pack(prob->grid, prob->c_mps, field, flag, opt->precision, s) != cudaSuccess) return RT_ECUDA;
    G.bad_field = flag;
    if (rt::launch_tof(G, field, opt->precision, theta, tof_us, hit_xy_mm, s) != cudaSuccess) return RT_ECUDA;
    return RT_OK;
}
