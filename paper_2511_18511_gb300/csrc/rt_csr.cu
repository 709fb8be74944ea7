// rt_csr.cu — products with the explicit system matrix written by
// rt_path_matrix (paper Sec. 3.1.1: the matrix of interpolation-weighted path
// lengths is sparse enough to be stored and applied explicitly), for the
// linearised inversion steps (SART, CG) that apply the matrix of one
// linearisation many times at fixed rays.
//
// y = L x: one warp per row, lanes stride over the row's entries, shuffle sum
// (a breast-workload row holds ~4,000 entries). y = L^T w: one warp per row,
// each entry adds val * w[row] to y[col] with an FP64 atomic (rows of one
// emitter overlap near the emitter, so colliding adds are common only there).
#include <string>

#include <cuda_runtime.h>

#include "rt_internal.h"

namespace rt {
namespace {

constexpr int kCsrBlock = 256;

__global__ void k_csr_matvec(int n_rows, int n_cols, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y) {
    const int warp = (blockIdx.x * kCsrBlock + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n_rows) return;
    const int64_t b = row_ptr[warp], e = row_ptr[warp + 1];
    double acc = 0.0;
    for (int64_t k = b + lane; k < e; k += 32) {
        const int c = col[k];
        if ((unsigned)c < (unsigned)n_cols) acc = fma(val[k], x[c], acc);   // entries outside the columns are skipped
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) y[warp] = acc;
}

__global__ void k_csr_rmatvec(int n_rows, int n_cols, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                              const double* __restrict__ val, const double* __restrict__ w, double* __restrict__ y) {
    const int warp = (blockIdx.x * kCsrBlock + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n_rows) return;
    const double wr = w[warp];
    if (wr == 0.0) return;
    const int64_t b = row_ptr[warp], e = row_ptr[warp + 1];
    for (int64_t k = b + lane; k < e; k += 32) {
        const int c = col[k];
        if ((unsigned)c < (unsigned)n_cols) atomicAdd(y + c, val[k] * wr);
    }
}

int check(rt_ctx* ctx, int32_t n_rows, int32_t n_cols, const void* row_ptr, const void* col, const void* val,
          const void* x, const void* y) {
    if (!ctx) return RT_EINVAL;
    ctx->err.clear();
    if (n_rows < 0 || n_cols < 1) return set_error(ctx, RT_EINVAL, "n_rows must be >= 0 and n_cols >= 1");
    if (n_rows > 0 && (!row_ptr || !x)) return set_error(ctx, RT_EINVAL, "row_ptr and the input vector are required");
    if (!y) return set_error(ctx, RT_EINVAL, "the output vector is required");
    (void)col;
    (void)val;
    return RT_OK;
}

}  // namespace
}  // namespace rt

extern "C" {

int rt_csr_matvec(rt_ctx* ctx, int32_t n_rows, int32_t n_cols, const int64_t* row_ptr, const int32_t* col,
                  const double* val, const double* x, double* y, void* stream) {
    int rc = rt::check(ctx, n_rows, n_cols, row_ptr, col, val, x, y);
    if (rc) return rc;
    if (n_rows == 0) return RT_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) {
        const long long threads = 32LL * n_rows;
        rt::k_csr_matvec<<<(unsigned)((threads + rt::kCsrBlock - 1) / rt::kCsrBlock), rt::kCsrBlock, 0,
                           (cudaStream_t)stream>>>(n_rows, n_cols, row_ptr, col, val, x, y);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? RT_OK : rt::set_error(ctx, RT_ECUDA, std::string("csr matvec: ") + cudaGetErrorString(e));
}

int rt_csr_rmatvec(rt_ctx* ctx, int32_t n_rows, int32_t n_cols, const int64_t* row_ptr, const int32_t* col,
                   const double* val, const double* w, double* y, void* stream) {
    int rc = rt::check(ctx, n_rows, n_cols, row_ptr, col, val, w, y);
    if (rc) return rc;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaMemsetAsync(y, 0, sizeof(double) * (size_t)n_cols, (cudaStream_t)stream);
    if (e == cudaSuccess && n_rows > 0) {
        const long long threads = 32LL * n_rows;
        rt::k_csr_rmatvec<<<(unsigned)((threads + rt::kCsrBlock - 1) / rt::kCsrBlock), rt::kCsrBlock, 0,
                            (cudaStream_t)stream>>>(n_rows, n_cols, row_ptr, col, val, w, y);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? RT_OK
                            : rt::set_error(ctx, RT_ECUDA, std::string("csr rmatvec: ") + cudaGetErrorString(e));
}

}  // extern "C"
