// rt_bspline.cu — coefficients and per-cell bicubics of the interpolating cubic
// B-spline sampler (paper Sec. 3.3.1, second scheme).
//
// Prefilter: the control coefficients a solve (a_{i-1} + 4 a_i + a_{i+1})/6 =
// f_i along each axis with the mirror extension a_{-1} = a_1, a_n = a_{n-2}.
// Each line is filtered by the recursive (causal + anti-causal) form of the
// inverse of that matrix (Unser, Aldroubi and Eden, "B-spline signal
// processing", IEEE Trans. Signal Process. 41, 1993: pole z = sqrt(3) - 2,
// gain 6, boundary values from the mirror-extended line), one thread per line,
// in FP64 for both marching precisions. The transposed system (the adjoint)
// reuses the same filter: with W = diag(1/2, 1, ..., 1, 1/2), W B is
// symmetric, so B^-T = W B^-1 W^-1 (scale the two end values by 2, filter,
// scale them back).
#include <cfloat>
#include <climits>
#include <string>

#include "rt_internal.h"
#include "rt_bspline.cuh"

namespace rt {
namespace {

constexpr double kZ = -0.2679491924311227;   // sqrt(3) - 2
constexpr int kHorizon = 40;                  // |z|^40 < 1e-22

// In-place filter of one strided line of n >= 3 values.
__device__ void filter_line(double* v, int n, size_t st, bool transpose) {
    if (transpose) {
        v[0] *= 2.0;
        v[(size_t)(n - 1) * st] *= 2.0;
    }
    // causal part, input scaled by the gain 6; its first value is the sum of
    // z^k f~_k over the mirror-extended line f~ (period 2n - 2)
    double c0 = 0.0;
    if (n > kHorizon) {
        double zk = 1.0;
        for (int k = 0; k < kHorizon; ++k) {
            c0 += zk * v[(size_t)k * st];
            zk *= kZ;
        }
    } else {
        double zn1 = 1.0;                        // z^(n-1)
        for (int k = 0; k < n - 1; ++k) zn1 *= kZ;
        double zk = kZ, zr = zn1 * zn1 / kZ;     // z^k and z^(2n-2-k) at k = 1
        c0 = v[0] + zn1 * v[(size_t)(n - 1) * st];
        for (int k = 1; k < n - 1; ++k) {
            c0 += v[(size_t)k * st] * (zk + zr);
            zk *= kZ;
            zr /= kZ;
        }
        c0 /= 1.0 - zn1 * zn1;
    }
    double prev = 6.0 * c0;
    v[0] = prev;
    for (int k = 1; k < n; ++k) {
        prev = 6.0 * v[(size_t)k * st] + kZ * prev;
        v[(size_t)k * st] = prev;
    }
    // anti-causal part
    double next = kZ / (kZ * kZ - 1.0) * (v[(size_t)(n - 1) * st] + kZ * v[(size_t)(n - 2) * st]);
    v[(size_t)(n - 1) * st] = next;
    for (int k = n - 2; k >= 0; --k) {
        next = kZ * (next - v[(size_t)k * st]);
        v[(size_t)k * st] = next;
    }
    if (transpose) {
        v[0] *= 0.5;
        v[(size_t)(n - 1) * st] *= 0.5;
    }
}

// nf fields of ny*nx values each, one thread per row (x) or column (y)
__global__ void k_filter_x(double* f, int nx, int ny, int nf, bool transpose) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ny * nf) return;
    filter_line(f + (size_t)t * nx, nx, 1, transpose);
}

__global__ void k_filter_y(double* f, int nx, int ny, int nf, bool transpose) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nx * nf) return;
    const int fld = t / nx, i = t - fld * nx;
    filter_line(f + (size_t)fld * nx * ny + i, ny, (size_t)nx, transpose);
}

// nodal c (mm/us) and s = 1/c into the two coefficient planes; flags c <= 0 or NaN
__global__ void k_nodal(const double* __restrict__ c_mps, size_t n, double* a, int* bad) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const double c = 1e-3 * c_mps[k];
        if (!(c > 0.0) || !isfinite(c)) atomicOr(bad, 1);
        a[k] = c;
        a[n + k] = 1.0 / c;
    }
}

// The bicubic of cell (i, j) in the power basis of its fractions from the 4 x 4
// coefficients around it: A = M W M^T with M the basis matrix of the uniform
// cubic B-spline (row p = coefficients of t^p in the four basis functions).
__device__ __forceinline__ void cell_bicubic(const double* a, int nx, int ny, int i, int j, double A[4][4]) {
    const double M[4][4] = {{1, 4, 1, 0}, {-3, 0, 3, 0}, {3, -6, 3, 0}, {-1, 3, -3, 1}};   // x 1/6
    double R[4][4];   // R[b][p] = sum_a M[p][a] w[b][a]
    for (int b = 0; b < 4; ++b) {
        const double* row = a + (size_t)mirror_index(j - 1 + b, ny) * nx;
        double w[4];
        for (int q = 0; q < 4; ++q) w[q] = row[mirror_index(i - 1 + q, nx)];
        for (int p = 0; p < 4; ++p) R[b][p] = M[p][0] * w[0] + M[p][1] * w[1] + M[p][2] * w[2] + M[p][3] * w[3];
    }
    for (int q = 0; q < 4; ++q)
        for (int p = 0; p < 4; ++p)
            A[q][p] = (M[q][0] * R[0][p] + M[q][1] * R[1][p] + M[q][2] * R[2][p] + M[q][3] * R[3][p]) / 36.0;
}

template <typename T>
__global__ void k_pack_bs(const double* __restrict__ a, int nx, int ny, CellBS<T>* F) {
    const int ncx = nx - 1, n = ncx * (ny - 1);
    const size_t nn = (size_t)nx * ny;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int j = k / ncx, i = k - j * ncx;
        CellBS<T> o;
        double A[4][4];
        cell_bicubic(a, nx, ny, i, j, A);
        for (int q = 0; q < 4; ++q) {
            o.c[q].x = (T)A[q][0]; o.c[q].y = (T)A[q][1]; o.c[q].z = (T)A[q][2]; o.c[q].w = (T)A[q][3];
        }
        cell_bicubic(a + nn, nx, ny, i, j, A);
        for (int q = 0; q < 4; ++q) {
            o.s[q].x = (T)A[q][0]; o.s[q].y = (T)A[q][1]; o.s[q].z = (T)A[q][2]; o.s[q].w = (T)A[q][3];
        }
        F[k] = o;
    }
}

}  // namespace

cudaError_t launch_bs_filter(double* f, int nx, int ny, int nf, bool transpose, cudaStream_t s) {
    k_filter_x<<<(ny * nf + 127) / 128, 128, 0, s>>>(f, nx, ny, nf, transpose);
    k_filter_y<<<(nx * nf + 127) / 128, 128, 0, s>>>(f, nx, ny, nf, transpose);
    return cudaGetLastError();
}

cudaError_t launch_pack_bs(const rt_grid& g, const double* c_mps, double* coef, void* field, int* dflag, int prec,
                           cudaStream_t s) {
    const size_t nn = (size_t)g.nx * g.ny;
    cudaError_t e = cudaMemsetAsync(dflag, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int nb = (int)((nn + 255) / 256 < 152 * 16 ? (nn + 255) / 256 : 152 * 16);
    k_nodal<<<nb, 256, 0, s>>>(c_mps, nn, coef, dflag);
    e = launch_bs_filter(coef, g.nx, g.ny, 2, false, s);
    if (e != cudaSuccess) return e;
    const int n = (g.nx - 1) * (g.ny - 1);
    const int blocks = (n + 255) / 256 < 152 * 16 ? (n + 255) / 256 : 152 * 16;
    if (prec == RT_FP64)
        k_pack_bs<double><<<blocks, 256, 0, s>>>(coef, g.nx, g.ny, (CellBS<double>*)field);
    else
        k_pack_bs<float><<<blocks, 256, 0, s>>>(coef, g.nx, g.ny, (CellBS<float>*)field);
    return cudaGetLastError();
}

}  // namespace rt

extern "C" {

int rt_bspline_coef(rt_ctx* ctx, int32_t nx, int32_t ny, const double* f, double* a, int32_t transpose,
                    void* stream) {
    if (!ctx) return RT_EINVAL;
    ctx->err.clear();
    if (nx < 3 || ny < 3 || (int64_t)nx * ny > (int64_t)INT32_MAX / 2)
        return rt::set_error(ctx, RT_EINVAL, "grid must have at least 3 nodes per axis");
    if (!f || !a) return rt::set_error(ctx, RT_EINVAL, "f and a are required");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess && a != f)
        e = cudaMemcpyAsync(a, f, sizeof(double) * (size_t)nx * ny, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = rt::launch_bs_filter(a, nx, ny, 1, transpose != 0, s);
    return e == cudaSuccess ? RT_OK : rt::set_error(ctx, RT_ECUDA, std::string("bspline filter: ") + cudaGetErrorString(e));
}

}  // extern "C"
