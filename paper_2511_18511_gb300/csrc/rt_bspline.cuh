// rt_bspline.cuh — the cubic B-spline sampler of the ToF path (paper Sec.
// 3.3.1, second scheme: a C^2 piecewise-cubic field defined by control points
// at the grid nodes, with analytic derivatives).
//
// The spline interpolates the nodal values: its control coefficients are the
// nodal field filtered by the inverse of the (1, 4, 1)/6 interpolation matrix
// along each axis, with the mirror extension a_{-1} = a_1, a_n = a_{n-2}
// (rt_bspline.cu). Over cell (i, j) the spline is a bicubic in the in-cell
// fractions (tx, ty) built from the 4 x 4 coefficients i-1..i+2, j-1..j+2. The
// pack kernel stores that bicubic per cell in the power basis, so a sample is
// two Horner passes: value, d/dtx and d/dty of c (the ray equations, in cell
// units, want h grad c = the fraction derivatives) and, once per step, the
// value of the slowness bicubic. The current cell's c coefficients are cached
// in registers (16 values, as many as the bilinear cache holds for four
// fields); the slowness coefficients are read from L2 when needed.
#pragma once

#include "rt_trace.cuh"

namespace rt {

// Per-cell bicubics of c and s: f(tx, ty) = sum_{p,q} a_pq tx^p ty^q, stored as
// one vector (a_0q, a_1q, a_2q, a_3q) per power q of ty. Cell (i, j) at
// j*(nx-1) + i, like the bilinear cells.
template <typename T>
struct CellBS {
    typename Vec4T<T>::type c[4], s[4];
};

// value of a bicubic at (tx, ty)
template <typename T, typename V4>
__device__ __forceinline__ T bicubic(const V4* a, T tx, T ty) {
    T r[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const V4 v = a[q];
        r[q] = (T)v.x + tx * ((T)v.y + tx * ((T)v.z + tx * (T)v.w));
    }
    return r[0] + ty * (r[1] + ty * (r[2] + ty * r[3]));
}

template <typename T>
struct CellS {
    using V = CellBS<T>;
    const V* __restrict__ F;
    int nx, ny;
    int pi, pj;             // cached cell
    const V* pc;            // its coefficients
    T a[16];                // c: a[4q + p] multiplies tx^p ty^q

    __device__ __forceinline__ void load(int i, int j) {
        pi = i;
        pj = j;
        // clamp for memory safety; rays stay inside by the ring/grid check
        i = min(max(i, 0), nx - 2);
        j = min(max(j, 0), ny - 2);
        pc = F + (size_t)j * (nx - 1) + i;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const auto v = pc->c[q];
            a[4 * q] = v.x;
            a[4 * q + 1] = v.y;
            a[4 * q + 2] = v.z;
            a[4 * q + 3] = v.w;
        }
    }

    // c and its fraction derivatives (= h dc/dx, h dc/dy) at (u, v) relative to (ci, cj)
    __device__ __forceinline__ void at(int ci, int cj, T u, T v, T& c, T& gx, T& gy, T& tx, T& ty) {
        int i, j;
        if (cell_locate(ci, cj, u, v, pi, pj, i, j, tx, ty)) load(i, j);
        const T tx3 = (T)3 * tx;
        T r[4], d[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const T a0 = a[4 * q], a1 = a[4 * q + 1], a2 = a[4 * q + 2], a3 = a[4 * q + 3];
            r[q] = a0 + tx * (a1 + tx * (a2 + tx * a3));
            d[q] = a1 + tx * ((T)2 * a2 + tx3 * a3);
        }
        c = r[0] + ty * (r[1] + ty * (r[2] + ty * r[3]));
        gx = d[0] + ty * (d[1] + ty * (d[2] + ty * d[3]));
        gy = r[1] + ty * ((T)2 * r[2] + (T)3 * ty * r[3]);
    }

    // slowness at fractions (tx, ty) of the cached cell
    __device__ __forceinline__ T slow(T tx, T ty) const { return bicubic<T>(pc->s, tx, ty); }
};

// Uniform cubic B-spline basis at t in [0, 1): weights of coefficients i-1..i+2.
template <typename T>
__device__ __forceinline__ void bspline_weights(T t, T b[4]) {
    const T u = (T)1 - t, t2 = t * t, t3 = t2 * t;
    const T sixth = (T)(1.0 / 6.0);
    b[0] = u * u * u * sixth;
    b[1] = ((T)3 * t3 - (T)6 * t2 + (T)4) * sixth;
    b[2] = (((T)-3 * t3 + (T)3 * t2) + ((T)3 * t + (T)1)) * sixth;
    b[3] = t3 * sixth;
}

// coefficient index i-1..i+2 of an interior cell, folded by the mirror at the
// grid edges (index -1 -> 1, n -> n-2)
__device__ __forceinline__ int mirror_index(int v, int n) {
    v = v < 0 ? -v : v;
    return v > n - 1 ? 2 * (n - 1) - v : v;
}

// Accumulates sum alpha_m bx_p(tx_m) by_q(ty_m) over consecutive points of one cell.
template <typename T>
struct CellAccBS {
    int ai, aj;
    T W[16];
    __device__ __forceinline__ void reset() {
        ai = INT_MIN;
        aj = INT_MIN;
#pragma unroll
        for (int k = 0; k < 16; ++k) W[k] = (T)0;
    }
    __device__ __forceinline__ void add(T tx, T ty, T a) {
        T bx[4], by[4];
        bspline_weights(tx, bx);
        bspline_weights(ty, by);
#pragma unroll
        for (int p = 0; p < 4; ++p) bx[p] *= a;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int p = 0; p < 4; ++p) W[4 * q + p] += bx[p] * by[q];
    }
};

// Adjoint scatter onto the slowness coefficients: w * alpha_m * B_pq(x_m). The
// weights of the 4 x 4 coefficients around the current cell accumulate in a
// window that slides with the ray: when the ray steps into a neighbouring cell
// only the column (or row) of coefficients that leaves the window is flushed
// (4 FP64 atomics instead of 16 per cell crossing), the rest shifts along;
// the whole window is flushed at the end of the trace (or on a jump of more
// than one cell). The coefficient-space result is mapped back to nodes by the
// transposed prefilter afterwards.
template <typename T>
struct AdjSinkBSp {
    double* g;
    T w;
    int nx, ny;
    int ai, aj;        // cell the window is centred on (INT_MIN: empty)
    T W[16];           // W[4 b + a]: coefficient (ai - 1 + a, aj - 1 + b)

    __device__ __forceinline__ void init() {
        ai = INT_MIN;
        aj = INT_MIN;
        clear();
    }

    __device__ __forceinline__ void put(int a, int b) {
        const int i = min(max(ai, 0), nx - 2), j = min(max(aj, 0), ny - 2);
        atomicAdd(g + (size_t)mirror_index(j - 1 + b, ny) * nx + mirror_index(i - 1 + a, nx), to_double(w * W[4 * b + a]));
    }
    __device__ __forceinline__ void flush_all() {
        if (ai == INT_MIN) return;
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int a = 0; a < 4; ++a) put(a, b);
    }
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int k = 0; k < 16; ++k) W[k] = (T)0;
    }
    __device__ __forceinline__ void add(int ci, int cj, T tx, T ty, T a) {
        if (ci != ai || cj != aj) {
            const int di = ci - ai, dj = cj - aj;
            if (ai == INT_MIN || di < -1 || di > 1 || dj < -1 || dj > 1) {
                flush_all();
                clear();
                ai = ci;
                aj = cj;
            } else {
                if (di == 1) {            // column a = 0 leaves, the others move left
#pragma unroll
                    for (int b = 0; b < 4; ++b) put(0, b);
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        W[4 * b] = W[4 * b + 1]; W[4 * b + 1] = W[4 * b + 2]; W[4 * b + 2] = W[4 * b + 3]; W[4 * b + 3] = (T)0;
                    }
                    ai += 1;
                } else if (di == -1) {    // column a = 3 leaves, the others move right
#pragma unroll
                    for (int b = 0; b < 4; ++b) put(3, b);
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        W[4 * b + 3] = W[4 * b + 2]; W[4 * b + 2] = W[4 * b + 1]; W[4 * b + 1] = W[4 * b]; W[4 * b] = (T)0;
                    }
                    ai -= 1;
                }
                if (dj == 1) {            // row b = 0 leaves, the others move down
#pragma unroll
                    for (int q = 0; q < 4; ++q) put(q, 0);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        W[q] = W[4 + q]; W[4 + q] = W[8 + q]; W[8 + q] = W[12 + q]; W[12 + q] = (T)0;
                    }
                    aj += 1;
                } else if (dj == -1) {    // row b = 3 leaves, the others move up
#pragma unroll
                    for (int q = 0; q < 4; ++q) put(q, 3);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        W[12 + q] = W[8 + q]; W[8 + q] = W[4 + q]; W[4 + q] = W[q]; W[q] = (T)0;
                    }
                    aj -= 1;
                }
            }
        }
        T bx[4], by[4];
        bspline_weights(tx, bx);
        bspline_weights(ty, by);
#pragma unroll
        for (int p = 0; p < 4; ++p) bx[p] *= a;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int p = 0; p < 4; ++p) W[4 * q + p] += bx[p] * by[q];
    }
    __device__ __forceinline__ void finish() {
        flush_all();
        clear();
        ai = INT_MIN;
        aj = INT_MIN;
    }
};

// System-matrix rows over the slowness coefficients: 16 entries per cell visit
// (counting pass) / written (filling pass).
template <typename T>
struct RowSinkBSp {
    int nx, ny;
    int32_t* col;
    double* val;
    int64_t pos;
    int64_t end;
    bool fill;
    CellAccBS<T> acc;
    __device__ __forceinline__ void flush() {
        if (acc.ai == INT_MIN) return;
        if (fill && pos + 16 <= end) {
            const int i = min(max(acc.ai, 0), nx - 2), j = min(max(acc.aj, 0), ny - 2);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t row = mirror_index(j - 1 + q, ny) * nx;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    col[pos + 4 * q + p] = row + mirror_index(i - 1 + p, nx);
                    val[pos + 4 * q + p] = (double)acc.W[4 * q + p];
                }
            }
        }
        pos += 16;
    }
    __device__ __forceinline__ void add(int ci, int cj, T tx, T ty, T a) {
        if (ci != acc.ai || cj != acc.aj) {
            flush();
            acc.reset();
            acc.ai = ci;
            acc.aj = cj;
        }
        acc.add(tx, ty, a);
    }
    __device__ __forceinline__ void finish() { flush(); }
};

}  // namespace rt
