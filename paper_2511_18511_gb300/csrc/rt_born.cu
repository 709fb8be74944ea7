// rt_born.cu — the ray-Born operator: first-arrival travel-time and amplitude
// maps of every transducer from ray fans traced with their paraxial rays, and
// the linearised Born map and its adjoint (arXiv:2511.18511 Sec. 3.5 and the
// Appendix: Green's functions g = A exp(i omega T) whose phase follows the
// eikonal and whose geometric amplitude follows the transport equation through
// the ray Jacobian, obtained from a paraxial ray traced with each ray).
//
// Fan maps (rtborn_maps). One thread per fan ray, K rays per transducer at
// evenly spaced angles over the inward half-plane (the two tangents excluded
// by a margin ds/R). The march is the FP32-compensated one of the ToF path
// (cell-local position with a two-sum residual, double-float direction, RK4 or
// Heun's RK2 in cell units) extended by the paraxial pair in cell units Q~ = Q/h:
//     dQ~/ds~ = c P,   dP/ds~ = -(h^2 c_nn / c^2) Q~,   Q~(0) = 0, P(0) = 1/c_t,
// with c_nn = n^T H n, H the Hessian of c from central second differences
// interpolated bilinearly. The travel time is the trapezoid rule over the
// interpolated slowness (Kahan-summed). Every sample point after the
// transducer offers each node of the 3 x 3 block around its nearest node whose
// foot on the ray lies within half a step (-ds/2 <= d.D < ds/2, D = node -
// sample, a = d.D, b = n.D) the time extrapolated to second order in the
// ray-centred frame from the foot of the node on the ray,
//     T + s a + (M/2) b^2,   M = P/Q_f,   Q_f = Q + a c P   (|Q_f| >= h where M < 0),
// paired with A = sqrt(c / (c_t max(|Q_f|, h))). A node's travel time is its
// earliest candidate (first arrival; a 32-bit atomicMin on order-preserving
// bits of T). Its amplitude is that of the candidate of least
// T + RTBORN_ETA_US (b/h)^2 (a 64-bit atomicMin on the ordered score << 32 |
// bits of A): rays next to a node arrive within far less than the rounding of
// T of one another, so the earliest alone would choose among them by
// rounding; the penalty takes the ray passing closest to the node.
//
// With the cubic B-spline sampler (rt_options.interpolator = RT_BSPLINE; the
// paper's choice for ray-Born, Sec. 3.3.1) c, its gradient and its Hessian come
// from the per-cell bicubic of the interpolating spline of c (the ToF path's
// packed CellBS field: 16 coefficients cached per cell, derivatives by Horner)
// and s from the bicubic of s; alpha0 stays bilinear.
//
// Absorption (the Appendix: wavenumber k + i alpha, alpha = alpha0 omega^y,
// the absorption amplitude accumulated along the ray): with an alpha0 map each
// fan ray also carries Lambda = int alpha0 ds (trapezoid, Kahan-summed), a
// node's candidate is Lambda + alpha0 a from the foot, and the node keeps the
// Lambda of the candidate that supplies A (a third 64-bit atomicMin with the
// same score; an exact tie of scores may pair A and Lambda of different rays).
// E_t = A_t exp(-omega_s^y Lambda_t) exp(i omega T_t), omega_s in rad/s.
//
// Born map (rtborn_apply), per frequency f (omega = 2 pi f rad/us):
//     d[f][e][r] = omega^2 h^2 sum_{|x| < R} E_e(x) E_r(x) dc(x),  e != r,
// E_t = A_t exp(i omega T_t) over the nodes inside the ring (a compact list),
// the phase reduced as 2 pi frac(f T) with a compensated product. The adjoint
// (rtborn_adjoint) is
//     dc~(x) = Re sum_f omega^2 h^2 sum_{e != r} conj(E_e E_r) d[f][e][r].
// Both contractions run in rt_born_tc.cu: on the tensor cores (tcgen05,
// two-term TF32 split, E formed in the kernels' operand producers; the
// default, RTBORN_GEMM_TF32X3) or as FP32 SIMT complex GEMMs over E and
// W = omega^2 h^2 dc E formed by k_born_efield below (RTBORN_GEMM_FP32).
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "rt_internal.h"
#include "rt_trace.cuh"
#include "rt_bspline.cuh"

namespace rt {
namespace {

constexpr double kPiB = 3.14159265358979323846;

// Nodal fields for the Born march: (c, h dc/dx, h dc/dy, s) and
// (h^2 d2c/dx2, h^2 d2c/dxdy, h^2 d2c/dy2, alpha0 per mm of path), mm/us units.
struct __align__(32) BNode {
    float4 a, b;
};

__global__ void k_born_pack(rt_grid g, const double* __restrict__ c_mps, const double* __restrict__ alpha0,
                            BNode* __restrict__ out, int* bad) {
    const int nx = g.nx, ny = g.ny;
    const long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(k / nx), i = (int)(k - (long long)j * nx);
        const double v = c_mps[k];
        if (!(v > 0.0) || !(v < 1e300)) atomicExch(bad, 1);
        auto C = [&](int ii, int jj) { return 1e-3 * c_mps[(size_t)jj * nx + ii]; };
        const double c = 1e-3 * v;
        const double gx = (i == 0) ? C(1, j) - c : (i == nx - 1) ? c - C(nx - 2, j) : 0.5 * (C(i + 1, j) - C(i - 1, j));
        const double gy = (j == 0) ? C(i, 1) - c : (j == ny - 1) ? c - C(i, ny - 2) : 0.5 * (C(i, j + 1) - C(i, j - 1));
        double hxx = 0.0, hxy = 0.0, hyy = 0.0;
        if (i > 0 && i < nx - 1 && j > 0 && j < ny - 1) {
            hxx = C(i + 1, j) - 2.0 * c + C(i - 1, j);
            hyy = C(i, j + 1) - 2.0 * c + C(i, j - 1);
            hxy = 0.25 * (C(i + 1, j + 1) - C(i - 1, j + 1) - C(i + 1, j - 1) + C(i - 1, j - 1));
        }
        float al = 0.f;
        if (alpha0) {
            const double a0 = alpha0[k];
            if (!(a0 >= 0.0) || !(a0 < 1e300)) atomicExch(bad, 1);
            al = (float)(1e-3 * a0);   // per mm of path
        }
        BNode o;
        o.a = make_float4((float)c, (float)gx, (float)gy, (float)(1.0 / c));
        o.b = make_float4((float)hxx, (float)hxy, (float)hyy, al);
        out[k] = o;
    }
}

// Register cache of one cell: the seven fields (eight with absorption) in
// bilinear coefficient form f = a + tx bx + ty (by + tx bxy), built from the
// cell's four nodes.
template <bool ABS>
struct BornCell {
    const BNode* __restrict__ F;
    int nx, ny, pi, pj;
    float c0, c1, c2, c3, x0, x1, x2, x3, y0, y1, y2, y3, s0, s1, s2, s3;
    float p0, p1, p2, p3, q0, q1, q2, q3, r0, r1, r2, r3;   // hxx, hxy, hyy
    float l0, l1, l2, l3;                                   // alpha0 (ABS only)

    __device__ __forceinline__ void init(const BNode* f, const CellBS<float>*, int nx_, int ny_) {
        F = f;
        nx = nx_;
        ny = ny_;
    }

    __device__ __forceinline__ void load(int i, int j) {
        pi = i;
        pj = j;
        i = min(max(i, 0), nx - 2);
        j = min(max(j, 0), ny - 2);
        const BNode* p = F + (size_t)j * nx + i;
        const float4 a00 = p[0].a, b00 = p[0].b, a10 = p[1].a, b10 = p[1].b;
        const float4 a01 = p[nx].a, b01 = p[nx].b, a11 = p[nx + 1].a, b11 = p[nx + 1].b;
#define BC_(v0, v1, v2, v3, A00, A10, A01, A11) \
    v0 = A00; v1 = A10 - A00; v2 = A01 - A00; v3 = (A11 - A10) - (A01 - A00);
        BC_(c0, c1, c2, c3, a00.x, a10.x, a01.x, a11.x)
        BC_(x0, x1, x2, x3, a00.y, a10.y, a01.y, a11.y)
        BC_(y0, y1, y2, y3, a00.z, a10.z, a01.z, a11.z)
        BC_(s0, s1, s2, s3, a00.w, a10.w, a01.w, a11.w)
        BC_(p0, p1, p2, p3, b00.x, b10.x, b01.x, b11.x)
        BC_(q0, q1, q2, q3, b00.y, b10.y, b01.y, b11.y)
        BC_(r0, r1, r2, r3, b00.z, b10.z, b01.z, b11.z)
        if (ABS) {
            BC_(l0, l1, l2, l3, b00.w, b10.w, b01.w, b11.w)
        }
#undef BC_
    }

    // Fields at fractions (u, v) of cell (ci, cj), as Cell::at of the ToF path.
    __device__ __forceinline__ void at(int ci, int cj, float u, float v, float& c, float& gx, float& gy, float& hxx,
                                       float& hxy, float& hyy, float& tx, float& ty) {
        // 0 <= u < 1 on the float bits (-0 takes the general path, to the same result)
        if (ci == pi && cj == pj && __float_as_uint(u) < 0x3f800000u && __float_as_uint(v) < 0x3f800000u) {
            tx = u;
            ty = v;
        } else {
            int i, j;
            if (u >= -1.f && u < 2.f && v >= -1.f && v < 2.f) {
                const bool ul = u < 0.f, uh = u >= 1.f, vl = v < 0.f, vh = v >= 1.f;
                tx = ul ? u + 1.f : (uh ? u - 1.f : u);
                ty = vl ? v + 1.f : (vh ? v - 1.f : v);
                i = ci + (ul ? -1 : (uh ? 1 : 0));
                j = cj + (vl ? -1 : (vh ? 1 : 0));
            } else {
                const float fu = floorf(u), fv = floorf(v);
                i = ci + (int)fu;
                j = cj + (int)fv;
                tx = u - fu;
                ty = v - fv;
            }
            if (i != pi || j != pj) load(i, j);
        }
        c = c0 + tx * c1 + ty * (c2 + tx * c3);
        gx = x0 + tx * x1 + ty * (x2 + tx * x3);
        gy = y0 + tx * y1 + ty * (y2 + tx * y3);
        hxx = p0 + tx * p1 + ty * (p2 + tx * p3);
        hxy = q0 + tx * q1 + ty * (q2 + tx * q3);
        hyy = r0 + tx * r1 + ty * (r2 + tx * r3);
    }
    __device__ __forceinline__ float slow(float tx, float ty) const { return s0 + tx * s1 + ty * (s2 + tx * s3); }
    __device__ __forceinline__ float alpha(float tx, float ty) const { return l0 + tx * l1 + ty * (l2 + tx * l3); }
};

// The same interface over the B-spline field: the 16 coefficients of the
// current cell's bicubic of c in registers, c and its first and second
// fraction derivatives by Horner; s from the cell's bicubic of s (L2); alpha0
// bilinear from the node field (ABS only).
template <bool ABS>
struct BornCellS {
    const CellBS<float>* __restrict__ B;
    const BNode* __restrict__ F;
    int nx, ny, pi, pj;
    const CellBS<float>* pc;
    float a[16];
    float l0, l1, l2, l3;

    __device__ __forceinline__ void init(const BNode* f, const CellBS<float>* b, int nx_, int ny_) {
        F = f;
        B = b;
        nx = nx_;
        ny = ny_;
    }

    __device__ __forceinline__ void load(int i, int j) {
        pi = i;
        pj = j;
        i = min(max(i, 0), nx - 2);
        j = min(max(j, 0), ny - 2);
        pc = B + (size_t)j * (nx - 1) + i;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = pc->c[q];
            a[4 * q] = v.x;
            a[4 * q + 1] = v.y;
            a[4 * q + 2] = v.z;
            a[4 * q + 3] = v.w;
        }
        if (ABS) {
            const BNode* p = F + (size_t)j * nx + i;
            const float w00 = p[0].b.w, w10 = p[1].b.w, w01 = p[nx].b.w, w11 = p[nx + 1].b.w;
            l0 = w00;
            l1 = w10 - w00;
            l2 = w01 - w00;
            l3 = (w11 - w10) - (w01 - w00);
        }
    }

    __device__ __forceinline__ void at(int ci, int cj, float u, float v, float& c, float& gx, float& gy, float& hxx,
                                       float& hxy, float& hyy, float& tx, float& ty) {
        int i, j;
        if (cell_locate(ci, cj, u, v, pi, pj, i, j, tx, ty)) load(i, j);
        const float tx3 = 3.f * tx, tx6 = 6.f * tx;
        float r[4], d[4], e[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float a0 = a[4 * q], a1 = a[4 * q + 1], a2 = a[4 * q + 2], a3 = a[4 * q + 3];
            r[q] = a0 + tx * (a1 + tx * (a2 + tx * a3));
            d[q] = a1 + tx * (2.f * a2 + tx3 * a3);
            e[q] = 2.f * a2 + tx6 * a3;
        }
        c = r[0] + ty * (r[1] + ty * (r[2] + ty * r[3]));
        gx = d[0] + ty * (d[1] + ty * (d[2] + ty * d[3]));
        hxx = e[0] + ty * (e[1] + ty * (e[2] + ty * e[3]));
        gy = r[1] + ty * (2.f * r[2] + 3.f * ty * r[3]);
        hxy = d[1] + ty * (2.f * d[2] + 3.f * ty * d[3]);
        hyy = 2.f * r[2] + 6.f * ty * r[3];
    }
    __device__ __forceinline__ float slow(float tx, float ty) const { return bicubic<float>(pc->s, tx, ty); }
    __device__ __forceinline__ float alpha(float tx, float ty) const { return l0 + tx * l1 + ty * (l2 + tx * l3); }
};

// ray and paraxial right-hand sides at stage direction (ex, ey)
__device__ __forceinline__ void born_rhs(float c, float gx, float gy, float hxx, float hxy, float hyy, float ex,
                                         float ey, float Q, float P, float& kx, float& ky, float& kQ, float& kP) {
    const float ic = rcp_approx(c);
    const float gd = gx * ex + gy * ey;
    kx = (gd * ex - gx) * ic;
    ky = (gd * ey - gy) * ic;
    const float cnn = ey * ey * hxx - 2.f * ex * ey * hxy + ex * ex * hyy;
    kQ = c * P;
    kP = -cnn * ic * ic * Q;
}

struct BornRay {
    RayState<float> S;
    float Q, P;
};

// One RK4 step of length H (cells). Stage 1 has already been evaluated at S
// (c1.., passed in), since the deposit of S needs it.
template <typename CellB>
__device__ __forceinline__ void born_rk4(CellB& C, const BornRay& B, float H, float c, float gx, float gy,
                                         float hxx, float hxy, float hyy, BornRay& N) {
    const float Hh = 0.5f * H, H6 = H / 6.f;
    const float dx = B.S.d.hx(), dy = B.S.d.hy();
    float tx, ty, k1x, k1y, k1Q, k1P, k2x, k2y, k2Q, k2P, k3x, k3y, k3Q, k3P, k4x, k4y, k4Q, k4P;
    born_rhs(c, gx, gy, hxx, hxy, hyy, dx, dy, B.Q, B.P, k1x, k1y, k1Q, k1P);
    float e2x = dx + Hh * k1x, e2y = dy + Hh * k1y, Q2 = B.Q + Hh * k1Q, P2 = B.P + Hh * k1P;
    C.at(B.S.ci, B.S.cj, B.S.fx + Hh * dx, B.S.fy + Hh * dy, c, gx, gy, hxx, hxy, hyy, tx, ty);
    born_rhs(c, gx, gy, hxx, hxy, hyy, e2x, e2y, Q2, P2, k2x, k2y, k2Q, k2P);
    float e3x = dx + Hh * k2x, e3y = dy + Hh * k2y, Q3 = B.Q + Hh * k2Q, P3 = B.P + Hh * k2P;
    C.at(B.S.ci, B.S.cj, B.S.fx + Hh * e2x, B.S.fy + Hh * e2y, c, gx, gy, hxx, hxy, hyy, tx, ty);
    born_rhs(c, gx, gy, hxx, hxy, hyy, e3x, e3y, Q3, P3, k3x, k3y, k3Q, k3P);
    float e4x = dx + H * k3x, e4y = dy + H * k3y, Q4 = B.Q + H * k3Q, P4 = B.P + H * k3P;
    C.at(B.S.ci, B.S.cj, B.S.fx + H * e3x, B.S.fy + H * e3y, c, gx, gy, hxx, hxy, hyy, tx, ty);
    born_rhs(c, gx, gy, hxx, hxy, hyy, e4x, e4y, Q4, P4, k4x, k4y, k4Q, k4P);
    N.Q = B.Q + H6 * (k1Q + 2.f * (k2Q + k3Q) + k4Q);
    N.P = B.P + H6 * (k1P + 2.f * (k2P + k3P) + k4P);
    float nfx = B.S.fx, nfy = B.S.fy;
    N.S.lx = B.S.lx;
    N.S.ly = B.S.ly;
    add_frac(nfx, N.S.lx, H6 * (dx + 2.f * (e2x + e3x) + e4x) + H * B.S.d.lx());
    add_frac(nfy, N.S.ly, H6 * (dy + 2.f * (e2y + e3y) + e4y) + H * B.S.d.ly());
    N.S.d = B.S.d;
    N.S.d.add_normalize(H6 * (k1x + 2.f * (k2x + k3x) + k4x), H6 * (k1y + 2.f * (k2y + k3y) + k4y));
    N.S.ci = B.S.ci;
    N.S.cj = B.S.cj;
    if (nfx >= 1.f) { N.S.ci += 1; nfx -= 1.f; } else if (nfx < 0.f) { N.S.ci -= 1; add_frac(nfx, N.S.lx, 1.f); }
    if (nfy >= 1.f) { N.S.cj += 1; nfy -= 1.f; } else if (nfy < 0.f) { N.S.cj -= 1; add_frac(nfy, N.S.ly, 1.f); }
    N.S.fx = nfx;
    N.S.fy = nfy;
}

// One step of Heun's second-order Runge-Kutta method on (x, d, Q, P) (the
// slopes at the start, given as stage 1, and at the Euler end point, averaged),
// in the same cell-unit, compensated form as born_rk4.
template <typename CellB>
__device__ __forceinline__ void born_heun(CellB& C, const BornRay& B, float H, float c, float gx, float gy,
                                          float hxx, float hxy, float hyy, BornRay& N) {
    const float Hh = 0.5f * H;
    const float dx = B.S.d.hx(), dy = B.S.d.hy();
    float tx, ty, k1x, k1y, k1Q, k1P, k2x, k2y, k2Q, k2P;
    born_rhs(c, gx, gy, hxx, hxy, hyy, dx, dy, B.Q, B.P, k1x, k1y, k1Q, k1P);
    const float e2x = dx + H * k1x, e2y = dy + H * k1y, Q2 = B.Q + H * k1Q, P2 = B.P + H * k1P;
    C.at(B.S.ci, B.S.cj, B.S.fx + H * dx, B.S.fy + H * dy, c, gx, gy, hxx, hxy, hyy, tx, ty);
    born_rhs(c, gx, gy, hxx, hxy, hyy, e2x, e2y, Q2, P2, k2x, k2y, k2Q, k2P);
    N.Q = B.Q + Hh * (k1Q + k2Q);
    N.P = B.P + Hh * (k1P + k2P);
    float nfx = B.S.fx, nfy = B.S.fy;
    N.S.lx = B.S.lx;
    N.S.ly = B.S.ly;
    add_frac(nfx, N.S.lx, Hh * (dx + e2x) + H * B.S.d.lx());
    add_frac(nfy, N.S.ly, Hh * (dy + e2y) + H * B.S.d.ly());
    N.S.d = B.S.d;
    N.S.d.add_normalize(Hh * (k1x + k2x), Hh * (k1y + k2y));
    N.S.ci = B.S.ci;
    N.S.cj = B.S.cj;
    if (nfx >= 1.f) { N.S.ci += 1; nfx -= 1.f; } else if (nfx < 0.f) { N.S.ci -= 1; add_frac(nfx, N.S.lx, 1.f); }
    if (nfy >= 1.f) { N.S.cj += 1; nfy -= 1.f; } else if (nfy < 0.f) { N.S.cj -= 1; add_frac(nfy, N.S.ly, 1.f); }
    N.S.fx = nfx;
    N.S.fy = nfy;
}

// square root by the hardware approximation (sqrt.approx.ftz.f32), for values
// whose last bits only need to be reproducible
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// order-preserving map of float bits to unsigned (negative values included)
__device__ __forceinline__ unsigned f2ord(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

struct FanArgs {
    int K;
    float hf;                     // h, mm
    float Hhalf;                  // ds / (2h), cells
    float eta;                    // us: penalty of the squared distance (cells) to the ray, amplitude choice
    unsigned* tfirst;             // [n_tx][ny*nx] order-preserving bits of the first arrival
    unsigned long long* near;     // [n_tx][ny*nx] (ordered bits of T + eta b^2) << 32 | A bits
    unsigned long long* lam;      // [n_tx][ny*nx] the same score << 32 | bits of Lambda (absorption only)
    long long nn;
    unsigned long long* steps;    // RK4 steps taken (summed over rays)
};

// Per-ray constants of the deposit: the transducer in cell coordinates and
// h / c_t, for the reference time T_ref = h |node - x_t| / c_t of a node,
// which is the same for every ray of the fan.
struct FanRef {
    float xt, yt, h_ct;
};

// Offer the nodes around sample B (Kahan pair T - Tc, stage-1 c and s) their
// candidates: the first arrival by a 32-bit atomicMin on the ordered time; the
// amplitude by a 64-bit atomicMin on (ordered score) << 32 | bits of A, with
// score = T_cand - T_ref + eta b^2. T and T_ref lie within a factor of two of
// each other, so their difference is exact and the score resolves ~1e-6 us
// where T itself rounds at ~1e-5 us.
template <bool ABS>
__device__ __forceinline__ void born_deposit(const Geom& G, const FanArgs& A, const FanRef& F,
                                             unsigned* __restrict__ tfirst, unsigned long long* __restrict__ near,
                                             unsigned long long* __restrict__ lam, const BornRay& B, float T,
                                             float Tc, float c, float s, float inv_ct_h, float Lm, float al_h) {
    const float fx = B.S.fx, fy = B.S.fy;
    const bool oi = fx >= 0.5f, oj = fy >= 0.5f;
    const float D0x = oi ? 1.f - fx : -fx, D0y = oj ? 1.f - fy : -fy;
    const float dx = B.S.d.hx(), dy = B.S.d.hy();
    const float al0 = dx * D0x + dy * D0y;
    const float ac0 = dx * D0y - dy * D0x;
    const int ic = B.S.ci + (oi ? 1 : 0), jc = B.S.cj + (oj ? 1 : 0);
    const float fic = (float)ic, fjc = (float)jc;
    const float cP = c * B.P;
    // Which of the nine nodes take a candidate (bit 3 (b + 1) + a + 1), then
    // one pass per taken node: the warp runs the candidate body as often as its
    // busiest lane has nodes (about once per sample at ds = h/10) instead of
    // once per block position that any of its lanes takes.
    // The window -ds/2 <= a < ds/2 as 0 <= a + ds/2 < ds on the float bits: a
    // non-negative float below ds has smaller bits than ds, and a negative one
    // (or NaN) larger. The whole block inside the grid is the rule (a ring at
    // least a cell and a step inside the grid); the per-node test is the
    // exception.
    unsigned take = 0;
    const unsigned wbits = __float_as_uint(2.f * A.Hhalf);
    const float sh = al0 + A.Hhalf;
#pragma unroll
    for (int b = -1; b <= 1; ++b) {
        const float t = sh + (float)b * dy;
#pragma unroll
        for (int a = -1; a <= 1; ++a)
            if (__float_as_uint(t + (float)a * dx) < wbits) take |= 1u << (3 * (b + 1) + (a + 1));
    }
    if (ic < 1 || ic >= G.nx - 1 || jc < 1 || jc >= G.ny - 1) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const int ni = ic + q % 3 - 1, nj = jc + q / 3 - 1;
            if (ni < 0 || ni >= G.nx || nj < 0 || nj >= G.ny) take &= ~(1u << q);
        }
    }
    while (take) {
        const int q = __ffs(take) - 1;
        take &= take - 1;
        const int b = (q >= 6) ? 1 : ((q >= 3) ? 0 : -1);
        const int a = q - 3 * (b + 1) - 1;
        const float fa = (float)a, fb = (float)b;
        const float al = al0 + fa * dx + fb * dy;
        const float ac = ac0 + fb * dx - fa * dy;
        const int ni = ic + a, nj = jc + b;
        // paraxial Q carried to the foot of the node (dQ~/ds~ = c P)
        const float Qf = B.Q + al * cP;
        const float aQ = fabsf(Qf);
        const float Qc = aQ >= 1.f ? aQ : 1.f;
        float M = B.P * rcp_approx(Qf);
        if (!(M >= 0.f)) M = B.P * rcp_approx(copysignf(Qc, Qf));
        const float ext = A.hf * (s * al + 0.5f * M * ac * ac) - Tc;
        const size_t node = (size_t)nj * G.nx + ni;
        atomicMin(tfirst + node, f2ord(T + ext));
        const float ux = (fic + fa) - F.xt, uy = (fjc + fb) - F.yt;   // node index sums are exact
        // the same value for every candidate of the node from this transducer's fan
        const float Tref = F.h_ct * sqrt_approx(ux * ux + uy * uy);
        const float score = ((T - Tref) + ext) + A.eta * ac * ac;
        const float amp = sqrtf(c * inv_ct_h * rcp_approx(Qc));
        const unsigned long long sk = (unsigned long long)f2ord(score) << 32;
        atomicMin(near + node, sk | __float_as_uint(amp));
        // Lambda >= 0: its float bits order like its value
        if (ABS) atomicMin(lam + node, sk | __float_as_uint(fmaxf(Lm + al_h * al, 0.f)));
    }
}

template <int BLOCK, int MINB, bool ABS, bool BS>
__global__ void __launch_bounds__(BLOCK, MINB) k_born_fan(const Geom G, const FanArgs A, const BNode* __restrict__ field,
                                                          const CellBS<float>* __restrict__ bsfield) {
    const long long id = blockIdx.x * (long long)BLOCK + threadIdx.x;
    if (id >= (long long)G.n_tx * A.K) return;
    if (*G.bad_field) return;   // c <= 0 or NaN somewhere: every node stays unreached
    const int t = (int)(id / A.K), k = (int)(id - (long long)t * A.K);
    const double xe = G.tx[2 * t], ye = G.tx[2 * t + 1];
    const double phi = atan2(ye, xe);
    double margin = G.ds / G.R;
    if (margin < 1e-9) margin = 1e-9;
    const double a_min = phi + 0.5 * kPiB + margin;
    const double step = ((phi + 1.5 * kPiB - margin) - a_min) / (A.K - 1);
    const double theta = a_min + k * step;
    unsigned* __restrict__ tfirst = A.tfirst + (size_t)t * A.nn;
    unsigned long long* __restrict__ near = A.near + (size_t)t * A.nn;
    unsigned long long* __restrict__ lam = ABS ? A.lam + (size_t)t * A.nn : nullptr;

    BornRay B;
    {
        const double u = (xe - G.x0) / G.h, v = (ye - G.y0) / G.h;
        const double fu = floor(u), fv = floor(v);
        B.S.ci = (int)fu;
        B.S.cj = (int)fv;
        B.S.fx = (float)(u - fu);
        B.S.fy = (float)(v - fv);
        B.S.lx = (float)((u - fu) - (double)B.S.fx);
        B.S.ly = (float)((v - fv) - (double)B.S.fy);
        B.S.d.set(theta);
    }
    typename std::conditional<BS, BornCellS<ABS>, BornCell<ABS>>::type C;
    C.init(field, bsfield, G.nx, G.ny);
    C.load(B.S.ci, B.S.cj);
    const float H = G.Hf;
    const float half_ds = 0.5f * G.dsf;
    float c, gx, gy, hxx, hxy, hyy, tx, ty;
    C.at(B.S.ci, B.S.cj, B.S.fx, B.S.fy, c, gx, gy, hxx, hxy, hyy, tx, ty);
    const float c_t = c;
    const float inv_ct_h = 1.f / (c_t * A.hf);
    FanRef F;
    F.xt = (float)((xe - G.x0) / G.h);
    F.yt = (float)((ye - G.y0) / G.h);
    F.h_ct = A.hf / c_t;
    B.Q = 0.f;
    B.P = 1.f / c_t;
    float s_prev = C.slow(tx, ty);
    float T = 0.f, Tc = 0.f;       // Kahan sum of the trapezoid increments
    float a_prev = ABS ? C.alpha(tx, ty) : 0.f;
    float Lm = 0.f, Lc = 0.f;      // Kahan sum of the absorption path integral (ABS)
    int safe = 0, nsteps = 0;
    for (int m = 1; m <= G.max_steps_i; ++m) {
        BornRay N;
        if (G.heun) born_heun(C, B, H, c, gx, gy, hxx, hxy, hyy, N);
        else born_rk4(C, B, H, c, gx, gy, hxx, hxy, hyy, N);
        ++nsteps;
        if (--safe < 0) {
            const float ex = ring_excess(G, N.S);
            if (ex >= 0.f) break;
            const float Rc = G.Rcf;
            const float r = sqrtf(Rc * Rc + ex);
            safe = (int)((-ex / (Rc + r)) * 0.98f / H) - 1;
        }
        B = N;
        C.at(B.S.ci, B.S.cj, B.S.fx, B.S.fy, c, gx, gy, hxx, hxy, hyy, tx, ty);
        const float s = C.slow(tx, ty);
        const float y = half_ds * (s_prev + s) - Tc;
        const float tt = T + y;
        Tc = (tt - T) - y;
        T = tt;
        s_prev = s;
        float al_h = 0.f;
        if (ABS) {
            const float a = C.alpha(tx, ty);
            const float ya = half_ds * (a_prev + a) - Lc;
            const float tl = Lm + ya;
            Lc = (tl - Lm) - ya;
            Lm = tl;
            a_prev = a;
            al_h = a * A.hf;   // per cell of the along-ray offset
        }
        born_deposit<ABS>(G, A, F, tfirst, near, lam, B, T, Tc, c, s, inv_ct_h, Lm - Lc, al_h);
    }
    const unsigned mask = __activemask();
    const unsigned tot = __reduce_add_sync(mask, (unsigned)nsteps);
    if ((threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(A.steps, (unsigned long long)tot);
}

__global__ void k_born_unpack(const unsigned* __restrict__ tfirst, const unsigned long long* __restrict__ near,
                              const unsigned long long* __restrict__ lam, long long n, float* __restrict__ T,
                              float* __restrict__ A, float* __restrict__ L) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const unsigned tf = tfirst[k];
        const unsigned long long key = near[k];
        const bool none = tf == 0xffffffffu || key == ~0ull;
        T[k] = tf == 0xffffffffu ? __uint_as_float(0x7f800000u) : ord2f(tf);
        A[k] = none ? 0.f : __uint_as_float((unsigned)key);
        if (L) {
            const unsigned long long lk = lam[k];
            L[k] = (none || lk == ~0ull) ? 0.f : __uint_as_float((unsigned)lk);
        }
    }
}

// E[t][p] = A exp(-wy L) exp(i 2 pi frac(f T)) at inside node idx[p] (L and
// wy = omega_s^y only with absorption); W = scale dc E.
__global__ void k_born_efield(int n_in, const int* __restrict__ idx, long long nn, const float* __restrict__ Tm,
                              const float* __restrict__ Am, const float* __restrict__ Lm, float wy, float f_hi,
                              float f_lo, float scale, const float* __restrict__ dc, float2* __restrict__ E,
                              float2* __restrict__ W) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_in) return;
    const int t = blockIdx.y;
    const int k = idx[p];
    const float Tv = Tm[(size_t)t * nn + k];
    float Av = Am[(size_t)t * nn + k];
    if (Lm) Av *= expf(-wy * Lm[(size_t)t * nn + k]);
    float2 e = make_float2(0.f, 0.f);
    if (Tv < __uint_as_float(0x7f800000u)) {
        // frac(f T) with f = f_hi + f_lo: the product's rounding error by FMA
        const float pr = f_hi * Tv;
        const float er = fmaf(f_hi, Tv, -pr);
        const float fr = (pr - rintf(pr)) + (er + f_lo * Tv);
        float sn, cs;
        sincospif(2.f * fr, &sn, &cs);
        e = make_float2(Av * cs, Av * sn);
    }
    const size_t o = (size_t)t * n_in + p;
    E[o] = e;
    if (W) {
        const float w = scale * dc[k];
        W[o] = make_float2(w * e.x, w * e.y);
    }
}

__global__ void k_zero_diag(float2* d, int n_tx, int n_freq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tx * n_freq) return;
    const int f = i / n_tx, e = i - f * n_tx;
    d[((size_t)f * n_tx + e) * n_tx + e] = make_float2(0.f, 0.f);
}

// Dc[r + e n] = conj(d[e][r]), 0 on the diagonal
__global__ void k_conj_nodiag(const float2* __restrict__ d, float2* __restrict__ Dc, int n_tx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tx * n_tx) return;
    const int e = i / n_tx, r = i - e * n_tx;
    const float2 v = d[i];
    Dc[i] = (e == r) ? make_float2(0.f, 0.f) : make_float2(v.x, -v.y);
}

// acc[p] (+)= scale * Re sum_e E[e][p] V[e][p]
__global__ void k_born_reduce(int n_in, int n_tx, const float2* __restrict__ E, const float2* __restrict__ V,
                              float scale, double* __restrict__ acc, int first) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_in) return;
    float s0 = 0.f, s1 = 0.f;
    int e = 0;
    for (; e + 1 < n_tx; e += 2) {
        const float2 a = E[(size_t)e * n_in + p], b = V[(size_t)e * n_in + p];
        const float2 a2 = E[(size_t)(e + 1) * n_in + p], b2 = V[(size_t)(e + 1) * n_in + p];
        s0 = fmaf(a.x, b.x, fmaf(-a.y, b.y, s0));
        s1 = fmaf(a2.x, b2.x, fmaf(-a2.y, b2.y, s1));
    }
    if (e < n_tx) {
        const float2 a = E[(size_t)e * n_in + p], b = V[(size_t)e * n_in + p];
        s0 = fmaf(a.x, b.x, fmaf(-a.y, b.y, s0));
    }
    const double v = (double)(scale * (s0 + s1));
    acc[p] = first ? v : acc[p] + v;
}

__global__ void k_born_scatter(int n_in, const int* __restrict__ idx, const double* __restrict__ acc,
                               float* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n_in) out[idx[p]] = (float)acc[p];
}

}  // namespace

}  // namespace rt

// ------------------------------------------------------------------ host side

namespace {

int bfail(rt_ctx* ctx, int code, const std::string& msg) { return rt::set_error(ctx, code, msg); }

int bcuda(rt_ctx* ctx, cudaError_t e, const char* where) {
    return bfail(ctx, RT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Grows one workspace buffer (never during stream capture).
int grow(rt_ctx* ctx, void** p, size_t* have, size_t need, cudaStream_t s, const char* what) {
    if (*have >= need) return RT_OK;
    if (rt::stream_capturing(s)) return bfail(ctx, RT_EINVAL, std::string(what) + " workspace too small during capture");
    if (*p) cudaFree(*p);
    *p = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc(p, need);
    if (e != cudaSuccess) return bfail(ctx, RT_ENOMEM, std::string(what) + " workspace: " + cudaGetErrorString(e));
    *have = need;
    return RT_OK;
}

int check_grid(rt_ctx* ctx, const rt_grid* g, double R) {
    if (!g) return bfail(ctx, RT_EINVAL, "grid pointer is NULL");
    if (g->nx < 3 || g->ny < 3 || (int64_t)g->nx * g->ny > (int64_t)INT32_MAX / 2)
        return bfail(ctx, RT_EINVAL, "grid size invalid");
    if (!(g->h_mm > 0) || !std::isfinite(g->h_mm) || !std::isfinite(g->x0_mm) || !std::isfinite(g->y0_mm))
        return bfail(ctx, RT_EINVAL, "grid spacing/origin invalid");
    if (!(R > 0) || !std::isfinite(R)) return bfail(ctx, RT_EINVAL, "ring radius must be > 0");
    return RT_OK;
}

// Compact list of the nodes strictly inside the ring (row-major order),
// cached on the context per (grid, radius).
int inside_list(rt_ctx* ctx, const rt_grid& g, double R, cudaStream_t s, int* n_in) {
    const bool same = ctx->born_idx && ctx->born_idx_key[0] == g.nx && ctx->born_idx_key[1] == g.ny &&
                      ctx->born_idx_geo[0] == g.h_mm && ctx->born_idx_geo[1] == g.x0_mm &&
                      ctx->born_idx_geo[2] == g.y0_mm && ctx->born_idx_geo[3] == R;
    if (same) {
        *n_in = ctx->born_n_in;
        return RT_OK;
    }
    if (rt::stream_capturing(s)) return bfail(ctx, RT_EINVAL, "inside-node list must be built outside capture");
    std::vector<int> idx;
    for (int j = 0; j < g.ny; ++j)
        for (int i = 0; i < g.nx; ++i) {
            const double x = g.x0_mm + i * g.h_mm, y = g.y0_mm + j * g.h_mm;
            if (x * x + y * y < R * R) idx.push_back(j * g.nx + i);
        }
    if (idx.empty()) return bfail(ctx, RT_EINVAL, "no grid node inside the ring");
    const int n_inside = (int)idx.size();
    // padded with node 0 to a multiple of 128 plus 128, so that whole tiles of
    // the contraction kernels read valid nodes
    idx.resize(((idx.size() + 127) / 128 + 1) * 128, 0);
    size_t have = ctx->born_idx_bytes;
    int rc = grow(ctx, (void**)&ctx->born_idx, &have, idx.size() * sizeof(int), s, "inside-node");
    if (rc) return rc;
    ctx->born_idx_bytes = have;
    cudaError_t e = cudaMemcpyAsync(ctx->born_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bcuda(ctx, e, "inside-node upload");
    ctx->born_idx_key[0] = g.nx;
    ctx->born_idx_key[1] = g.ny;
    ctx->born_idx_geo[0] = g.h_mm;
    ctx->born_idx_geo[1] = g.x0_mm;
    ctx->born_idx_geo[2] = g.y0_mm;
    ctx->born_idx_geo[3] = R;
    ctx->born_n_in = n_inside;
    *n_in = ctx->born_n_in;
    return RT_OK;
}

int check_born_args(rt_ctx* ctx, const rt_grid* grid, double R, int32_t n_tx, const float* T, const float* A,
                    int32_t n_freq, const double* f_mhz, int32_t mode) {
    int rc = check_grid(ctx, grid, R);
    if (rc) return rc;
    if (n_tx < 2 || n_tx > 65535) return bfail(ctx, RT_EINVAL, "n_tx must be in [2, 65535]");
    if (!T || !A) return bfail(ctx, RT_EINVAL, "T and A maps are required");
    if (n_freq < 0 || (n_freq > 0 && !f_mhz)) return bfail(ctx, RT_EINVAL, "frequencies invalid");
    for (int f = 0; f < n_freq; ++f)
        if (!std::isfinite(f_mhz[f])) return bfail(ctx, RT_EINVAL, "frequency not finite");
    if (mode != RTBORN_GEMM_FP32 && mode != RTBORN_GEMM_TF32X3) return bfail(ctx, RT_EINVAL, "unknown GEMM mode");
    return RT_OK;
}

// SIMT path: per-frequency E and W (or V) [n_tx][n_in] complex64, d^H or the
// adjoint's FP64 accumulator
int born_ws_simt(rt_ctx* ctx, int n_tx, int n_in, cudaStream_t s) {
    const size_t eb = sizeof(float2) * (size_t)n_tx * (size_t)n_in;
    int rc = grow(ctx, &ctx->born_E, &ctx->born_E_bytes, eb, s, "Born E");
    if (!rc) rc = grow(ctx, &ctx->born_W, &ctx->born_W_bytes, eb, s, "Born W");
    if (!rc) rc = grow(ctx, &ctx->born_aux, &ctx->born_aux_bytes,
                       std::max(sizeof(float2) * (size_t)n_tx * n_tx, sizeof(double) * (size_t)n_in), s, "Born aux");
    if (!rc) rc = grow(ctx, &ctx->born_acc, &ctx->born_acc_bytes, sizeof(double) * (size_t)n_in, s, "Born acc");
    return rc;
}

// tensor-core path: the error word and, per launch of up to kBornFreqMax
// frequencies, the apply's partial sums or the adjoint's D' tiles and
// per-frequency node sums
int born_ws_tc(rt_ctx* ctx, int n_tx, int n_in, int n_freq, bool adjoint, cudaStream_t s) {
    const int nf = std::min(n_freq, rt::kBornFreqMax);
    int rc = grow(ctx, &ctx->born_err, &ctx->born_err_bytes, 256, s, "Born error word");
    if (rc) return rc;
    if (!adjoint) return grow(ctx, &ctx->born_acc, &ctx->born_acc_bytes, rt::born_tc_acc_bytes(n_tx, nf), s, "Born sums");
    rc = grow(ctx, &ctx->born_E, &ctx->born_E_bytes, rt::born_tc_bd_bytes(n_tx, nf), s, "Born D' tiles");
    if (!rc) rc = grow(ctx, &ctx->born_aux, &ctx->born_aux_bytes, sizeof(float) * (size_t)nf * n_in, s, "Born sums");
    return rc;
}

// absorption power law: y in [0, 3], frequencies >= 0 and omega_s^y finite in
// FP32 at every frequency
int check_power_law(rt_ctx* ctx, double y, int32_t n_freq, const double* f_mhz) {
    if (!(y >= 0.0 && y <= 3.0)) return bfail(ctx, RT_EINVAL, "power-law exponent y must be in [0, 3]");
    for (int f = 0; f < n_freq; ++f) {
        if (!(f_mhz[f] >= 0.0)) return bfail(ctx, RT_EINVAL, "frequencies must be >= 0 with absorption");
        const double w = std::pow(2.0 * rt::kPiB * f_mhz[f] * 1e6, y);
        if (!(w < 3.0e38)) return bfail(ctx, RT_EINVAL, "omega^y overflows at this frequency and exponent");
    }
    return RT_OK;
}

// per-frequency constants: f = fh + fl (MHz), omega_s^y (y < 0: no
// absorption), omega^2 h^2
rt::BornFreq born_freq(double f_mhz, double h_mm, double y) {
    rt::BornFreq q;
    q.fh = (float)f_mhz;
    q.fl = (float)(f_mhz - (double)q.fh);
    q.wy = y >= 0.0 ? (float)std::pow(2.0 * rt::kPiB * f_mhz * 1e6, y) : 0.f;
    const double om = 2.0 * rt::kPiB * f_mhz;
    q.scale = (float)(om * om * h_mm * h_mm);
    return q;
}

}  // namespace

extern "C" {

int rtborn_maps(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, int32_t fan_rays, float* T_out,
                float* A_out, void* stream) {
    return rtborn_maps_abs(ctx, prob, opt, fan_rays, nullptr, T_out, A_out, nullptr, stream);
}

int rtborn_maps_abs(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, int32_t fan_rays,
                    const double* alpha0, float* T_out, float* A_out, float* L_out, void* stream) {
    if (!ctx) return RT_EINVAL;
    ctx->err.clear();
    cudaStream_t s = (cudaStream_t)stream;
    if (!opt) return bfail(ctx, RT_EINVAL, "options pointer is NULL");
    if (opt->precision != RT_FP32_COMP) return bfail(ctx, RT_EINVAL, "fan maps are computed in RT_FP32_COMP only");
    if (!(opt->ds_mm > 0) || !std::isfinite(opt->ds_mm)) return bfail(ctx, RT_EINVAL, "ds_mm must be > 0");
    if (fan_rays < 2 || fan_rays > (1 << 20)) return bfail(ctx, RT_EINVAL, "fan_rays must be in [2, 2^20]");
    if (opt->integrator != RT_RK4 && opt->integrator != RT_HEUN) return bfail(ctx, RT_EINVAL, "unknown integrator");
    if (opt->interpolator != RT_BILINEAR && opt->interpolator != RT_BSPLINE)
        return bfail(ctx, RT_EINVAL, "unknown interpolator");
    const bool spline = opt->interpolator == RT_BSPLINE;
    if (!T_out || !A_out) return bfail(ctx, RT_EINVAL, "T and A outputs are required");
    if (alpha0 && !L_out) return bfail(ctx, RT_EINVAL, "an alpha0 map needs the L_out output");
    const bool lossy = alpha0 != nullptr;
    if (opt->ds_mm > (prob ? prob->grid.h_mm : 0.0)) return bfail(ctx, RT_EINVAL, "ds_mm must not exceed the grid spacing");
    rt::Geom G;
    int rc = rt::make_geom(ctx, prob, opt, &G);
    if (rc) return rc;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return bcuda(ctx, e, "cudaSetDevice");
    const long long nn = (long long)G.nx * G.ny;
    rc = grow(ctx, &ctx->born_field, &ctx->born_field_bytes, sizeof(rt::BNode) * (size_t)nn, s, "Born field");
    if (rc) return rc;
    const size_t n_ent = (size_t)nn * prob->n_tx;
    const size_t key_bytes = ((lossy ? 2 : 1) * sizeof(unsigned long long) + sizeof(unsigned)) * n_ent;
    rc = grow(ctx, &ctx->born_keys, &ctx->born_keys_bytes, key_bytes, s, "fan-map keys");
    if (rc) return rc;
    unsigned long long* near = (unsigned long long*)ctx->born_keys;
    unsigned long long* lam = lossy ? near + n_ent : nullptr;
    unsigned* tfirst = (unsigned*)(near + (lossy ? 2 : 1) * n_ent);
    e = cudaMemsetAsync(ctx->dflag, 0, sizeof(int), s);
    if (e != cudaSuccess) return bcuda(ctx, e, "flag reset");
    G.bad_field = ctx->dflag;
    const rt::CellBS<float>* bsf = nullptr;
    if (spline) {
        // coefficients and per-cell bicubics of c and s (clears and sets the flag first)
        rc = grow(ctx, (void**)&ctx->bs_coef, &ctx->bs_coef_bytes, 2 * sizeof(double) * (size_t)nn, s, "B-spline");
        if (!rc) rc = grow(ctx, &ctx->born_bsf, &ctx->born_bsf_bytes,
                           sizeof(rt::CellBS<float>) * (size_t)(G.nx - 1) * (size_t)(G.ny - 1), s, "B-spline field");
        if (rc) return rc;
        e = rt::launch_pack_bs(prob->grid, prob->c_mps, ctx->bs_coef, ctx->born_bsf, ctx->dflag, RT_FP32_COMP, s);
        if (e != cudaSuccess) return bcuda(ctx, e, "B-spline pack");
        bsf = (const rt::CellBS<float>*)ctx->born_bsf;
    }
    rt::k_born_pack<<<std::min<long long>((nn + 255) / 256, 152 * 32), 256, 0, s>>>(
        prob->grid, prob->c_mps, alpha0, (rt::BNode*)ctx->born_field, ctx->dflag);
    e = cudaMemsetAsync(ctx->born_keys, 0xff, key_bytes, s);
    if (e != cudaSuccess) return bcuda(ctx, e, "key reset");
    rt::FanArgs A;
    A.K = fan_rays;
    A.hf = (float)G.h;
    A.Hhalf = (float)(0.5 * G.ds / G.h);
    A.eta = RTBORN_ETA_US;
    A.tfirst = tfirst;
    A.near = near;
    A.lam = lam;
    A.nn = nn;
    A.steps = ctx->counters + 7;
    e = cudaMemsetAsync(ctx->counters, 0, 8 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return bcuda(ctx, e, "counter reset");
    const long long rays = (long long)prob->n_tx * fan_rays;
    const rt::BNode* fld = (const rt::BNode*)ctx->born_field;
    // kernel variants: resident 128-thread blocks per SM the kernel is compiled for
    const int minb = opt->blocks_per_sm ? opt->blocks_per_sm : (lossy ? 5 : 6);   // lossy at 6 spills
    const unsigned blocks = (unsigned)((rays + 127) / 128);
    switch (minb) {
#define FAN_V(MB)                                                                               \
    case MB:                                                                                    \
        if (spline) {                                                                           \
            if (lossy) rt::k_born_fan<128, MB, true, true><<<blocks, 128, 0, s>>>(G, A, fld, bsf);   \
            else rt::k_born_fan<128, MB, false, true><<<blocks, 128, 0, s>>>(G, A, fld, bsf);        \
        } else {                                                                                \
            if (lossy) rt::k_born_fan<128, MB, true, false><<<blocks, 128, 0, s>>>(G, A, fld, bsf);  \
            else rt::k_born_fan<128, MB, false, false><<<blocks, 128, 0, s>>>(G, A, fld, bsf);       \
        }                                                                                       \
        break;
        FAN_V(4)
        FAN_V(5)
        FAN_V(6)
        FAN_V(8)
#undef FAN_V
        default:
            return bfail(ctx, RT_EINVAL, "rtborn_maps: blocks_per_sm must be 0 (= 6), 4, 5, 6 or 8");
    }
    rt::k_born_unpack<<<(unsigned)std::min<long long>(((long long)n_ent + 255) / 256, 152 * 64), 256, 0, s>>>(
        tfirst, near, lam, (long long)n_ent, T_out, A_out, lossy ? L_out : nullptr);
    e = cudaGetLastError();
    ctx->last_stream = s;
    return e == cudaSuccess ? RT_OK : bcuda(ctx, e, "fan-map kernels");
}

int rtborn_apply(rt_ctx* ctx, const rt_grid* grid, double ring_radius_mm, int32_t n_tx, const float* T,
                 const float* A, int32_t n_freq, const double* f_mhz, const float* dc_mps, int32_t gemm_mode,
                 float* d_out, void* stream) {
    return rtborn_apply_abs(ctx, grid, ring_radius_mm, n_tx, T, A, nullptr, 0.0, n_freq, f_mhz, dc_mps, gemm_mode,
                            d_out, stream);
}

int rtborn_apply_abs(rt_ctx* ctx, const rt_grid* grid, double ring_radius_mm, int32_t n_tx, const float* T,
                     const float* A, const float* L, double y, int32_t n_freq, const double* f_mhz,
                     const float* dc_mps, int32_t gemm_mode, float* d_out, void* stream) {
    if (!ctx) return RT_EINVAL;
    ctx->err.clear();
    cudaStream_t s = (cudaStream_t)stream;
    int rc = check_born_args(ctx, grid, ring_radius_mm, n_tx, T, A, n_freq, f_mhz, gemm_mode);
    if (rc) return rc;
    if (L && (rc = check_power_law(ctx, y, n_freq, f_mhz))) return rc;
    if (!dc_mps || (!d_out && n_freq > 0)) return bfail(ctx, RT_EINVAL, "dc_mps and d_out are required");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return bcuda(ctx, e, "cudaSetDevice");
    if (n_freq == 0) return RT_OK;
    int n_in = 0;
    rc = inside_list(ctx, *grid, ring_radius_mm, s, &n_in);
    if (rc) return rc;
    const long long nn = (long long)grid->nx * grid->ny;
    float2* d = (float2*)d_out;
    if (gemm_mode == RTBORN_GEMM_TF32X3) {
        if ((rc = born_ws_tc(ctx, n_tx, n_in, n_freq, false, s))) return rc;
        e = cudaMemsetAsync(ctx->born_err, 0, sizeof(int), s);
        for (int f0 = 0; e == cudaSuccess && f0 < n_freq; f0 += rt::kBornFreqMax) {
            const int nf = std::min(n_freq - f0, rt::kBornFreqMax);
            rt::BornFreq fq[rt::kBornFreqMax];
            for (int f = 0; f < nf; ++f) fq[f] = born_freq(f_mhz[f0 + f], grid->h_mm, L ? y : -1.0);
            const rt::BornTCJob job{n_tx, nf, n_in, nn, ctx->born_idx, T, A, L, dc_mps, fq, 0};
            e = rt::launch_born_apply_tc(ctx->device, job, (float*)ctx->born_acc, d + (size_t)f0 * n_tx * n_tx,
                                         (int*)ctx->born_err, s);
        }
        ctx->last_stream = s;
        return e == cudaSuccess ? RT_OK : bcuda(ctx, e, "Born apply kernels");
    }
    if ((rc = born_ws_simt(ctx, n_tx, n_in, s))) return rc;
    float2* E = (float2*)ctx->born_E;
    float2* W = (float2*)ctx->born_W;
    const dim3 eg((n_in + 255) / 256, n_tx);
    e = cudaMemsetAsync(d, 0, sizeof(float2) * (size_t)n_freq * n_tx * n_tx, s);
    for (int f = 0; e == cudaSuccess && f < n_freq; ++f) {
        const rt::BornFreq q = born_freq(f_mhz[f], grid->h_mm, L ? y : -1.0);
        rt::k_born_efield<<<eg, 256, 0, s>>>(n_in, ctx->born_idx, nn, T, A, L, q.wy, q.fh, q.fl, q.scale, dc_mps, E, W);
        // d[e][r] = sum_p E[e][p] W[r][p]
        e = rt::launch_cgemm(n_tx, n_tx, n_in, E, n_in, 1, W, n_in, 1, d + (size_t)f * n_tx * n_tx, n_tx, 1,
                             ctx->device, s);
    }
    if (e == cudaSuccess) {
        rt::k_zero_diag<<<(n_tx * n_freq + 255) / 256, 256, 0, s>>>(d, n_tx, n_freq);
        e = cudaGetLastError();
    }
    ctx->last_stream = s;
    return e == cudaSuccess ? RT_OK : bcuda(ctx, e, "Born apply kernels");
}

int rtborn_adjoint(rt_ctx* ctx, const rt_grid* grid, double ring_radius_mm, int32_t n_tx, const float* T,
                   const float* A, int32_t n_freq, const double* f_mhz, const float* d_in, int32_t gemm_mode,
                   float* dc_out, void* stream) {
    return rtborn_adjoint_abs(ctx, grid, ring_radius_mm, n_tx, T, A, nullptr, 0.0, n_freq, f_mhz, d_in, gemm_mode,
                              dc_out, stream);
}

int rtborn_adjoint_abs(rt_ctx* ctx, const rt_grid* grid, double ring_radius_mm, int32_t n_tx, const float* T,
                       const float* A, const float* L, double y, int32_t n_freq, const double* f_mhz,
                       const float* d_in, int32_t gemm_mode, float* dc_out, void* stream) {
    if (!ctx) return RT_EINVAL;
    ctx->err.clear();
    cudaStream_t s = (cudaStream_t)stream;
    int rc = check_born_args(ctx, grid, ring_radius_mm, n_tx, T, A, n_freq, f_mhz, gemm_mode);
    if (rc) return rc;
    if (L && (rc = check_power_law(ctx, y, n_freq, f_mhz))) return rc;
    if (!dc_out || (!d_in && n_freq > 0)) return bfail(ctx, RT_EINVAL, "d_in and dc_out are required");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return bcuda(ctx, e, "cudaSetDevice");
    const long long nn = (long long)grid->nx * grid->ny;
    e = cudaMemsetAsync(dc_out, 0, sizeof(float) * (size_t)nn, s);
    if (e != cudaSuccess) return bcuda(ctx, e, "dc reset");
    if (n_freq == 0) return RT_OK;
    int n_in = 0;
    rc = inside_list(ctx, *grid, ring_radius_mm, s, &n_in);
    if (rc) return rc;
    const float2* d = (const float2*)d_in;
    if (gemm_mode == RTBORN_GEMM_TF32X3) {
        if ((rc = born_ws_tc(ctx, n_tx, n_in, n_freq, true, s))) return rc;
        e = cudaMemsetAsync(ctx->born_err, 0, sizeof(int), s);
        for (int f0 = 0; e == cudaSuccess && f0 < n_freq; f0 += rt::kBornFreqMax) {
            const int nf = std::min(n_freq - f0, rt::kBornFreqMax);
            rt::BornFreq fq[rt::kBornFreqMax];
            for (int f = 0; f < nf; ++f) fq[f] = born_freq(f_mhz[f0 + f], grid->h_mm, L ? y : -1.0);
            const rt::BornTCJob job{n_tx, nf, n_in, nn, ctx->born_idx, T, A, L, nullptr, fq, 0};
            e = rt::launch_born_adjoint_tc(ctx->device, job, d + (size_t)f0 * n_tx * n_tx, (float*)ctx->born_E,
                                           (float*)ctx->born_aux, dc_out, f0 > 0, (int*)ctx->born_err, s);
        }
        ctx->last_stream = s;
        return e == cudaSuccess ? RT_OK : bcuda(ctx, e, "Born adjoint kernels");
    }
    if ((rc = born_ws_simt(ctx, n_tx, n_in, s))) return rc;
    float2* E = (float2*)ctx->born_E;
    float2* V = (float2*)ctx->born_W;
    float2* Dc = (float2*)ctx->born_aux;
    double* acc = (double*)ctx->born_acc;
    const dim3 eg((n_in + 255) / 256, n_tx);
    for (int f = 0; e == cudaSuccess && f < n_freq; ++f) {
        const rt::BornFreq q = born_freq(f_mhz[f], grid->h_mm, L ? y : -1.0);
        rt::k_born_efield<<<eg, 256, 0, s>>>(n_in, ctx->born_idx, nn, T, A, L, q.wy, q.fh, q.fl, 0.f, nullptr, E,
                                             nullptr);
        rt::k_conj_nodiag<<<(n_tx * n_tx + 255) / 256, 256, 0, s>>>(d + (size_t)f * n_tx * n_tx, Dc, n_tx);
        // V[e][p] = sum_r E[r][p] conj(d[e][r]), conj(d[e][r]) at Dc[e n_tx + r]
        e = cudaMemsetAsync(V, 0, sizeof(float2) * (size_t)n_tx * n_in, s);
        if (e == cudaSuccess)
            e = rt::launch_cgemm(n_in, n_tx, n_tx, E, 1, n_in, Dc, n_tx, 1, V, 1, n_in, ctx->device, s);
        if (e == cudaSuccess) {
            rt::k_born_reduce<<<(n_in + 255) / 256, 256, 0, s>>>(n_in, n_tx, E, V, q.scale, acc, f == 0);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        rt::k_born_scatter<<<(n_in + 255) / 256, 256, 0, s>>>(n_in, ctx->born_idx, acc, dc_out);
        e = cudaGetLastError();
    }
    ctx->last_stream = s;
    return e == cudaSuccess ? RT_OK : bcuda(ctx, e, "Born adjoint kernels");
}

}  // extern "C"
