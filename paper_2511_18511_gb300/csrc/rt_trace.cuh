// rt_trace.cuh — device-side ray tracer for the two-point ray-tracing library.
//
// One ray per thread. The sound-speed field is packed per node as
// (c, h*dc/dx, h*dc/dy, s=1/c) (float4 or 32-byte double4), L2-resident, and
// sampled bilinearly (paper Sec. 3.3.1: field and gradient are interpolated
// from the four vertices of the enclosing cell). Positions are kept
// cell-local: an integer cell (ci, cj) plus a fraction in [0, 1) per axis,
// so FP32 keeps ~1e-8 of a cell of resolution anywhere on a 1024^2 grid. The
// current cell's bilinear coefficients are cached in registers and reloaded
// only when a sample falls in another cell (about once per 8 steps at
// ds = h/10), which turns the march from L2-gather-bound into FMA-bound.
//
// Ray equations (paper Sec. 3.2.3: x and unit d evolve from the sound speed
// and its gradient), written in cell units s~ = s/h:
//     dX/ds~ = d,    dd/ds~ = -(g - (g.d) d) / c,    g = h grad c,
// marched with classic RK4 at a fixed step and d renormalised after each step.
// A trace ends at the first step (after the first) that ends on or outside the
// ring |x| = R; the last point is replaced by the boundary interception, reached
// by a shortened RK4 step ds' (paper Sec. 4.2), found from the chord-circle
// root plus two Newton corrections in FP64. The travel time is the trapezoid
// rule over the points with the interpolated slowness plus the first-order
// endpoint correction s(x_M) d_M.(x_r - x_M) (Appendix: grad T.grad T = c^-2,
// so grad T = s d along the ray).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rt {

struct __align__(32) D4 {
    double x, y, z, w;
};

template <typename T> struct Vec4T;
template <> struct Vec4T<float> { using type = float4; };
template <> struct Vec4T<double> { using type = D4; };

// Bilinear coefficients of one grid cell for the four sampled fields
// (c, h dc/dx, h dc/dy, s): f(tx, ty) = a + tx bx + ty (by + tx bxy), each field
// one vector (a, bx, by, bxy). Cell (i, j) spans nodes i..i+1, j..j+1 and is
// stored at j*(nx-1) + i. A cell reload is four contiguous vector loads.
template <typename T>
struct CellCoef {
    typename Vec4T<T>::type c, gx, gy, s;
};

template <typename T> struct NodeT { using type = CellCoef<T>; };

// Per-launch geometry (kernel parameter).
struct Geom {
    int nx, ny;
    double h, x0, y0, R;
    double inv_R2;          // 1 / R^2
    int heun;               // 1: Heun's second-order Runge-Kutta, 0: classic RK4
    int interp;             // enum rt_interpolator of the packed field
    double ds;              // mm
    int Ox, Oy;             // floor of the ring centre in cell coordinates (-x0/h, -y0/h)
    double oxf, oyf;        // fractional parts of the ring centre
    long long Q;            // floor((R/h)^2)
    double q;               // (R/h)^2 - Q
    long long max_steps;    // ceil(8 R / ds)
    int max_steps_i;
    const double* tx;       // [2 n_tx]
    int n_tx;
    const int* pairs;       // [2 n_pairs] or null
    int n_pairs;
    const int* bad_field;   // device flag set by the pack kernel (c <= 0 or NaN)
    const double* tx_phi;   // [n_tx] polar angle of each transducer, NaN if off the ring; null = compute
    // FP32 copies of the per-step constants, so the FP32 march issues no FP64
    float Hf, dsf, Rcf, oxff, oyff, qf;
    int Qi;                 // Q as 32-bit (grids up to 32k cells per side)
};

// Per-step constants in the marching precision.
template <typename T> struct StepK;
template <> struct StepK<float> {
    __device__ __forceinline__ static float H(const Geom& G) { return G.Hf; }
    __device__ __forceinline__ static float ds(const Geom& G) { return G.dsf; }
    __device__ __forceinline__ static float Rc(const Geom& G) { return G.Rcf; }
    __device__ __forceinline__ static float oxf(const Geom& G) { return G.oxff; }
    __device__ __forceinline__ static float oyf(const Geom& G) { return G.oyff; }
    __device__ __forceinline__ static float q(const Geom& G) { return G.qf; }
};
template <> struct StepK<double> {
    __device__ __forceinline__ static double H(const Geom& G) { return G.ds / G.h; }
    __device__ __forceinline__ static double ds(const Geom& G) { return G.ds; }
    __device__ __forceinline__ static double Rc(const Geom& G) { return G.R / G.h; }
    __device__ __forceinline__ static double oxf(const Geom& G) { return G.oxf; }
    __device__ __forceinline__ static double oyf(const Geom& G) { return G.oyf; }
    __device__ __forceinline__ static double q(const Geom& G) { return G.q; }
};

__device__ __forceinline__ void pair_of(const Geom& G, int k, int& e, int& r) {
    if (G.pairs) {
        e = G.pairs[2 * k];
        r = G.pairs[2 * k + 1];
    } else {
        int n1 = G.n_tx - 1;
        e = k / n1;
        int rr = k - e * n1;
        r = rr + (rr >= e);
    }
}

// 1/c for the ray equations: the hardware approximation (about 1 ulp) in FP32.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double rcp_approx(double x) { return 1.0 / x; }

// ---------------------------------------------------------------- field cache

// The cell (i, j) and in-cell fractions (tx, ty) of a point given by fractions
// (u, v) relative to cell (ci, cj); returns whether (i, j) differs from the
// cached cell (pi, pj). Stage points lie within one cell of the current one
// when ds <= h, so the offsets come from comparisons (no conversion
// instructions, which are slow on this part); larger offsets take the floor path.
template <typename T>
__device__ __forceinline__ bool cell_locate(int ci, int cj, T u, T v, int pi, int pj, int& i, int& j, T& tx,
                                            T& ty) {
    if (ci == pi && cj == pj && u >= (T)0 && u < (T)1 && v >= (T)0 && v < (T)1) {
        tx = u;
        ty = v;
        return false;
    }
    if (u >= (T)-1 && u < (T)2 && v >= (T)-1 && v < (T)2) {
        const bool ul = u < (T)0, uh = u >= (T)1, vl = v < (T)0, vh = v >= (T)1;
        tx = ul ? u + (T)1 : (uh ? u - (T)1 : u);
        ty = vl ? v + (T)1 : (vh ? v - (T)1 : v);
        i = ci + (ul ? -1 : (uh ? 1 : 0));
        j = cj + (vl ? -1 : (vh ? 1 : 0));
    } else {
        const T fu = floor(u), fv = floor(v);
        i = ci + (int)fu;
        j = cj + (int)fv;
        tx = u - fu;
        ty = v - fv;
    }
    return i != pi || j != pj;
}

template <typename T>
struct Cell {
    using V = CellCoef<T>;
    const V* __restrict__ F;
    int nx, ny;
    int pi, pj;                       // cached cell
    T ca, cbx, cby, cbxy;             // c      = ca + tx cbx + ty (cby + tx cbxy)
    T xa, xbx, xby, xbxy;             // h dc/dx
    T ya, ybx, yby, ybxy;             // h dc/dy
    T sa, sbx, sby, sbxy;             // s

    __device__ __forceinline__ void load(int i, int j) {
        pi = i;
        pj = j;
        // clamp for memory safety; rays stay inside by the ring/grid check
        i = min(max(i, 0), nx - 2);
        j = min(max(j, 0), ny - 2);
        const V* p = F + (size_t)j * (nx - 1) + i;
        const auto c = p->c, x = p->gx, y = p->gy, w = p->s;
        ca = c.x; cbx = c.y; cby = c.z; cbxy = c.w;
        xa = x.x; xbx = x.y; xby = x.z; xbxy = x.w;
        ya = y.x; ybx = y.y; yby = y.z; ybxy = y.w;
        sa = w.x; sbx = w.y; sby = w.z; sbxy = w.w;
    }

    // (u, v): fractions relative to cell (ci, cj), possibly outside [0, 1)
    __device__ __forceinline__ void at(int ci, int cj, T u, T v, T& c, T& gx, T& gy, T& tx, T& ty) {
        int i, j;
        if (cell_locate(ci, cj, u, v, pi, pj, i, j, tx, ty)) load(i, j);
        c = ca + tx * cbx + ty * (cby + tx * cbxy);
        gx = xa + tx * xbx + ty * (xby + tx * xbxy);
        gy = ya + tx * ybx + ty * (yby + tx * ybxy);
    }

    // slowness at fractions (tx, ty) of the cached cell
    __device__ __forceinline__ T slow(T tx, T ty) const { return sa + tx * sbx + ty * (sby + tx * sbxy); }
};

// ---------------------------------------------------------------- direction

template <typename T> struct Dir;

// FP64: plain unit vector
template <> struct Dir<double> {
    double x, y;
    __device__ __forceinline__ void set(double th) { sincos(th, &y, &x); }
    __device__ __forceinline__ void set_cs(double c, double s) { x = c; y = s; }
    __device__ __forceinline__ double hx() const { return x; }
    __device__ __forceinline__ double hy() const { return y; }
    __device__ __forceinline__ double lx() const { return 0.0; }
    __device__ __forceinline__ double ly() const { return 0.0; }
    __device__ __forceinline__ void add_normalize(double ix, double iy) {
        x += ix;
        y += iy;
        double n = sqrt(x * x + y * y);
        x /= n;
        y /= n;
    }
    __device__ __forceinline__ double dx() const { return x; }
    __device__ __forceinline__ double dy() const { return y; }
};

// FP32-compensated: double-float unit vector (hi + lo), so that thousands of
// small RK4 increments do not random-walk the ray angle by FP32 rounding.
template <> struct Dir<float> {
    float x, y, ex, ey;   // value = (x + ex, y + ey)
    __device__ __forceinline__ void set(double th) {
        double c, s;
        sincos(th, &s, &c);
        set_cs(c, s);
    }
    __device__ __forceinline__ void set_cs(double c, double s) {
        x = (float)c; ex = (float)(c - (double)x);
        y = (float)s; ey = (float)(s - (double)y);
    }
    __device__ __forceinline__ float hx() const { return x; }
    __device__ __forceinline__ float hy() const { return y; }
    __device__ __forceinline__ float lx() const { return ex; }
    __device__ __forceinline__ float ly() const { return ey; }
    __device__ __forceinline__ void add_normalize(float ix, float iy) {
        // two-sum of hi + increment, error into lo
        float s = x + ix, bb = s - x;
        ex += (x - (s - bb)) + (ix - bb);
        x = s;
        s = y + iy; bb = s - y;
        ey += (y - (s - bb)) + (iy - bb);
        y = s;
        // |d|^2 - 1 to first order in lo, then d *= 1/sqrt(1+e) = 1 + delta
        float e = fmaf(x, x, fmaf(y, y, -1.0f)) + 2.0f * (x * ex + y * ey);
        float delta = e * fmaf(0.375f, e, -0.5f);
        ex = fmaf(x + ex, delta, ex);
        ey = fmaf(y + ey, delta, ey);
        // renormalise the hi/lo split (fast two-sum, |hi| >= |lo|)
        s = x + ex; ex -= s - x; x = s;
        s = y + ey; ey -= s - y; y = s;
    }
    __device__ __forceinline__ double dx() const { return (double)x + (double)ex; }
    __device__ __forceinline__ double dy() const { return (double)y + (double)ey; }
};

// ---------------------------------------------------------------- RK4 in cell units

template <typename T>
struct RayState {
    int ci, cj;
    T fx, fy;      // fraction of the cell
    T lx, ly;      // FP32: rounding residual of the fraction (two-sum), FP64: 0
    Dir<T> d;
};

// fraction += inc, keeping the rounding error in the residual (FP32 only)
__device__ __forceinline__ void add_frac(float& f, float& lo, float inc) {
    const float s = f + inc, bb = s - f;
    lo += (f - (s - bb)) + (inc - bb);
    const float s2 = s + lo;
    lo -= s2 - s;
    f = s2;
}
__device__ __forceinline__ void add_frac(double& f, double&, double inc) { f += inc; }

// (g.e) e - g over c for stage direction e
template <typename T>
__device__ __forceinline__ void ray_rhs(T c, T gx, T gy, T ex, T ey, T& kx, T& ky) {
    T ic = rcp_approx(c);
    T gd = gx * ex + gy * ey;
    kx = (gd * ex - gx) * ic;
    ky = (gd * ey - gy) * ic;
}

// One RK4 step of length H (cell units) from S into N. s_here receives the
// slowness at S's position (stage-1 sample) for the trapezoid rule.
template <typename T, typename CellT>
__device__ __forceinline__ void rk4_step(CellT& C, const RayState<T>& S, T H, RayState<T>& N, T& s_here,
                                         T& tx1, T& ty1, int& i1, int& j1) {
    const T Hh = (T)0.5 * H, H6 = H / (T)6;
    const T dx = S.d.hx(), dy = S.d.hy();
    T c, gx, gy, tx, ty, k1x, k1y, k2x, k2y, k3x, k3y, k4x, k4y;
    C.at(S.ci, S.cj, S.fx, S.fy, c, gx, gy, tx1, ty1);
    i1 = C.pi;
    j1 = C.pj;
    s_here = C.slow(tx1, ty1);
    ray_rhs(c, gx, gy, dx, dy, k1x, k1y);
    T e2x = dx + Hh * k1x, e2y = dy + Hh * k1y;
    C.at(S.ci, S.cj, S.fx + Hh * dx, S.fy + Hh * dy, c, gx, gy, tx, ty);
    ray_rhs(c, gx, gy, e2x, e2y, k2x, k2y);
    T e3x = dx + Hh * k2x, e3y = dy + Hh * k2y;
    C.at(S.ci, S.cj, S.fx + Hh * e2x, S.fy + Hh * e2y, c, gx, gy, tx, ty);
    ray_rhs(c, gx, gy, e3x, e3y, k3x, k3y);
    T e4x = dx + H * k3x, e4y = dy + H * k3y;
    C.at(S.ci, S.cj, S.fx + H * e3x, S.fy + H * e3y, c, gx, gy, tx, ty);
    ray_rhs(c, gx, gy, e4x, e4y, k4x, k4y);
    // every stage direction carries the low part of d, so the position
    // increment gets it in full: H d_lo (zero in FP64); the fraction is
    // accumulated with its rounding residual in FP32
    T nfx = S.fx, nfy = S.fy;
    N.lx = S.lx;
    N.ly = S.ly;
    add_frac(nfx, N.lx, H6 * (dx + (T)2 * (e2x + e3x) + e4x) + H * S.d.lx());
    add_frac(nfy, N.ly, H6 * (dy + (T)2 * (e2y + e3y) + e4y) + H * S.d.ly());
    N.d = S.d;
    N.d.add_normalize(H6 * (k1x + (T)2 * (k2x + k3x) + k4x), H6 * (k1y + (T)2 * (k2y + k3y) + k4y));
    N.ci = S.ci;
    N.cj = S.cj;
    // f - 1 is exact for f in [1, 2); f + 1 for f in [-1, 0) rounds, so it goes
    // through the residual too
    if (nfx >= (T)1) { N.ci += 1; nfx -= (T)1; } else if (nfx < (T)0) { N.ci -= 1; add_frac(nfx, N.lx, (T)1); }
    if (nfy >= (T)1) { N.cj += 1; nfy -= (T)1; } else if (nfy < (T)0) { N.cj -= 1; add_frac(nfy, N.ly, (T)1); }
    N.fx = nfx;
    N.fy = nfy;
}

// One step of Heun's second-order Runge-Kutta method (the slopes at S and at
// the Euler end point S + H (d, k1), averaged), in the same cell-unit,
// compensated form as rk4_step.
template <typename T, typename CellT>
__device__ __forceinline__ void heun_step(CellT& C, const RayState<T>& S, T H, RayState<T>& N, T& s_here,
                                          T& tx1, T& ty1, int& i1, int& j1) {
    const T Hh = (T)0.5 * H;
    const T dx = S.d.hx(), dy = S.d.hy();
    T c, gx, gy, tx, ty, k1x, k1y, k2x, k2y;
    C.at(S.ci, S.cj, S.fx, S.fy, c, gx, gy, tx1, ty1);
    i1 = C.pi;
    j1 = C.pj;
    s_here = C.slow(tx1, ty1);
    ray_rhs(c, gx, gy, dx, dy, k1x, k1y);
    const T e2x = dx + H * k1x, e2y = dy + H * k1y;
    C.at(S.ci, S.cj, S.fx + H * dx, S.fy + H * dy, c, gx, gy, tx, ty);
    ray_rhs(c, gx, gy, e2x, e2y, k2x, k2y);
    T nfx = S.fx, nfy = S.fy;
    N.lx = S.lx;
    N.ly = S.ly;
    add_frac(nfx, N.lx, Hh * (dx + e2x) + H * S.d.lx());
    add_frac(nfy, N.ly, Hh * (dy + e2y) + H * S.d.ly());
    N.d = S.d;
    N.d.add_normalize(Hh * (k1x + k2x), Hh * (k1y + k2y));
    N.ci = S.ci;
    N.cj = S.cj;
    if (nfx >= (T)1) { N.ci += 1; nfx -= (T)1; } else if (nfx < (T)0) { N.ci -= 1; add_frac(nfx, N.lx, (T)1); }
    if (nfy >= (T)1) { N.cj += 1; nfy -= (T)1; } else if (nfy < (T)0) { N.cj -= 1; add_frac(nfy, N.ly, (T)1); }
    N.fx = nfx;
    N.fy = nfy;
}

// The step of the configured integrator (uniform over a launch).
template <typename T, typename CellT>
__device__ __forceinline__ void ray_step(CellT& C, const Geom& G, const RayState<T>& S, T H, RayState<T>& N,
                                         T& s_here, T& tx1, T& ty1, int& i1, int& j1) {
    if (G.heun) heun_step(C, S, H, N, s_here, tx1, ty1, i1, j1);
    else rk4_step(C, S, H, N, s_here, tx1, ty1, i1, j1);
}

// |x|^2 - (R/h)^2 in cell^2 units, exact integer part plus a small fractional
// part, so the sign is reliable to ~1e-7 cell even in FP32.
template <typename T>
__device__ __forceinline__ T ring_excess(const Geom& G, const RayState<T>& S) {
    const int Ix = S.ci - G.Ox, Iy = S.cj - G.Oy;
    const T px = S.fx - StepK<T>::oxf(G), py = S.fy - StepK<T>::oyf(G);
    const int I2 = Ix * Ix + Iy * Iy - G.Qi;
    const T d0 = (T)I2 - StepK<T>::q(G);
    return d0 + (T)2 * ((T)Ix * px + (T)Iy * py) + px * px + py * py;
}

template <typename T>
__device__ __forceinline__ void abs_pos(const Geom& G, const RayState<T>& S, double& X, double& Y) {
    X = G.x0 + G.h * ((double)S.ci + ((double)S.fx + (double)S.lx));
    Y = G.y0 + G.h * ((double)S.cj + ((double)S.fy + (double)S.ly));
}

// ---------------------------------------------------------------- scatter (adjoint / matrix rows)

// Exact float -> double by integer bit operations (normal numbers; zeros and
// subnormals give +-0), avoiding a conversion instruction.
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned ex = (u >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    if (ex == 0) return __longlong_as_double((long long)sign);
    if (ex == 0xffu)   // inf / NaN keep their class
        return __longlong_as_double((long long)(sign | (0x7ffull << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
    const unsigned long long bits = sign | ((unsigned long long)(ex + 896u) << 52) |
                                    ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double to_double(float f) { return f2d_bits(f); }
__device__ __forceinline__ double to_double(double d) { return d; }

// Accumulates the trapezoid-weighted bilinear weights of consecutive points
// that fall in one cell, as (sum w, sum w tx, sum w ty, sum w tx ty).
template <typename T>
struct CellAcc {
    int ai, aj;
    T W, Wx, Wy, Wxy;
    __device__ __forceinline__ void reset() { ai = INT_MIN; aj = INT_MIN; W = Wx = Wy = Wxy = (T)0; }
    __device__ __forceinline__ void node_weights(double& w00, double& w10, double& w01, double& w11) const {
        w11 = (double)Wxy;
        w10 = (double)Wx - w11;
        w01 = (double)Wy - w11;
        w00 = (double)W - (double)Wx - (double)Wy + w11;
    }
};

// Trace outcome.
struct TraceOut {
    double T;          // travel time (us) incl. endpoint correction
    double hx, hy;     // interception
    int flags;         // bit0: step cap, bit1: left outward at once
    long long steps;   // RK4 steps taken (incl. landing)
};

// Sink interface used by trace(): add(ci, cj, tx, ty, w) for each point.
struct NoSink {
    template <typename T>
    __device__ __forceinline__ void add(int, int, T, T, T) {}
    __device__ __forceinline__ void finish() {}
};

// Resumable trace: begin / step (until it reports the end) / end. The
// persistent linking kernel interleaves traces of different pairs per lane.
template <typename T>
struct TraceState {
    RayState<T> S;
    T s_first, s_cur;
    T Ssum, Scomp;            // Kahan sum of s at points 1..M-1
    int m;                    // index of the current point
    int safe;                 // steps that cannot reach the ring (exit test skipped)
    int flags;                // bit0 step cap, bit1 left outward at once
    int iL, jL;               // cell and fractions of the last full-step point
    T txL, tyL;
    int steps;                // RK4 steps of this trace (incl. landing)
};

// Starts a trace at (xe, ye) with unit launch direction (c, s).
template <typename T>
__device__ __forceinline__ void trace_begin_cs(TraceState<T>& ts, const Geom& G, double xe, double ye, double c,
                                               double s) {
    const double u = (xe - G.x0) / G.h, v = (ye - G.y0) / G.h;
    const double fu = floor(u), fv = floor(v);
    ts.S.ci = (int)fu;
    ts.S.cj = (int)fv;
    ts.S.fx = (T)(u - fu);
    ts.S.fy = (T)(v - fv);
    ts.S.lx = (T)((u - fu) - (double)ts.S.fx);
    ts.S.ly = (T)((v - fv) - (double)ts.S.fy);
    ts.S.d.set_cs(c, s);
    ts.s_first = ts.s_cur = (T)0;
    ts.Ssum = ts.Scomp = (T)0;
    ts.m = 0;
    ts.safe = 0;
    ts.flags = 0;
    ts.iL = ts.jL = 0;
    ts.txL = ts.tyL = (T)0;
    ts.steps = 0;
}

template <typename T>
__device__ __forceinline__ void trace_begin(TraceState<T>& ts, const Geom& G, double xe, double ye, double theta) {
    double c, s;
    sincos(theta, &s, &c);
    trace_begin_cs(ts, G, xe, ye, c, s);
}

// One RK4 step. Returns true when the trace has ended: the step ended on or
// outside the ring (flags bit1 if that was the very first step) or the step
// cap was reached (flags bit0). On exit ts.S is still the last inside point.
template <typename T, typename CellT, typename Sink>
__device__ __forceinline__ bool trace_step(CellT& C, const Geom& G, TraceState<T>& ts, Sink& sink) {
    if (ts.m >= G.max_steps_i) {
        ts.flags |= 1;
        return true;
    }
    const T H = StepK<T>::H(G);
    const T dsT = StepK<T>::ds(G);
    RayState<T> N;
    T tx1, ty1;
    int i1, j1;
    ray_step(C, G, ts.S, H, N, ts.s_cur, tx1, ty1, i1, j1);
    ++ts.steps;
    bool ends_out = false;
    if (--ts.safe < 0) {
        const T ex = ring_excess(G, N);
        ends_out = ex >= (T)0;
        if (!ends_out) {
            // distance to the ring in cells, -ex / (R + r); no step moves farther than ~H
            const T Rc = StepK<T>::Rc(G);
            const T r = sqrt(Rc * Rc + ex);
            const T dist = -ex / (Rc + r);
            ts.safe = (int)(dist * (T)0.98 / H) - 1;
        }
    }
    if (ts.m == 0) {
        if (ends_out) {   // left outward: no path, no weights
            ts.flags |= 2;
            return true;
        }
        ts.s_first = ts.s_cur;
        sink.add(i1, j1, tx1, ty1, (T)0.5 * dsT);
    } else {
        const T y = ts.s_cur - ts.Scomp;
        const T t = ts.Ssum + y;
        ts.Scomp = (t - ts.Ssum) - y;
        ts.Ssum = t;
        sink.add(i1, j1, tx1, ty1, dsT);
        if (ends_out) {
            ts.iL = i1; ts.jL = j1; ts.txL = tx1; ts.tyL = ty1;
            return true;
        }
    }
    ts.S = N;
    ++ts.m;
    return false;
}

// Landing, travel time and final weights of an ended trace. The endpoint
// correction is taken toward (xr, yr).
template <typename T, typename CellT, typename Sink>
__device__ TraceOut trace_end(CellT& C, const Geom& G, TraceState<T>& ts, double xe, double ye, double xr,
                              double yr, Sink& sink) {
    TraceOut out;
    out.flags = ts.flags;
    if (ts.flags & 1) {
        // step cap: no interception; report the current point
        abs_pos(G, ts.S, out.hx, out.hy);
        out.T = G.ds * (0.5 * (double)ts.s_first + ((double)ts.Ssum - (double)ts.Scomp));
        out.steps = ts.steps;
        sink.finish();
        return out;
    }
    if (ts.flags & 2) {
        out.T = 0.0;
        out.hx = xe;
        out.hy = ye;
        out.steps = ts.steps;
        sink.finish();
        return out;
    }
    const RayState<T>& S = ts.S;
    RayState<T> N;
    double X, Y;
    abs_pos(G, S, X, Y);
    double b = X * S.d.dx() + Y * S.d.dy();
    double qq = X * X + Y * Y - G.R * G.R;
    double disc = b * b - qq;
    if (disc < 0) disc = 0;
    double sq = sqrt(disc);
    double t = (b >= 0) ? (-qq) / (b + sq) : (sq - b);
    if (!(t >= 0)) t = 0;
    if (t > G.ds) t = G.ds;
    T s_dummy, txd, tyd;
    int id, jd;
    for (int it = 0; it < 2; ++it) {
        ray_step(C, G, S, (T)(t / G.h), N, s_dummy, txd, tyd, id, jd);
        ++ts.steps;
        double NX, NY;
        abs_pos(G, N, NX, NY);
        double r = sqrt(NX * NX + NY * NY);
        double drdt = (NX * N.d.dx() + NY * N.d.dy()) / r;
        if (drdt > 0) t -= (r - G.R) / drdt;
        if (!(t >= 0)) t = 0;
        if (t > G.ds) t = G.ds;
    }
    ray_step(C, G, S, (T)(t / G.h), N, s_dummy, txd, tyd, id, jd);
    ++ts.steps;
    double MX, MY;
    abs_pos(G, N, MX, MY);
    T c_, gx_, gy_, txM, tyM;
    C.at(N.ci, N.cj, N.fx, N.fy, c_, gx_, gy_, txM, tyM);
    const int iM = C.pi, jM = C.pj;
    const double sM = (double)C.slow(txM, tyM);
    const double sL = (double)ts.s_cur;   // slowness at x_{M-1}
    const double corr = N.d.dx() * (xr - MX) + N.d.dy() * (yr - MY);
    const double S_int = (double)ts.Ssum - (double)ts.Scomp;   // s_1 + ... + s_{M-1}
    out.T = G.ds * (0.5 * (double)ts.s_first + S_int - 0.5 * sL) + 0.5 * t * (sL + sM) + sM * corr;
    out.hx = MX;
    out.hy = MY;
    out.steps = ts.steps;
    // alpha_{M-1} = (ds + ds')/2 (ds was given by trace_step), alpha_M = ds'/2 + corr
    sink.add(ts.iL, ts.jL, ts.txL, ts.tyL, (T)(0.5 * (t - G.ds)));
    sink.add(iM, jM, txM, tyM, (T)(0.5 * t + corr));
    sink.finish();
    return out;
}

// Traces one ray from (xe, ye) at angle theta (begin + steps + end). With a
// sink, every sample point m reports its trapezoid weight alpha_m (and the
// endpoint weight) with its cell and fractions.
template <typename T, typename CellT, typename Sink>
__device__ TraceOut trace_ray(CellT& C, const Geom& G, double xe, double ye, double theta, double xr,
                              double yr, Sink& sink) {
    TraceState<T> ts;
    trace_begin(ts, G, xe, ye, theta);
    while (!trace_step(C, G, ts, sink)) {
    }
    return trace_end(C, G, ts, xe, ye, xr, yr, sink);
}

}  // namespace rt
