/*
 * FP64 CPU oracle for the ray-Born operator: per-transducer travel-time and
 * amplitude maps from ray fans traced with their paraxial rays, and the
 * linearised Born map and its adjoint.
 *
 * TEST INFRASTRUCTURE ONLY, like oracle.c: the tests, the smoke check and the
 * benchmark's CPU legs call it, the library never does, and it shares no code
 * with the CUDA path. Plain FP64, one fan per OpenMP iteration, every sample
 * interpolated afresh.
 *
 * arXiv:2511.18511 states the model (Sec. 3.5 and the Appendix: a Green's
 * function g = A exp(i phi) whose phase follows the eikonal and whose
 * geometric amplitude follows the transport equation through the ray Jacobian
 * of a paraxial ray); the discretisation below is this oracle's reading of it:
 *   B1 fields: nodal c, gradient (central differences, one-sided at edges, as
 *      in oracle.c), slowness s = 1/c, and the Hessian of c by central second
 *      differences (zero on the outermost nodes, which rays never reach); all
 *      seven interpolated bilinearly, as Sec. 3.3.1 does for c and its gradient;
 *   B2 fan: per transducer, K rays at evenly spaced angles over the inward
 *      half-plane, the two tangent directions excluded by a margin ds/R (the
 *      same fan as the linking's cold start);
 *   B3 march: classic RK4 (or, with orc_set_integrator(1), Heun's RK2, the
 *      paper's default) at fixed ds on (x, d, Q, P) together, with
 *      dx/ds = d, dd/ds = -(grad c - (grad c . d) d)/c and the paraxial pair
 *      dQ/ds = c P, dP/ds = -(c_nn / c^2) Q, c_nn = n^T H n for the unit normal
 *      n of d (Sec. 3.5, paraxial ray, default); Q(0) = 0, P(0) = 1/c_t with c_t
 *      the sound speed at the transducer; d renormalised after every step; the
 *      ray stops at the first step that ends on or outside the ring, and that
 *      end point is not used; travel time by the trapezoid rule over the
 *      interpolated slowness, as for the ToF;
 *   B4 amplitude (2D transport equation): A = sqrt(c(x) / (c_t max(|Q|, h)));
 *      the clamp at the grid spacing h bounds it at the source and at caustics;
 *   B5 maps: every sample point after the transducer offers each node of the
 *      3 x 3 block around its nearest node whose foot on the ray lies within
 *      half a step of it (a = d_m.D in [-ds/2, ds/2), D = node - sample,
 *      b = n_m.D) the travel time extrapolated to second order in the
 *      ray-centred frame, T_m + s_m a + (M / 2) b^2, with M = P/Q_f the
 *      curvature of the paraxial wavefront at the foot, Q_f = Q_m + a c_m P_m
 *      (for M < 0, a converging front, |Q_f| is clamped to >= h so that a focus
 *      cannot send the time to -inf), with the amplitude A from Q_f. A node's
 *      travel time is its earliest candidate (first arrival). Its amplitude is
 *      that of the candidate of least T + eta (b/h)^2 (ties to the smaller A):
 *      rays next to a node arrive within far less than any rounding of T of
 *      one another, so the earliest alone would pick among them by rounding,
 *      while their amplitudes differ by the spreading across the fan; the
 *      penalty eta (b/h)^2 (eta = 1e-2 us) takes the ray passing closest to
 *      the node; since the first-arrival branch passes within half a ray
 *      spacing (< h/2) of every node it reaches, another branch can supply A
 *      only if it arrives less than eta/4 after the first (a phase of 0.02 rad
 *      at 1.5 MHz). Unreached nodes keep T = +inf, A = 0;
 *   B6 Born map, per frequency f (MHz; omega = 2 pi f rad/us):
 *      d[f][e][r] = omega^2 h^2 sum_x E_e(x) E_r(x) dc(x) for e != r, 0 for
 *      e == r, E_t = A_t exp(i omega T_t) (0 where unreached), x over the nodes
 *      strictly inside the ring (dc in m/s as given);
 *   B7 adjoint under Re<a, b> = Re sum conj(a) b on the data and the plain dot
 *      product on dc: dc~(x) = Re sum_f omega^2 h^2 sum_{e != r}
 *      conj(E_e(x) E_r(x)) d[f][e][r], 0 outside the ring;
 *   B9 absorption (the Appendix: complex wavenumber k + i alpha with the power
 *      law alpha = alpha0 omega^y, alpha0 varying in space, in Np (rad/s)^-y
 *      m^-1; the absorption amplitude is accumulated along the ray, A =
 *      A_geom A_abs): nodal alpha0 interpolated bilinearly, its path integral
 *      Lambda = int alpha0 ds (ds in metres) by the trapezoid rule over the
 *      sample points, carried to a node from its foot to first order
 *      (Lambda + alpha0 a), and taken from the candidate that supplies A; then
 *      A_abs = exp(-omega_s^y Lambda) with omega_s = 2 pi f in rad/s, so
 *      E_t = A_t exp(-omega_s^y Lambda_t) exp(i omega T_t). Without alpha0,
 *      Lambda = 0 (the maps of B1-B5 exactly);
 *   B10 with orc_set_interpolator(1) (the paper's choice for ray-Born, Sec.
 *      3.3.1: the cubic B-spline gives analytic first and second derivatives)
 *      c, its gradient and its Hessian are the interpolating B-spline of the
 *      nodal c and its exact derivatives, and s is the spline of the nodal s
 *      (the spline of oracle.c's readings S1 and S4: coefficients from
 *      orc_bspline_coef, 4 x 4 per sample, mirror at the edges); alpha0 stays
 *      bilinear.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "oracle.h"

enum { F_C, F_GX, F_GY, F_S, F_HXX, F_HXY, F_HYY, F_AL, F_N };

typedef struct {
    int nx, ny;
    double h, x0, y0;
    double* v[F_N]; /* nodal fields, [ny*nx] each */
    double *ac, *as; /* B10: spline coefficients of c and s, or NULL */
} BField;

static void bfield_free(BField* F) {
    for (int q = 0; q < F_N; ++q) free(F->v[q]);
    free(F->ac);
    free(F->as);
    memset(F, 0, sizeof(*F));
}

/* B1 (and B9: alpha0 as given, or 0) */
static int bfield_make(BField* F, const orc_grid* g, const double* c_mps, const double* alpha0) {
    memset(F, 0, sizeof(*F));
    if (!g || !c_mps || g->nx < 3 || g->ny < 3 || !(g->h > 0)) return ORC_EINVAL;
    const int nx = g->nx, ny = g->ny;
    const double h = g->h;
    F->nx = nx; F->ny = ny; F->h = h; F->x0 = g->x0; F->y0 = g->y0;
    const size_t n = (size_t)nx * ny;
    for (int q = 0; q < F_N; ++q) {
        F->v[q] = calloc(n, sizeof(double));
        if (!F->v[q]) { bfield_free(F); return ORC_ENOMEM; }
    }
    double* c = F->v[F_C];
    for (size_t k = 0; k < n; ++k) {
        if (!(c_mps[k] > 0) || !isfinite(c_mps[k])) { bfield_free(F); return ORC_EINVAL; }
        c[k] = 1e-3 * c_mps[k];
        F->v[F_S][k] = 1.0 / c[k];
        if (alpha0) {
            if (!(alpha0[k] >= 0) || !isfinite(alpha0[k])) { bfield_free(F); return ORC_EINVAL; }
            F->v[F_AL][k] = alpha0[k];
        }
    }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const size_t k = (size_t)j * nx + i;
            F->v[F_GX][k] = (i == 0) ? (c[k + 1] - c[k]) / h
                          : (i == nx - 1) ? (c[k] - c[k - 1]) / h
                          : (c[k + 1] - c[k - 1]) / (2 * h);
            F->v[F_GY][k] = (j == 0) ? (c[k + nx] - c[k]) / h
                          : (j == ny - 1) ? (c[k] - c[k - nx]) / h
                          : (c[k + nx] - c[k - nx]) / (2 * h);
            if (i > 0 && i < nx - 1 && j > 0 && j < ny - 1) {
                F->v[F_HXX][k] = (c[k + 1] - 2 * c[k] + c[k - 1]) / (h * h);
                F->v[F_HYY][k] = (c[k + nx] - 2 * c[k] + c[k - nx]) / (h * h);
                F->v[F_HXY][k] = (c[k + nx + 1] - c[k + nx - 1] - c[k - nx + 1] + c[k - nx - 1]) / (4 * h * h);
            }
        }
    if (orc_get_interpolator() == 1) {
        F->ac = malloc(n * sizeof(double));
        F->as = malloc(n * sizeof(double));
        if (!F->ac || !F->as || orc_bspline_coef(g, c, F->ac, 0) || orc_bspline_coef(g, F->v[F_S], F->as, 0)) {
            bfield_free(F);
            return ORC_ENOMEM;
        }
    }
    return ORC_OK;
}

/* B10: uniform cubic B-spline basis at t in [0, 1) for coefficients i-1..i+2,
 * with its first and second derivatives in t */
static void basis2(double t, double b[4], double d1[4], double d2[4]) {
    const double u = 1.0 - t;
    b[0] = u * u * u / 6.0;
    b[1] = (3.0 * t * t * t - 6.0 * t * t + 4.0) / 6.0;
    b[2] = (-3.0 * t * t * t + 3.0 * t * t + 3.0 * t + 1.0) / 6.0;
    b[3] = t * t * t / 6.0;
    d1[0] = -u * u / 2.0;
    d1[1] = (3.0 * t * t - 4.0 * t) / 2.0;
    d1[2] = (-3.0 * t * t + 2.0 * t + 1.0) / 2.0;
    d1[3] = t * t / 2.0;
    d2[0] = u;
    d2[1] = 3.0 * t - 2.0;
    d2[2] = -3.0 * t + 1.0;
    d2[3] = t;
}

static int mirror_ix(int v, int n) {
    if (v < 0) v = -v;
    if (v > n - 1) v = 2 * (n - 1) - v;
    return v;
}

/* all fields at (x, y), bilinear; the cell index is clamped into the grid */
static void bsample(const BField* F, double x, double y, double f[F_N]) {
    const double u = (x - F->x0) / F->h, v = (y - F->y0) / F->h;
    double fi = floor(u), fj = floor(v);
    if (!(fi >= 0)) fi = 0;
    if (fi > F->nx - 2) fi = F->nx - 2;
    if (!(fj >= 0)) fj = 0;
    if (fj > F->ny - 2) fj = F->ny - 2;
    const int i = (int)fi, j = (int)fj;
    const double tx = u - i, ty = v - j;
    const size_t k00 = (size_t)j * F->nx + i, k10 = k00 + 1, k01 = k00 + F->nx, k11 = k01 + 1;
    const double w00 = (1 - tx) * (1 - ty), w10 = tx * (1 - ty), w01 = (1 - tx) * ty, w11 = tx * ty;
    for (int q = 0; q < F_N; ++q) {
        const double* a = F->v[q];
        f[q] = w00 * a[k00] + w10 * a[k10] + w01 * a[k01] + w11 * a[k11];
    }
    if (F->ac) {   /* B10: c, its derivatives and s from the splines (alpha0 stays bilinear) */
        double bx[4], dx1[4], dx2[4], by[4], dy1[4], dy2[4];
        basis2(tx, bx, dx1, dx2);
        basis2(ty, by, dy1, dy2);
        double c = 0, cx = 0, cy = 0, cxx = 0, cxy = 0, cyy = 0, sv = 0;
        for (int b = 0; b < 4; ++b) {
            const size_t row = (size_t)mirror_ix(j - 1 + b, F->ny) * F->nx;
            for (int a = 0; a < 4; ++a) {
                const size_t k = row + (size_t)mirror_ix(i - 1 + a, F->nx);
                const double ak = F->ac[k];
                c += bx[a] * by[b] * ak;
                cx += dx1[a] * by[b] * ak;
                cy += bx[a] * dy1[b] * ak;
                cxx += dx2[a] * by[b] * ak;
                cxy += dx1[a] * dy1[b] * ak;
                cyy += bx[a] * dy2[b] * ak;
                sv += bx[a] * by[b] * F->as[k];
            }
        }
        const double h = F->h;
        f[F_C] = c;
        f[F_GX] = cx / h;
        f[F_GY] = cy / h;
        f[F_HXX] = cxx / (h * h);
        f[F_HXY] = cxy / (h * h);
        f[F_HYY] = cyy / (h * h);
        f[F_S] = sv;
    }
}

/* B3: state (x, y, dx, dy, Q, P) */
static void brhs(const BField* F, const double st[6], double k[6]) {
    double f[F_N];
    bsample(F, st[0], st[1], f);
    const double dx = st[2], dy = st[3];
    const double gd = f[F_GX] * dx + f[F_GY] * dy;
    k[0] = dx;
    k[1] = dy;
    k[2] = -(f[F_GX] - gd * dx) / f[F_C];
    k[3] = -(f[F_GY] - gd * dy) / f[F_C];
    /* n = (-dy, dx) / |d| */
    const double cnn = (dy * dy * f[F_HXX] - 2.0 * dx * dy * f[F_HXY] + dx * dx * f[F_HYY]) / (dx * dx + dy * dy);
    k[4] = f[F_C] * st[5];
    k[5] = -cnn / (f[F_C] * f[F_C]) * st[4];
}

/* B3 with orc_set_integrator(1): Heun's second-order Runge-Kutta on the same
 * state (x, d, Q, P), the slopes at the start and at the Euler end averaged. */
static void bheun(const BField* F, const double st[6], double hs, double out[6]) {
    double k1[6], k2[6], t[6];
    brhs(F, st, k1);
    for (int q = 0; q < 6; ++q) t[q] = st[q] + hs * k1[q];
    brhs(F, t, k2);
    for (int q = 0; q < 6; ++q) out[q] = st[q] + 0.5 * hs * (k1[q] + k2[q]);
    const double n = sqrt(out[2] * out[2] + out[3] * out[3]);
    out[2] /= n;
    out[3] /= n;
}

static void brk4(const BField* F, const double st[6], double hs, double out[6]) {
    if (orc_get_integrator() == 1) {
        bheun(F, st, hs, out);
        return;
    }
    double k1[6], k2[6], k3[6], k4[6], t[6];
    brhs(F, st, k1);
    for (int q = 0; q < 6; ++q) t[q] = st[q] + 0.5 * hs * k1[q];
    brhs(F, t, k2);
    for (int q = 0; q < 6; ++q) t[q] = st[q] + 0.5 * hs * k2[q];
    brhs(F, t, k3);
    for (int q = 0; q < 6; ++q) t[q] = st[q] + hs * k3[q];
    brhs(F, t, k4);
    for (int q = 0; q < 6; ++q) out[q] = st[q] + hs / 6.0 * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]);
    const double n = sqrt(out[2] * out[2] + out[3] * out[3]);
    out[2] /= n;
    out[3] /= n;
}

/* One sample point of a fan ray (L: absorption path integral, al: alpha0 there). */
typedef struct { double x, y, dx, dy, T, Q, P, c, s, L, al; } BSample;

typedef void (*visit_fn)(void* ctx, const BSample* p);

/* B3: march one fan ray from (xe, ye) at angle theta; visit every sample point
 * strictly before the step that leaves the ring. */
static void fan_ray(const BField* F, double R, double xe, double ye, double theta, double ds,
                    double c_t, void* ctx, visit_fn visit) {
    const int64_t maxstep = (int64_t)ceil(8.0 * R / ds);
    double f[F_N];
    double st[6] = {xe, ye, cos(theta), sin(theta), 0.0, 1.0 / c_t}, nx[6];
    bsample(F, xe, ye, f);
    BSample p = {st[0], st[1], st[2], st[3], 0.0, st[4], st[5], f[F_C], f[F_S], 0.0, f[F_AL]};
    visit(ctx, &p);
    for (int64_t m = 1; m <= maxstep; ++m) {
        brk4(F, st, ds, nx);
        if (nx[0] * nx[0] + nx[1] * nx[1] >= R * R) break;
        bsample(F, nx[0], nx[1], f);
        const double T = p.T + ds * 0.5 * (p.s + f[F_S]);
        const double L = p.L + 1e-3 * ds * 0.5 * (p.al + f[F_AL]);   /* B9: ds in metres */
        memcpy(st, nx, sizeof(st));
        p = (BSample){st[0], st[1], st[2], st[3], T, st[4], st[5], f[F_C], f[F_S], L, f[F_AL]};
        visit(ctx, &p);
    }
}

typedef struct {
    const BField* F;
    double c_t, ds;
    double *T, *A;    /* map mode: [ny*nx] of one transducer */
    double* L;        /* map mode: absorption path integral of the kept A (B9), or NULL */
    double* rec;      /* record mode: 9 values per sample */
    int64_t cap, n;
    double* S;                  /* map mode: score of the candidate whose A is kept */
    double eta;                 /* map mode: penalty of the distance to the ray */
} MapCtx;

static double clamp_q(double q, double h) {
    if (fabs(q) >= h) return q;
    return q < 0 ? -h : h;
}

typedef void (*offer_fn)(MapCtx* M, size_t k, double cand, double b, double A, double L);

/* B4 + B5: every candidate (node k, time, amplitude) of sample p */
static void candidates(MapCtx* M, const BSample* p, offer_fn offer) {
    const BField* F = M->F;
    const double h = F->h;
    if (p->T == 0.0) return; /* the transducer itself */
    const int ic = (int)floor((p->x - F->x0) / h + 0.5), jc = (int)floor((p->y - F->y0) / h + 0.5);
    for (int j = jc - 1; j <= jc + 1; ++j) {
        if (j < 0 || j >= F->ny) continue;
        for (int i = ic - 1; i <= ic + 1; ++i) {
            if (i < 0 || i >= F->nx) continue;
            const double Dx = F->x0 + i * h - p->x, Dy = F->y0 + j * h - p->y;
            const double along = p->dx * Dx + p->dy * Dy, across = -p->dy * Dx + p->dx * Dy;
            if (!(along >= -0.5 * M->ds && along < 0.5 * M->ds)) continue;
            /* paraxial Q carried to the foot of the node: dQ/ds = c P */
            const double Qf = p->Q + along * p->c * p->P;
            double curv = p->P / Qf;
            if (!(curv >= 0)) curv = p->P / clamp_q(Qf, h);
            const double A = sqrt(p->c / (M->c_t * fabs(clamp_q(Qf, h))));
            const double L = p->L + 1e-3 * p->al * along;   /* B9: first order from the foot */
            offer(M, (size_t)j * F->nx + i, p->T + p->s * along + 0.5 * curv * across * across, fabs(across), A, L);
        }
    }
}

/* the first arrival (earliest candidate) for T; for A the candidate of least
 * T + eta (b/h)^2, ties to the smaller amplitude */
static void keep(MapCtx* M, size_t k, double cand, double b, double A, double L) {
    if (cand < M->T[k]) M->T[k] = cand;
    const double q = b / M->F->h;
    const double score = cand + M->eta * q * q;
    if (score < M->S[k] || (score == M->S[k] && A < M->A[k])) {
        M->S[k] = score;
        M->A[k] = A;
        if (M->L) M->L[k] = L;
    }
}

static void deposit(void* vctx, const BSample* p) { candidates((MapCtx*)vctx, p, keep); }

static void record(void* vctx, const BSample* p) {
    MapCtx* M = (MapCtx*)vctx;
    if (M->n < M->cap) {
        double* r = M->rec + 9 * M->n;
        r[0] = p->x; r[1] = p->y; r[2] = p->dx; r[3] = p->dy; r[4] = p->T;
        r[5] = p->Q; r[6] = p->P; r[7] = p->c; r[8] = p->s;
    }
    M->n++;
}

/* B2 */
static void fan_angles(double xe, double ye, double R, double ds, int K, double* a_min, double* step) {
    const double phi = atan2(ye, xe);
    double margin = ds / R;
    if (margin < 1e-9) margin = 1e-9;
    *a_min = phi + 0.5 * M_PI + margin;
    *step = ((phi + 1.5 * M_PI - margin) - *a_min) / (K - 1);
}

static int nthreads_of(int32_t n) {
#ifdef _OPENMP
    return n > 0 ? n : omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static double c_at(const BField* F, double x, double y) {
    double f[F_N];
    bsample(F, x, y, f);
    return f[F_C];
}

int orc_fan_ray(const orc_grid* g, const double* c_mps, double R, double xe, double ye, double theta,
                double ds, int64_t cap, double* rec9, int64_t* n_out) {
    if (!n_out || !(ds > 0) || !(R > 0) || (cap > 0 && !rec9)) return ORC_EINVAL;
    BField F;
    int rc = bfield_make(&F, g, c_mps, NULL);
    if (rc) return rc;
    MapCtx M = {0};
    M.F = &F;
    M.rec = rec9;
    M.cap = cap;
    fan_ray(&F, R, xe, ye, theta, ds, c_at(&F, xe, ye), &M, record);
    *n_out = M.n;
    bfield_free(&F);
    return ORC_OK;
}

int orc_fan_angles(double xe, double ye, double R, double ds, int32_t K, double* a_min, double* step) {
    if (K < 2 || !(ds > 0) || !(R > 0) || !a_min || !step) return ORC_EINVAL;
    fan_angles(xe, ye, R, ds, K, a_min, step);
    return ORC_OK;
}

int orc_fan_maps(const orc_grid* g, const double* c_mps, int32_t n_tx, const double* tx, double R,
                 double ds, int32_t K, double eta, double* T, double* A, int32_t nthreads) {
    return orc_fan_maps_abs(g, c_mps, NULL, n_tx, tx, R, ds, K, eta, T, A, NULL, nthreads);
}

int orc_fan_maps_abs(const orc_grid* g, const double* c_mps, const double* alpha0, int32_t n_tx, const double* tx,
                     double R, double ds, int32_t K, double eta, double* T, double* A, double* Lam,
                     int32_t nthreads) {
    if (!g || !tx || n_tx < 1 || K < 2 || !T || !A || !(ds > 0) || !(R > 0) || !(eta >= 0)) return ORC_EINVAL;
    BField F;
    int rc = bfield_make(&F, g, c_mps, alpha0);
    if (rc) return rc;
    const size_t nn = (size_t)F.nx * F.ny;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads_of(nthreads)) reduction(| : bad)
    for (int32_t t = 0; t < n_tx; ++t) {
        MapCtx M = {0};
        M.F = &F;
        M.T = T + (size_t)t * nn;
        M.A = A + (size_t)t * nn;
        M.L = Lam ? Lam + (size_t)t * nn : NULL;
        M.S = malloc(nn * sizeof(double));
        if (!M.S) { bad = 1; continue; }
        M.eta = eta;
        for (size_t k = 0; k < nn; ++k) { M.T[k] = INFINITY; M.A[k] = 0.0; M.S[k] = INFINITY; }
        if (M.L) for (size_t k = 0; k < nn; ++k) M.L[k] = 0.0;
        const double xe = tx[2 * t], ye = tx[2 * t + 1];
        M.c_t = c_at(&F, xe, ye);
        M.ds = ds;
        double a_min, step;
        fan_angles(xe, ye, R, ds, K, &a_min, &step);
        for (int k = 0; k < K; ++k) fan_ray(&F, R, xe, ye, a_min + k * step, ds, M.c_t, &M, deposit);
        free(M.S);
    }
    bfield_free(&F);
    return bad ? ORC_ENOMEM : ORC_OK;
}

/* E_t(x) = A exp(-wy L) exp(i omega T), 0 where unreached (wy = omega_s^y of
 * B9, L = Lambda); the phase is reduced mod 2 pi */
static void efield(double T, double A, double L, double wy, double omega, double* re, double* im) {
    if (!isfinite(T)) { *re = *im = 0.0; return; }
    double ph = omega * T;
    ph -= 2.0 * M_PI * floor(ph / (2.0 * M_PI));
    const double amp = A * exp(-wy * L);
    *re = amp * cos(ph);
    *im = amp * sin(ph);
}

/* B9: omega_s^y for f in MHz (omega_s = 2 pi f 1e6 rad/s) */
static double omega_pow(double f_mhz, double y) { return pow(2.0 * M_PI * f_mhz * 1e6, y); }

/* nodes strictly inside the ring, row-major order */
static int64_t inside_nodes(const orc_grid* g, double R, int64_t* idx) {
    int64_t n = 0;
    for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i) {
            const double x = g->x0 + i * g->h, y = g->y0 + j * g->h;
            if (x * x + y * y < R * R) {
                if (idx) idx[n] = (int64_t)j * g->nx + i;
                ++n;
            }
        }
    return n;
}

/* B6. Pairs (pairs[2k], pairs[2k+1]) or, with pairs == NULL, the full
 * n_tx x n_tx matrix; d_out complex interleaved, [n_freq][n_out]. */
int orc_born_apply(const orc_grid* g, double R, int32_t n_tx, const double* T, const double* A,
                   int32_t n_freq, const double* f_mhz, const double* dc, int32_t n_pairs,
                   const int32_t* pairs, double* d_out, int32_t nthreads) {
    return orc_born_apply_abs(g, R, n_tx, T, A, NULL, 0.0, n_freq, f_mhz, dc, n_pairs, pairs, d_out, nthreads);
}

int orc_born_apply_abs(const orc_grid* g, double R, int32_t n_tx, const double* T, const double* A,
                       const double* Lam, double y, int32_t n_freq, const double* f_mhz, const double* dc,
                       int32_t n_pairs, const int32_t* pairs, double* d_out, int32_t nthreads) {
    if (!g || n_tx < 1 || !T || !A || n_freq < 0 || (n_freq > 0 && !f_mhz) || !dc || !d_out) return ORC_EINVAL;
    if (Lam && !(y >= 0)) return ORC_EINVAL;
    const int64_t n_out = pairs ? n_pairs : (int64_t)n_tx * n_tx;
    const size_t nn = (size_t)g->nx * g->ny;
    const int64_t n_in = inside_nodes(g, R, NULL);
    int64_t* idx = malloc((size_t)(n_in > 0 ? n_in : 1) * sizeof(int64_t));
    if (!idx) return ORC_ENOMEM;
    inside_nodes(g, R, idx);
    for (int32_t f = 0; f < n_freq; ++f) {
        const double omega = 2.0 * M_PI * f_mhz[f];
        const double scale = omega * omega * g->h * g->h;
        const double wy = Lam ? omega_pow(f_mhz[f], y) : 0.0;
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads_of(nthreads))
        for (int64_t q = 0; q < n_out; ++q) {
            const int e = pairs ? pairs[2 * q] : (int)(q / n_tx);
            const int r = pairs ? pairs[2 * q + 1] : (int)(q % n_tx);
            double sre = 0.0, sim = 0.0;
            if (e != r && e >= 0 && r >= 0 && e < n_tx && r < n_tx) {
                for (int64_t p = 0; p < n_in; ++p) {
                    const size_t k = (size_t)idx[p];
                    double ar, ai, br, bi;
                    efield(T[(size_t)e * nn + k], A[(size_t)e * nn + k], Lam ? Lam[(size_t)e * nn + k] : 0.0, wy,
                           omega, &ar, &ai);
                    efield(T[(size_t)r * nn + k], A[(size_t)r * nn + k], Lam ? Lam[(size_t)r * nn + k] : 0.0, wy,
                           omega, &br, &bi);
                    sre += (ar * br - ai * bi) * dc[k];
                    sim += (ar * bi + ai * br) * dc[k];
                }
            }
            d_out[2 * ((size_t)f * n_out + q)] = scale * sre;
            d_out[2 * ((size_t)f * n_out + q) + 1] = scale * sim;
        }
    }
    free(idx);
    return ORC_OK;
}

/* B7; d_in is the full [n_freq][n_tx][n_tx] complex array (its diagonal is ignored). */
int orc_born_adjoint(const orc_grid* g, double R, int32_t n_tx, const double* T, const double* A,
                     int32_t n_freq, const double* f_mhz, const double* d_in, double* dc_out,
                     int32_t nthreads) {
    return orc_born_adjoint_abs(g, R, n_tx, T, A, NULL, 0.0, n_freq, f_mhz, d_in, dc_out, nthreads);
}

int orc_born_adjoint_abs(const orc_grid* g, double R, int32_t n_tx, const double* T, const double* A,
                         const double* Lam, double y, int32_t n_freq, const double* f_mhz, const double* d_in,
                         double* dc_out, int32_t nthreads) {
    if (!g || n_tx < 1 || !T || !A || n_freq < 0 || (n_freq > 0 && !f_mhz) || !d_in || !dc_out) return ORC_EINVAL;
    if (Lam && !(y >= 0)) return ORC_EINVAL;
    const size_t nn = (size_t)g->nx * g->ny;
    const int nt = nthreads_of(nthreads);
    const int64_t n_in = inside_nodes(g, R, NULL);
    int64_t* idx = malloc((size_t)(n_in > 0 ? n_in : 1) * sizeof(int64_t));
    double* E = malloc(2 * (size_t)n_tx * sizeof(double) * (size_t)nt);
    if (!idx || !E) { free(idx); free(E); return ORC_ENOMEM; }
    inside_nodes(g, R, idx);
    for (size_t k = 0; k < nn; ++k) dc_out[k] = 0.0;
#pragma omp parallel num_threads(nt)
    {
#ifdef _OPENMP
        double* Et = E + 2 * (size_t)n_tx * omp_get_thread_num();
#else
        double* Et = E;
#endif
#pragma omp for schedule(dynamic, 64)
        for (int64_t p = 0; p < n_in; ++p) {
            const size_t k = (size_t)idx[p];
            double acc = 0.0;
            for (int32_t f = 0; f < n_freq; ++f) {
                const double omega = 2.0 * M_PI * f_mhz[f];
                const double scale = omega * omega * g->h * g->h;
                const double wy = Lam ? omega_pow(f_mhz[f], y) : 0.0;
                for (int32_t t = 0; t < n_tx; ++t)
                    efield(T[(size_t)t * nn + k], A[(size_t)t * nn + k], Lam ? Lam[(size_t)t * nn + k] : 0.0, wy,
                           omega, &Et[2 * t], &Et[2 * t + 1]);
                for (int32_t e = 0; e < n_tx; ++e) {
                    const double ar = Et[2 * e], ai = Et[2 * e + 1];
                    if (ar == 0.0 && ai == 0.0) continue;
                    for (int32_t r = 0; r < n_tx; ++r) {
                        if (r == e) continue;
                        const double br = Et[2 * r], bi = Et[2 * r + 1];
                        const double pr = ar * br - ai * bi, pi = ar * bi + ai * br;
                        const double* dd = d_in + 2 * (((size_t)f * n_tx + e) * n_tx + r);
                        acc += scale * (pr * dd[0] + pi * dd[1]);
                    }
                }
            }
            dc_out[k] = acc;
        }
    }
    free(idx);
    free(E);
    return ORC_OK;
}
