/*
 * FP64 CPU oracle for two-point ray tracing (ToF, system matrix, adjoint).
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the library. It shares no code with
 * the CUDA path. Written for clarity, not speed: plain FP64, absolute
 * coordinates, one ray per OpenMP iteration, every sample interpolated afresh.
 *
 * Where the paper (arXiv:2511.18511) is silent, the readings below are used:
 *   R1 gradient: dc/dx, dc/dy from grid values by central differences (one-sided
 *      at edges), then interpolated bilinearly like c itself (Sec. 3.3.1: the
 *      gradient is obtained by interpolating grid values, not by differentiating
 *      the interpolant);
 *   R2 out-of-grid samples clamp the cell index (never reached: the ring lies
 *      inside the grid with a margin, which is checked);
 *   R3 ray equations dx/ds = d, dd/ds = -(grad c - (grad c . d) d)/c (the
 *      refractive-index form of Sec. 3.2.3 with n = c0/c), classic RK4 at fixed
 *      ds (or, with orc_set_integrator(1), Heun's second-order Runge-Kutta, the
 *      paper's default), d renormalised after every step;
 *   R4 a trace ends at the first step, after the first one, whose end lies on
 *      or outside |x| = R; the last point is then replaced by the boundary
 *      interception, reached by an RK4 step of length ds' <= ds (Sec. 4.2: last
 *      point replaced, shortened last step). ds' starts from the chord-circle
 *      root and takes two Newton corrections. A first step that already ends
 *      outside means the ray left outward: its interception is the emitter;
 *   R5 travel time = trapezoid rule over the sample points with the
 *      interpolated nodal slowness (Sec. 4.2's acoustic-length formula with the
 *      slowness in place of n), plus the first-order endpoint correction
 *      s(x_M) d_M.(x_r - x_M) that follows from grad T = s d (Appendix,
 *      grad T . grad T = c^-2); the correction is a weight on the last point,
 *      so T = L s still holds exactly;
 *   R6 linking (Sec. 3.4): misfit m = R (psi_hit - psi_r), the signed arc from
 *      the receiver to the boundary interception (the discrepancy of the two in
 *      the angular domain), with both angles measured counter-clockwise from
 *      the emitter in [0, 2pi) so that m is continuous over the inward fan of
 *      launch angles; converged when |x_hit - x_r| <= tol; first angle the
 *      straight line to the receiver (Sec. 3.4.1) or a warm start; the fan
 *      ends bracket the root, a probe ray next to the fan's lower end tells
 *      whether the sweep runs counter-clockwise or (through a focus) clockwise;
 *      second angle from the straight-chord slope |dm/dtheta| = 2R; then Secant
 *      updates from the two latest angles (Sec. 3.4, default) while they stay
 *      inside the bracket, else Regula-Falsi (Sec. 3.4) with the Illinois
 *      halving; at most max_iter traces (the probe counts); the reported ray
 *      is the evaluated one closest to the receiver;
 *   R8 fan start for cold starts (optional, see link_pair_fan);
 *   R13 corrected fan model for the second and third angles of a fan start
 *      (optional, orc_set_link_rule(1), see link_pair_fan);
 *   S1-S4 cubic B-spline option (orc_set_interpolator(1); Sec. 3.3.1's second
 *      scheme, the one behind the paper's Sec. 4 experiments): S1 the spline
 *      interpolates the nodal values: its control coefficients, one per node,
 *      solve (a_{i-1} + 4 a_i + a_{i+1})/6 = f_i along each axis with the
 *      mirror extension a_{-1} = a_1, a_n = a_{n-2}, and a sample weights the
 *      4 x 4 coefficients around its cell by the uniform cubic B-spline basis
 *      of its in-cell fractions (taking the nodal values themselves as the
 *      coefficients would smooth the field by h^2/6 times its Laplacian,
 *      which measured twice the bilinear error on the Sec. 4 lens, against
 *      the paper's statement that the spline is the more accurate scheme);
 *      S2 c and grad c are the spline of c and its exact derivative
 *      (replacing R1); S3 the slowness of the travel time is the spline of
 *      the nodal slowness, so T = L a_s with a_s its coefficients, the
 *      system-matrix row holding the basis weights (16 per sample), and the
 *      adjoint is P^-T L^T; S4 coefficient indices -1 and n fold back by the
 *      mirror (never reached by a ring that lies inside the grid with a
 *      margin);
 *   R7 adjoint: the rays are frozen at the linked angles (Fermat: the first
 *      order path change does not move T), so the gradient is the transpose
 *      of the system matrix whose rows are interpolation-weighted path lengths
 *      (Sec. 3.1.1), chained with ds/dc = -1/c^2.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny;
    double h, x0, y0;
    double *c, *gx, *gy, *s;
    double *ac, *as;    /* B-spline control coefficients of c and s (S1), else NULL */
} Field;

static void field_free(Field* F) {
    free(F->c); free(F->gx); free(F->gy); free(F->s); free(F->ac); free(F->as);
    memset(F, 0, sizeof(*F));
}

static int g_interp;
static int bspline_coef(int nx, int ny, const double* f, double* a, int transpose);

/* R1: nodal c (mm/us), central-difference gradient, slowness. */
static int field_make(Field* F, const orc_grid* g, const double* c_mps) {
    memset(F, 0, sizeof(*F));
    if (!g || !c_mps || g->nx < 3 || g->ny < 3 || !(g->h > 0)) return ORC_EINVAL;
    F->nx = g->nx; F->ny = g->ny; F->h = g->h; F->x0 = g->x0; F->y0 = g->y0;
    size_t n = (size_t)g->nx * (size_t)g->ny;
    F->c = malloc(n * sizeof(double)); F->gx = malloc(n * sizeof(double));
    F->gy = malloc(n * sizeof(double)); F->s = malloc(n * sizeof(double));
    if (!F->c || !F->gx || !F->gy || !F->s) { field_free(F); return ORC_ENOMEM; }
    for (size_t k = 0; k < n; ++k) {
        double v = c_mps[k];
        if (!(v > 0) || !isfinite(v)) { field_free(F); return ORC_EINVAL; }
        F->c[k] = v * 1e-3;
        F->s[k] = 1.0 / F->c[k];
    }
    const int nx = F->nx, ny = F->ny;
    const double h = F->h;
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            size_t k = (size_t)j * nx + i;
            if (i == 0) F->gx[k] = (F->c[k + 1] - F->c[k]) / h;
            else if (i == nx - 1) F->gx[k] = (F->c[k] - F->c[k - 1]) / h;
            else F->gx[k] = (F->c[k + 1] - F->c[k - 1]) / (2.0 * h);
            if (j == 0) F->gy[k] = (F->c[k + nx] - F->c[k]) / h;
            else if (j == ny - 1) F->gy[k] = (F->c[k] - F->c[k - nx]) / h;
            else F->gy[k] = (F->c[k + nx] - F->c[k - nx]) / (2.0 * h);
        }
    }
    if (g_interp == 1) {
        F->ac = malloc(n * sizeof(double));
        F->as = malloc(n * sizeof(double));
        if (!F->ac || !F->as || bspline_coef(nx, ny, F->c, F->ac, 0) || bspline_coef(nx, ny, F->s, F->as, 0)) {
            field_free(F);
            return ORC_ENOMEM;
        }
    }
    return ORC_OK;
}

/* The interpolator every sample uses: 0 = bilinear (default), 1 = cubic
 * B-spline (readings S1-S4 in the header). */
static int g_interp = 0;

int orc_set_interpolator(int32_t k) {
    if (k != 0 && k != 1) return ORC_EINVAL;
    g_interp = k;
    return ORC_OK;
}

int orc_get_interpolator(void) { return g_interp; }

/* S1: the interpolation matrix of one axis, (B a)_i = (a_{i-1} + 4 a_i +
 * a_{i+1}) / 6 with the mirror extension a_{-1} = a_1, a_n = a_{n-2}: its
 * sub- and super-diagonal entries of row i (the diagonal is 4/6). */
static double bs_sub(int i, int n) { return i == n - 1 ? 2.0 / 6.0 : 1.0 / 6.0; }
static double bs_sup(int i, int n) { return i == 0 ? 2.0 / 6.0 : 1.0 / 6.0; }

/* Solves B x = v (or B^T x = v) in place for the strided vector v[k * st],
 * k < n, by tridiagonal elimination (Thomas algorithm); cp: n doubles. */
static void bs_solve_1d(int n, double* v, size_t st, int transpose, double* cp) {
    const double dg = 4.0 / 6.0;
    double sub, sup, m;
    sup = transpose ? bs_sub(1, n) : bs_sup(0, n);
    cp[0] = sup / dg;
    v[0] = v[0] / dg;
    for (int i = 1; i < n; ++i) {
        sub = transpose ? bs_sup(i - 1, n) : bs_sub(i, n);
        sup = (i + 1 < n) ? (transpose ? bs_sub(i + 1, n) : bs_sup(i, n)) : 0.0;
        m = dg - sub * cp[i - 1];
        cp[i] = sup / m;
        v[(size_t)i * st] = (v[(size_t)i * st] - sub * v[(size_t)(i - 1) * st]) / m;
    }
    for (int i = n - 2; i >= 0; --i) v[(size_t)i * st] -= cp[i] * v[(size_t)(i + 1) * st];
}

/* S1: control coefficients a = P^-1 f of the 2D interpolating spline (P =
 * B_y (x) B_x, one axis after the other); transpose = 1 applies P^-T. */
static int bspline_coef(int nx, int ny, const double* f, double* a, int transpose) {
    double* cp = malloc((size_t)(nx > ny ? nx : ny) * sizeof(double));
    if (!cp) return ORC_ENOMEM;
    memcpy(a, f, (size_t)nx * ny * sizeof(double));
    for (int j = 0; j < ny; ++j) bs_solve_1d(nx, a + (size_t)j * nx, 1, transpose, cp);
    for (int i = 0; i < nx; ++i) bs_solve_1d(ny, a + i, (size_t)nx, transpose, cp);
    free(cp);
    return ORC_OK;
}

/* Nodes and weights of one sample: n = 4 (bilinear) or 16 (B-spline); wx, wy
 * are the weights of the analytic derivative d/dx, d/dy (B-spline only). For
 * the B-spline the k[] index the control coefficients (one per node). */
typedef struct { int n; size_t k[16]; double w[16], wx[16], wy[16]; } Stencil;

/* S1: uniform cubic B-spline basis at t in [0, 1): the weights of coefficients
 * i-1, i, i+1, i+2 of a cell spanning nodes i..i+1, and their derivatives d/dt. */
static void bspline_basis(double t, double b[4], double db[4]) {
    const double u = 1.0 - t;
    b[0] = u * u * u / 6.0;
    b[1] = (3.0 * t * t * t - 6.0 * t * t + 4.0) / 6.0;
    b[2] = (-3.0 * t * t * t + 3.0 * t * t + 3.0 * t + 1.0) / 6.0;
    b[3] = t * t * t / 6.0;
    db[0] = -u * u / 2.0;
    db[1] = (3.0 * t * t - 4.0 * t) / 2.0;
    db[2] = (-3.0 * t * t + 2.0 * t + 1.0) / 2.0;
    db[3] = t * t / 2.0;
}

/* S4: coefficient index -1 or n folds back by the mirror extension. */
static int mirror(int v, int n) {
    if (v < 0) v = -v;
    if (v > n - 1) v = 2 * (n - 1) - v;
    return v;
}

/* The enclosing cell (R2 clamps) and the sample's weights: the four vertices
 * bilinearly, or (S1, S4) the 4 x 4 coefficients around the cell by the
 * B-spline basis. */
static void stencil_at(const Field* F, double x, double y, Stencil* S) {
    double u = (x - F->x0) / F->h, v = (y - F->y0) / F->h;
    double fi = floor(u), fj = floor(v);
    if (!(fi >= 0)) fi = 0;
    if (fi > F->nx - 2) fi = F->nx - 2;
    if (!(fj >= 0)) fj = 0;
    if (fj > F->ny - 2) fj = F->ny - 2;
    int i = (int)fi, j = (int)fj;
    double tx = u - i, ty = v - j;
    if (g_interp == 1) {
        double bx[4], dbx[4], by[4], dby[4];
        bspline_basis(tx, bx, dbx);
        bspline_basis(ty, by, dby);
        S->n = 16;
        for (int b = 0; b < 4; ++b) {
            const size_t row = (size_t)mirror(j - 1 + b, F->ny) * F->nx;
            for (int a = 0; a < 4; ++a) {
                const int q = 4 * b + a;
                S->k[q] = row + (size_t)mirror(i - 1 + a, F->nx);
                S->w[q] = bx[a] * by[b];
                S->wx[q] = dbx[a] * by[b] / F->h;
                S->wy[q] = bx[a] * dby[b] / F->h;
            }
        }
        return;
    }
    S->n = 4;
    S->k[0] = (size_t)j * F->nx + i;        S->w[0] = (1 - tx) * (1 - ty);
    S->k[1] = S->k[0] + 1;                  S->w[1] = tx * (1 - ty);
    S->k[2] = S->k[0] + F->nx;              S->w[2] = (1 - tx) * ty;
    S->k[3] = S->k[2] + 1;                  S->w[3] = tx * ty;
}

/* f = (c, dc/dx, dc/dy, s) at (x, y): bilinear with R1's nodal gradient, or
 * (S2, S3) the splines of c and s with the spline's own gradient. */
static void sample(const Field* F, double x, double y, double f[4]) {
    Stencil S;
    stencil_at(F, x, y, &S);
    f[0] = f[1] = f[2] = f[3] = 0;
    for (int q = 0; q < S.n; ++q) {
        const size_t k = S.k[q];
        if (g_interp == 1) {
            f[0] += S.w[q] * F->ac[k];
            f[1] += S.wx[q] * F->ac[k];
            f[2] += S.wy[q] * F->ac[k];
            f[3] += S.w[q] * F->as[k];
        } else {
            f[0] += S.w[q] * F->c[k];
            f[1] += S.w[q] * F->gx[k];
            f[2] += S.w[q] * F->gy[k];
            f[3] += S.w[q] * F->s[k];
        }
    }
}

/* R3: right-hand side of the ray equations for the state (x, y, dx, dy). */
static void rhs(const Field* F, const double st[4], double k[4]) {
    double f[4];
    sample(F, st[0], st[1], f);
    double gd = f[1] * st[2] + f[2] * st[3];
    k[0] = st[2];
    k[1] = st[3];
    k[2] = -(f[1] - gd * st[2]) / f[0];
    k[3] = -(f[2] - gd * st[3]) / f[0];
}

/* R3: one classic RK4 step of length hs, then d renormalised. */
static void step_rk4(const Field* F, const double st[4], double hs, double out[4]) {
    double k1[4], k2[4], k3[4], k4[4], t[4];
    rhs(F, st, k1);
    for (int q = 0; q < 4; ++q) t[q] = st[q] + 0.5 * hs * k1[q];
    rhs(F, t, k2);
    for (int q = 0; q < 4; ++q) t[q] = st[q] + 0.5 * hs * k2[q];
    rhs(F, t, k3);
    for (int q = 0; q < 4; ++q) t[q] = st[q] + hs * k3[q];
    rhs(F, t, k4);
    for (int q = 0; q < 4; ++q) out[q] = st[q] + hs / 6.0 * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]);
    double n = sqrt(out[2] * out[2] + out[3] * out[3]);
    out[2] /= n;
    out[3] /= n;
}

/* R3 (option, the paper's default, Sec. 3.2.3): one step of Heun's
 * second-order Runge-Kutta method of length hs (the slope at the start, then
 * the slope at the Euler end point, averaged), then d renormalised. */
static void step_heun(const Field* F, const double st[4], double hs, double out[4]) {
    double k1[4], k2[4], t[4];
    rhs(F, st, k1);
    for (int q = 0; q < 4; ++q) t[q] = st[q] + hs * k1[q];
    rhs(F, t, k2);
    for (int q = 0; q < 4; ++q) out[q] = st[q] + 0.5 * hs * (k1[q] + k2[q]);
    double n = sqrt(out[2] * out[2] + out[3] * out[3]);
    out[2] /= n;
    out[3] /= n;
}

/* The integrator every trace uses: 0 = classic RK4 (default), 1 = Heun. */
static int g_integrator = 0;

int orc_set_integrator(int32_t k) {
    if (k != 0 && k != 1) return ORC_EINVAL;
    g_integrator = k;
    return ORC_OK;
}

int orc_get_integrator(void) { return g_integrator; }

static void rk4(const Field* F, const double st[4], double hs, double out[4]) {
    if (g_integrator == 1) step_heun(F, st, hs, out);
    else step_rk4(F, st, hs, out);
}

/* R4: from an inside state st, the step length ds' in [0, ds] whose RK4 end
 * lies on |x| = R: chord-circle root, then two Newton corrections. */
static double land(const Field* F, const double st[4], double R, double ds, double out[4]) {
    double b = st[0] * st[2] + st[1] * st[3];
    double q = st[0] * st[0] + st[1] * st[1] - R * R;
    double disc = b * b - q;
    if (disc < 0) disc = 0;
    double sq = sqrt(disc);
    double t = (b >= 0) ? (-q) / (b + sq) : (sq - b);
    if (!(t >= 0)) t = 0;
    if (t > ds) t = ds;
    for (int it = 0; it < 2; ++it) {
        rk4(F, st, t, out);
        double r = sqrt(out[0] * out[0] + out[1] * out[1]);
        double drdt = (out[0] * out[2] + out[1] * out[3]) / r;
        if (drdt > 0) t -= (r - R) / drdt;
        if (!(t >= 0)) t = 0;
        if (t > ds) t = ds;
    }
    rk4(F, st, t, out);
    return t;
}

typedef struct {
    double T, hit[2], dir[2], dsp;
    int64_t n_pts;
    int flags;
} TraceRes;

static int64_t step_cap(double R, double ds) { return (int64_t)ceil(8.0 * R / ds); }

/* R4 + R5. pts/alpha (capacity cap) optional. */
static void trace(const Field* F, double R, double xe, double ye, double xr, double yr,
                  double theta, double ds, double* pts, double* alpha, int64_t cap,
                  TraceRes* res) {
    const int64_t maxstep = step_cap(R, ds);
    double st[4] = {xe, ye, cos(theta), sin(theta)}, nx[4], f[4];
    sample(F, st[0], st[1], f);
    double s_prev = f[3];
    double T = 0.0, dsp = ds;
    int64_t m = 0;
    int flags = 0;
    if (pts && cap > 0) { pts[0] = st[0]; pts[1] = st[1]; }
    for (;;) {
        if (m >= maxstep) { flags |= 1; dsp = ds; break; }
        rk4(F, st, ds, nx);
        if (nx[0] * nx[0] + nx[1] * nx[1] >= R * R) {
            if (m == 0) { flags |= 2; break; }
            dsp = land(F, st, R, ds, nx);
            sample(F, nx[0], nx[1], f);
            T += dsp * 0.5 * (s_prev + f[3]);
            s_prev = f[3];
            memcpy(st, nx, sizeof(st));
            ++m;
            if (pts && m < cap) { pts[2 * m] = st[0]; pts[2 * m + 1] = st[1]; }
            break;
        }
        sample(F, nx[0], nx[1], f);
        T += ds * 0.5 * (s_prev + f[3]);
        s_prev = f[3];
        memcpy(st, nx, sizeof(st));
        ++m;
        if (pts && m < cap) { pts[2 * m] = st[0]; pts[2 * m + 1] = st[1]; }
    }
    double corr = 0.0;
    if (flags & 2) {
        /* left outward: no path; the interception is the emitter itself */
        T = 0.0;
        res->hit[0] = xe; res->hit[1] = ye;
        res->dir[0] = cos(theta); res->dir[1] = sin(theta);
        res->dsp = 0.0;
        m = 0;
    } else {
        res->hit[0] = st[0]; res->hit[1] = st[1];
        res->dir[0] = st[2]; res->dir[1] = st[3];
        res->dsp = dsp;
        if (!(flags & 1)) {
            corr = st[2] * (xr - st[0]) + st[3] * (yr - st[1]);
            T += s_prev * corr;
        }
    }
    res->T = T;
    res->n_pts = m + 1;
    res->flags = flags;
    if (alpha && cap >= m + 1) {
        /* alpha_k = (l_k + l_{k+1})/2 with l_0 = l_{M+1} = 0, l_M = ds' */
        for (int64_t k = 0; k <= m; ++k) {
            double lk = (k == 0) ? 0.0 : ((k == m) ? res->dsp : ds);
            double lk1 = (k == m) ? 0.0 : ((k + 1 == m) ? res->dsp : ds);
            alpha[k] = 0.5 * (lk + lk1);
        }
        alpha[m] += corr;
    }
}

static int ring_ok(const orc_grid* g, double R, double ds) {
    if (!(R > 0) || !(ds > 0)) return 0;
    double lo_x = g->x0, hi_x = g->x0 + (g->nx - 1) * g->h;
    double lo_y = g->y0, hi_y = g->y0 + (g->ny - 1) * g->h;
    double need = R + ds + g->h;
    return (-need >= lo_x) && (need <= hi_x) && (-need >= lo_y) && (need <= hi_y);
}

static int pair_of(int32_t n_tx, const int32_t* pairs, int64_t k, int* e, int* r) {
    if (pairs) { *e = pairs[2 * k]; *r = pairs[2 * k + 1]; }
    else {
        int64_t ee = k / (n_tx - 1), rr = k % (n_tx - 1);
        *e = (int)ee; *r = (int)(rr + (rr >= ee));
    }
    return (*e >= 0 && *e < n_tx && *r >= 0 && *r < n_tx && *e != *r);
}

static int on_ring(const double* p, double R) {
    double r = sqrt(p[0] * p[0] + p[1] * p[1]);
    return fabs(r - R) <= 1e-9 * R;
}

typedef struct { double theta, m, dist; TraceRes tr; } Eval;

static double mod_2pi(double a) { return a - 2.0 * M_PI * floor(a / (2.0 * M_PI)); }

/* R6: misfit of one trace. psi = angle of the interception measured
 * counter-clockwise from the emitter, in [0, 2pi); m = R (psi - psi_r), the
 * signed arc from the receiver, unwrapped at the emitter so that it is
 * continuous over the whole inward fan. A ray that left outward at once has no
 * interception; it gets the value of the fan end it is closest to. */
static void evaluate(const Field* F, double R, const double* xe, const double* xr, double phi_e,
                     double psi_r, double th_lo, double th_hi, double psi_at_lo, double ds,
                     double theta, Eval* E) {
    E->theta = theta;
    trace(F, R, xe[0], xe[1], xr[0], xr[1], theta, ds, NULL, NULL, 0, &E->tr);
    double dx = E->tr.hit[0] - xr[0], dy = E->tr.hit[1] - xr[1];
    E->dist = sqrt(dx * dx + dy * dy);
    double psi;
    if (E->tr.flags & 3) {
        /* no interception (left outward at once, or still inside after the
         * step cap, which near-tangent rays that circle back to the emitter
         * can do): the fan-end value, and never the reported ray */
        psi = (theta - th_lo < th_hi - theta) ? psi_at_lo : 2.0 * M_PI - psi_at_lo;
        E->dist = INFINITY;
    } else {
        psi = mod_2pi(atan2(E->tr.hit[1], E->tr.hit[0]) - phi_e);
    }
    E->m = R * (psi - psi_r);
}

/* Sign-changing bracket (ta, fa < 0), (tb, fb > 0) with the Illinois rule:
 * when the same end is replaced twice in a row, the other end's value halves. */
typedef struct { double ta, fa, tb, fb; int last; } Bracket;

static void br_insert(Bracket* B, double t, double m) {
    if (!(t > fmin(B->ta, B->tb) && t < fmax(B->ta, B->tb))) return;
    if (m < 0) {
        B->ta = t; B->fa = m;
        if (B->last == -1) B->fb *= 0.5;
        B->last = -1;
    } else {
        B->tb = t; B->fb = m;
        if (B->last == 1) B->fa *= 0.5;
        B->last = 1;
    }
}

/* R6 linking of one pair: shooting over the inward fan of launch angles
 * (phi_e + pi/2, phi_e + 3pi/2). Over that fan the interception sweeps the
 * whole ring once, so the fan's two ends bracket the root. The sweep runs
 * counter-clockwise in straight-like media and clockwise when rays cross
 * through a focus (the fish-eye lens); a probe ray launched next to the fan's
 * lower end tells which, since it returns next to the emitter on that side.
 * Secant steps (Sec. 3.4, default) are taken while they stay inside the
 * bracket; otherwise a Regula-Falsi step on the bracket with the Illinois
 * halving of a twice-retained end. */
static void link_pair(const Field* F, double R, const double* xe, const double* xr, double ds,
                      double tol, int max_iter, double theta_in, Eval* best, int* status,
                      int* n_eval_out) {
    const double phi_e = atan2(xe[1], xe[0]);
    const double psi_r = mod_2pi(atan2(xr[1], xr[0]) - phi_e);
    const double th_lo = phi_e + 0.5 * M_PI, th_hi = phi_e + 1.5 * M_PI;
    double margin = ds / R;
    if (margin < 1e-9) margin = 1e-9;
    const double a_min = th_lo + margin, a_max = th_hi - margin;
    if (max_iter < 2) max_iter = 2;

    double th0 = isnan(theta_in) ? atan2(xr[1] - xe[1], xr[0] - xe[0]) : theta_in;
    th0 = th_lo + mod_2pi(th0 - th_lo);
    if (th0 < a_min) th0 = a_min;
    if (th0 > a_max) th0 = a_max;

    Eval e0, ep;
    int n_eval = 0, conv = 0;
    double psi_at_lo = 0.0; /* interception angle at the lo end of the fan (0 or 2pi) */

    evaluate(F, R, xe, xr, phi_e, psi_r, th_lo, th_hi, psi_at_lo, ds, th0, &e0);
    ++n_eval;
    *best = e0;
    if (e0.dist <= tol) conv = 1;
    if (!conv) {
        /* orientation probe next to the lo end of the fan */
        evaluate(F, R, xe, xr, phi_e, psi_r, th_lo, th_hi, psi_at_lo, ds, a_min, &ep);
        ++n_eval;
        if (ep.dist < best->dist) *best = ep;
        if (ep.dist <= tol) conv = 1;
        const int ccw = (ep.m / R + psi_r) < M_PI;
        psi_at_lo = ccw ? 0.0 : 2.0 * M_PI;
        if (e0.tr.flags & 3)
            evaluate(F, R, xe, xr, phi_e, psi_r, th_lo, th_hi, psi_at_lo, ds, th0, &e0);
        if (ep.tr.flags & 3)
            ep.m = R * (psi_at_lo - psi_r);
        Bracket B;
        B.ta = ccw ? th_lo : th_hi; B.fa = -R * psi_r;
        B.tb = ccw ? th_hi : th_lo; B.fb = R * (2.0 * M_PI - psi_r);
        B.last = 0;
        br_insert(&B, ep.theta, ep.m);
        br_insert(&B, e0.theta, e0.m);
        B.last = 0;
        /* second angle from the straight-chord slope |dm/dtheta| = 2R */
        double next = th0 - e0.m / (ccw ? 2.0 * R : -2.0 * R);
        Eval prev = e0, cur = e0;
        int first = 1;
        while (!conv && n_eval < max_iter) {
            if (!first) {
                double den = cur.m - prev.m;
                int ok = (den != 0.0);
                next = ok ? cur.theta - cur.m * (cur.theta - prev.theta) / den : 0.0;
                if (!ok) next = NAN;
            }
            first = 0;
            if (!(isfinite(next) && next > fmin(B.ta, B.tb) && next < fmax(B.ta, B.tb)))
                next = (B.ta * B.fb - B.tb * B.fa) / (B.fb - B.fa);
            Eval e;
            evaluate(F, R, xe, xr, phi_e, psi_r, th_lo, th_hi, psi_at_lo, ds, next, &e);
            ++n_eval;
            if (e.dist < best->dist) *best = e;
            if (e.dist <= tol) { conv = 1; break; }
            br_insert(&B, e.theta, e.m);
            prev = cur;
            cur = e;
        }
    }
    /* a pair none of whose traces reached the ring reports the step cap */
    *status = conv ? ORC_RAY_OK : (isinf(best->dist) ? ORC_RAY_STEPCAP : ORC_RAY_MAXITER);
    *n_eval_out = n_eval;
}

/* R8 fan start (an option; fan_rays = 0 keeps the straight-line start of
 * Sec. 3.4.1). A fan of K rays per emitter at evenly spaced angles over the
 * inward fan, theta_k = a_min + k (a_max - a_min)/(K-1), gives the
 * interception angle psi_k of each; ray 0 (next to the fan's lower end) fixes
 * the sweep orientation exactly as the probe does. For a pair, the sequence of
 * misfits (fan end, rays 0..K-1, fan end) is scanned for sign changes; the one
 * whose middle lies closest to the straight-line angle, both counted in fan-ray
 * index units, is taken and its ends form the bracket. The first angle is the
 * root of the inverse interpolating polynomial (theta as a polynomial in the
 * misfit, evaluated at misfit 0) through the eight fan rays around the
 * interval, else through the four around it, each when those rays exist,
 * their misfits are strictly monotone and the root falls inside the interval;
 * else the linear interpolation of the interval. When the first trace misses
 * the receiver, the second angle is the root of the inverse polynomial through
 * that trace and the four fan rays (when those were usable and the trace
 * reached the ring), else the secant of the first trace and the interval end
 * with the smaller |misfit|; from there on the secant of the last two traces.
 * Either candidate outside the bracket gives way to the Regula-Falsi point.
 * The fan only predicts: its rays may be traced at their own step fan_ds
 * (0 = the linking step ds), while their launch angles, the fan margin ds/R
 * and every linking trace keep ds, so the bracket rule and the predictions
 * are the same functions of the fan's interceptions.
 *
 * R12 sub-fan (an option, subfan = M > 0): when the second trace of a
 * fan-started pair misses too, M more rays at fan_ds, evenly spaced strictly
 * inside the bracket, theta_q = ta + (tb - ta) q / (M + 1), q = 1..M (ta the
 * end of negative misfit), refine it before the third trace. In the sequence
 * (ta, the sub-fan rays that reach the ring, tb) the neighbours with no
 * missing ray between them whose misfits differ in sign by less than pi R (a
 * crossing, not the jump where hits wrap around the emitter or rays stop
 * reaching the ring) and hold the angle the plain rule would trace third
 * (the secant of the two traces, else Regula Falsi) become the bracket (the
 * Illinois state restarts); the third angle is the root of the inverse cubic
 * through the four sub-fan rays around that interval (when all four are
 * sub-fan rays, their misfits are strictly monotone and the root falls
 * inside), else the Regula-Falsi point of the interval; the secant then starts
 * from the interval end of smaller |misfit|. When no crossing holds it, the
 * plain rule's angle is traced unchanged. Like the fan, the sub-fan only
 * predicts; the linking traces keep ds.
 *
 * R13 corrected fan model (an option, orc_set_link_rule(1); not combined with
 * R12). The fan's misfits, traced at fan_ds, carry the shape of the misfit
 * around the root (its curvature over the fan spacing) but are offset from the
 * misfit of the linking traces at ds. The model is the forward interpolating
 * polynomial P(theta) through the widest window of 8, 6, 4 or 2 fan rays
 * centred on the bracketing interval whose misfits exist and change strictly
 * monotonically. When the first trace (theta_1, m_1) misses, the second angle
 * is the root of P(theta) + a with a = m_1 - P(theta_1) (the model moved onto
 * the trace); when the second trace (theta_2, m_2) misses too, the third
 * angle is the root of P(theta) + a + b (theta - theta_1), the offset a and
 * tilt b fitted through both traces. Each root is sought in the current
 * bracket, where the model must change sign; otherwise, or when a trace did
 * not reach the ring, the R8 rule picks the angle. From the fourth angle on
 * the secant continues as in R8. Like the fan, the model only predicts. */
static double fan_theta(double a_min, double step, int k) { return a_min + k * step; }

static int g_link_rule = 0;

int orc_set_link_rule(int32_t k) {
    if (k != 0 && k != 1) return ORC_EINVAL;
    g_link_rule = k;
    return ORC_OK;
}

int orc_get_link_rule(void) { return g_link_rule; }

/* Forward interpolating polynomial through (t[q], m[q]), q < n, and its
 * derivative at x (Lagrange form, derivative by the product rule). */
static void poly_eval(const double* t, const double* m, int n, double x, double* p, double* dp) {
    double v = 0.0, d = 0.0;
    for (int a = 0; a < n; ++a) {
        double l = 1.0;
        for (int b = 0; b < n; ++b)
            if (b != a) l *= (x - t[b]) / (t[a] - t[b]);
        v += l * m[a];
        double dl = 0.0;
        for (int k = 0; k < n; ++k) {
            if (k == a) continue;
            double term = 1.0 / (t[a] - t[k]);
            for (int b = 0; b < n; ++b)
                if (b != a && b != k) term *= (x - t[b]) / (t[a] - t[b]);
            dl += term;
        }
        d += dl * m[a];
    }
    *p = v;
    *dp = d;
}

/* R13: root in (lo, hi) of g(x) = P(x) + a + b (x - x1), P the fan
 * polynomial, by Newton steps kept inside the shrinking sign-change interval
 * (bisection when a step leaves it); NAN when g does not change sign over
 * (lo, hi). */
static double r13_root(const double* t, const double* m, int n, double a, double b, double x1, double lo,
                       double hi) {
    double glo, ghi, d;
    poly_eval(t, m, n, lo, &glo, &d);
    glo += a + b * (lo - x1);
    poly_eval(t, m, n, hi, &ghi, &d);
    ghi += a + b * (hi - x1);
    if (!(glo * ghi < 0.0)) return NAN;
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        double g, dg;
        poly_eval(t, m, n, x, &g, &dg);
        g += a + b * (x - x1);
        dg += b;
        if (g == 0.0) return x;
        if ((g < 0.0) == (glo < 0.0)) { lo = x; glo = g; } else { hi = x; ghi = g; }
        double xn = (dg != 0.0) ? x - g / dg : NAN;
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (fabs(xn - x) <= 1e-15 * fmax(1.0, fabs(x))) return xn;
        x = xn;
    }
    return x;
}

/* R13 angle: the fan model through the trace (x1, m1) (offset a) or, with
 * two = 1, through (x1, m1) and (x2, m2) (offset a and tilt b), and its root
 * in (lo, hi); NAN when the model does not change sign there. */
static double r13_angle(const double* t, const double* m, int n, double x1, double m1, double x2, double m2,
                        int two, double lo, double hi) {
    double p1, p2, d;
    poly_eval(t, m, n, x1, &p1, &d);
    const double a = m1 - p1;
    double b = 0.0;
    if (two) {
        poly_eval(t, m, n, x2, &p2, &d);
        b = ((m2 - p2) - a) / (x2 - x1);
    }
    return r13_root(t, m, n, a, b, x1, lo, hi);
}

int orc_r13_angle(const double* t, const double* m, int32_t n, double x1, double m1, double x2, double m2,
                  int32_t two, double lo, double hi, double* out) {
    if (!t || !m || !out || n < 2 || n > 8) return ORC_EINVAL;
    *out = r13_angle(t, m, n, x1, m1, x2, m2, two, lo, hi);
    return ORC_OK;
}

/* Value at m = 0 of the polynomial theta(m) through the n points (m_q, t_q),
 * Lagrange form. */
static double inverse_poly_root(const double* t, const double* m, int n) {
    double v = 0.0;
    for (int a = 0; a < n; ++a) {
        double l = 1.0;
        for (int b = 0; b < n; ++b)
            if (b != a) l *= (0.0 - m[b]) / (m[a] - m[b]);
        v += l * t[a];
    }
    return v;
}

/* Fan rays k_first .. k_first + n - 1 as (theta, misfit) points; 1 when all of
 * them exist and intercept the ring and their misfits change strictly
 * monotonically, in the direction of the middle pair (n/2 - 1, n/2). */
static int fan_points(const double* psi, int K, int k_first, int n, double a_min, double step, double R,
                      double psi_r, double* t, double* m) {
    if (k_first < 0 || k_first + n > K) return 0;
    for (int q = 0; q < n; ++q) {
        const int k = k_first + q;
        if (isnan(psi[k])) return 0;
        t[q] = fan_theta(a_min, step, k);
        m[q] = R * (psi[k] - psi_r);
    }
    const double dir = m[n / 2] - m[n / 2 - 1];
    for (int q = 0; q + 1 < n; ++q)
        if (!((m[q + 1] - m[q]) * dir > 0)) return 0;
    return 1;
}

static void fan_for_emitter(const Field* F, double R, const double* xe, double ds, double fan_ds, int K,
                            double* psi) {
    const double phi_e = atan2(xe[1], xe[0]);
    const double th_lo = phi_e + 0.5 * M_PI, th_hi = phi_e + 1.5 * M_PI;
    double margin = ds / R;
    if (margin < 1e-9) margin = 1e-9;
    const double a_min = th_lo + margin, a_max = th_hi - margin;
    const double step = (a_max - a_min) / (K - 1);
    for (int k = 0; k < K; ++k) {
        TraceRes tr;
        trace(F, R, xe[0], xe[1], xe[0], xe[1], fan_theta(a_min, step, k), fan_ds, NULL, NULL, 0, &tr);
        psi[k] = (tr.flags & 3) ? NAN : mod_2pi(atan2(tr.hit[1], tr.hit[0]) - phi_e);
    }
}

/* R12 prediction from the sequence (st[i], sm[i]), i = 0..n-1, of the
 * bracket end of negative misfit, the sub-fan rays that reached the ring (in
 * angle order, interior[i] = 1) and the other bracket end, around c3, the
 * angle the plain rule would trace next; pos[i] is the entry's place in the
 * full sequence (the bracket ends 0 and M + 1, sub-fan ray q at q). A
 * crossing is a pair of entries adjacent in the full sequence (no ray that
 * missed the ring between them) whose misfits differ in sign by less than
 * pi R (where the hit wraps around the emitter the misfit jumps by about
 * 2 pi R, which is no root). The
 * crossing that holds c3 becomes the bracket B (Illinois state restarted);
 * the third angle is the root of the inverse cubic through the four sub-fan
 * rays around it when they are all sub-fan rays with strictly monotone
 * misfits and the root falls inside, else its Regula-Falsi point, and *start
 * is its end of smaller |misfit|, where the secant starts. Returns 1; returns
 * 0, leaving B alone, when no crossing holds c3 (the plain rule then traces
 * c3 as it would have). */
static int subfan_predict(const double* st, const double* sm, const int* interior, const int* pos, int n,
                          double c3, double R, Bracket* B, double* th3, double* start_theta, double* start_m) {
    int j = -1;
    for (int i = 1; i < n && j < 0; ++i) {
        if ((sm[i - 1] < 0) == (sm[i] < 0) || !(fabs(sm[i] - sm[i - 1]) < M_PI * R) || pos[i] != pos[i - 1] + 1)
            continue;
        if (c3 >= fmin(st[i - 1], st[i]) && c3 <= fmax(st[i - 1], st[i])) j = i;
    }
    if (j < 0) return 0;
    const int neg = sm[j - 1] < 0 ? j - 1 : j, nonneg = sm[j - 1] < 0 ? j : j - 1;
    B->ta = st[neg]; B->fa = sm[neg];
    B->tb = st[nonneg]; B->fb = sm[nonneg];
    B->last = 0;
    double th = B->ta - B->fa * (B->tb - B->ta) / (B->fb - B->fa);
    if (j - 2 >= 0 && j + 1 < n && interior[j - 2] && interior[j - 1] && interior[j] && interior[j + 1]) {
        const int up = sm[j - 2] < sm[j - 1] && sm[j - 1] < sm[j] && sm[j] < sm[j + 1];
        const int down = sm[j - 2] > sm[j - 1] && sm[j - 1] > sm[j] && sm[j] > sm[j + 1];
        if (up || down) {
            const double v = inverse_poly_root(st + j - 2, sm + j - 2, 4);
            if (v > fmin(B->ta, B->tb) && v < fmax(B->ta, B->tb)) th = v;
        }
    }
    const int lo = fabs(B->fa) <= fabs(B->fb);
    *start_theta = lo ? B->ta : B->tb;
    *start_m = lo ? B->fa : B->fb;
    *th3 = th;
    return 1;
}

/* Angle of sub-fan ray q = 1..M inside the bracket (ta, tb). */
static double subfan_angle(double ta, double tb, int q, int M) { return ta + (tb - ta) * q / (M + 1); }

/* R12: trace the M sub-fan rays of bracket B at fan_ds and predict around
 * c3; returns 0 (B untouched) when no crossing holds c3. */
static int subfan_refine(const Field* F, double R, const double* xe, double phi_e, double psi_r, double fan_ds,
                         int M, double c3, Bracket* B, double* th3, Eval* start) {
    double st[ORC_SUBFAN_MAX + 2], sm[ORC_SUBFAN_MAX + 2];
    int interior[ORC_SUBFAN_MAX + 2], pos[ORC_SUBFAN_MAX + 2];
    int n = 0;
    st[n] = B->ta; sm[n] = B->fa; interior[n] = 0; pos[n++] = 0;
    for (int q = 1; q <= M; ++q) {
        const double th = subfan_angle(B->ta, B->tb, q, M);
        TraceRes tr;
        trace(F, R, xe[0], xe[1], xe[0], xe[1], th, fan_ds, NULL, NULL, 0, &tr);
        if (tr.flags & 3) continue;
        st[n] = th;
        sm[n] = R * (mod_2pi(atan2(tr.hit[1], tr.hit[0]) - phi_e) - psi_r);
        interior[n] = 1;
        pos[n++] = q;
    }
    st[n] = B->tb; sm[n] = B->fb; interior[n] = 0; pos[n++] = M + 1;
    return subfan_predict(st, sm, interior, pos, n, c3, R, B, th3, &start->theta, &start->m);
}

int orc_subfan_angles(double ta, double tb, int32_t M, double* theta) {
    if (M < 1 || M > ORC_SUBFAN_MAX || !theta) return ORC_EINVAL;
    for (int q = 1; q <= M; ++q) theta[q - 1] = subfan_angle(ta, tb, q, M);
    return ORC_OK;
}

int orc_subfan_predict(int32_t n, const double* st, const double* sm, const int32_t* pos, double c3, double R,
                       double* out7) {
    if (n < 2 || n > ORC_SUBFAN_MAX + 2 || !st || !sm || !pos || !out7 || !(R > 0)) return ORC_EINVAL;
    int in[ORC_SUBFAN_MAX + 2], ps[ORC_SUBFAN_MAX + 2];
    for (int i = 0; i < n; ++i) {
        ps[i] = pos[i];
        in[i] = i > 0 && i < n - 1;
    }
    Bracket B = {st[0], sm[0], st[n - 1], sm[n - 1], 0};
    double th = c3, s_th = NAN, s_m = NAN;
    const int refined = subfan_predict(st, sm, in, ps, n, c3, R, &B, &th, &s_th, &s_m);
    out7[0] = th; out7[1] = B.ta; out7[2] = B.tb; out7[3] = s_th; out7[4] = s_m;
    out7[5] = (B.fa < 0 && B.fb >= 0) ? 1.0 : 0.0;
    out7[6] = refined;
    return ORC_OK;
}

static void link_pair_fan(const Field* F, double R, const double* xe, const double* xr, double ds,
                          double tol, int max_iter, const double* psi, int K, double fan_ds, int subfan,
                          Eval* best, int* status, int* n_eval_out) {
    const double phi_e = atan2(xe[1], xe[0]);
    const double psi_r = mod_2pi(atan2(xr[1], xr[0]) - phi_e);
    const double th_lo = phi_e + 0.5 * M_PI, th_hi = phi_e + 1.5 * M_PI;
    double margin = ds / R;
    if (margin < 1e-9) margin = 1e-9;
    const double a_min = th_lo + margin, a_max = th_hi - margin;
    if (max_iter < 2) max_iter = 2;
    const int ccw = isnan(psi[0]) ? 1 : (psi[0] < M_PI);
    const double psi_at_lo = ccw ? 0.0 : 2.0 * M_PI;
    const double step = (a_max - a_min) / (K - 1);
    double th_s = atan2(xr[1] - xe[1], xr[0] - xe[0]);
    th_s = th_lo + mod_2pi(th_s - th_lo);
    const double u_s = (th_s - a_min) / step;   /* straight-line angle in fan-index units */
    const double psi_hi_end = 2.0 * M_PI - psi_at_lo;
    /* sequence index j: 0 fan lower end, 1..K rays 0..K-1, K+1 fan upper end;
     * the interval (j-1, j) has its middle at fan index j - 1.5 */
    int neg_prev = psi_at_lo < psi_r;
    int jsel = K + 1;
    double best_gap = INFINITY;
    for (int j = 1; j <= K + 1; ++j) {
        double p;
        if (j <= K) {
            const int k = j - 1;
            p = isnan(psi[k]) ? ((k < K / 2) ? psi_at_lo : psi_hi_end) : psi[k];
        } else {
            p = psi_hi_end;
        }
        const int neg = p < psi_r;
        if (neg != neg_prev) {
            const double gap = fabs((j - 1.5) - u_s);
            if (gap < best_gap) { best_gap = gap; jsel = j; }
        }
        neg_prev = neg;
    }
    /* ends of the chosen interval */
    double t0, m0, t1, m1;
    {
        const int ja = jsel - 1, jb = jsel;
        double pa, pb;
        if (ja == 0) { t0 = th_lo; pa = psi_at_lo; }
        else { const int k = ja - 1; t0 = fan_theta(a_min, step, k); pa = isnan(psi[k]) ? ((k < K / 2) ? psi_at_lo : psi_hi_end) : psi[k]; }
        if (jb == K + 1) { t1 = th_hi; pb = psi_hi_end; }
        else { const int k = jb - 1; t1 = fan_theta(a_min, step, k); pb = isnan(psi[k]) ? ((k < K / 2) ? psi_at_lo : psi_hi_end) : psi[k]; }
        m0 = R * (pa - psi_r);
        m1 = R * (pb - psi_r);
    }
    Bracket B;
    if (m0 < 0) { B.ta = t0; B.fa = m0; B.tb = t1; B.fb = m1; }
    else { B.ta = t1; B.fa = m1; B.tb = t0; B.fb = m0; }
    B.last = 0;
    double th0 = t0 - m0 * (t1 - t0) / (m1 - m0);
    /* rays around the interval (j-1, j): k0 = j-2 and k0+1 = j-1 */
    const int k0 = jsel - 2;
    double t8[8], m8[8], t4[4], m4[4];
    int done = 0;
    if (fan_points(psi, K, k0 - 3, 8, a_min, step, R, psi_r, t8, m8)) {
        const double v = inverse_poly_root(t8, m8, 8);
        if (v > fmin(t0, t1) && v < fmax(t0, t1)) { th0 = v; done = 1; }
    }
    const int ok4 = fan_points(psi, K, k0 - 1, 4, a_min, step, R, psi_r, t4, m4);
    if (ok4 && !done) {
        const double v = inverse_poly_root(t4, m4, 4);
        if (v > fmin(t0, t1) && v < fmax(t0, t1)) th0 = v;
    }
    /* R13 model window: the widest monotone one of 8, 6, 4, 2 rays around (k0, k0+1) */
    double tw[8], mw[8];
    int nw = 0;
    if (g_link_rule == 1 && subfan == 0)
        for (int n = 8; n >= 2 && !nw; n -= 2)
            if (fan_points(psi, K, k0 - (n / 2 - 1), n, a_min, step, R, psi_r, tw, mw)) nw = n;
    if (!(th0 > fmin(B.ta, B.tb) && th0 < fmax(B.ta, B.tb))) th0 = 0.5 * (B.ta + B.tb);
    Eval prev, cur;
    memset(&prev, 0, sizeof prev);   /* a fan interval end, not a trace */
    prev.theta = (fabs(m0) <= fabs(m1)) ? t0 : t1;
    prev.m = (fabs(m0) <= fabs(m1)) ? m0 : m1;
    cur = prev;
    int n_eval = 0, conv = 0;
    double next = th0;
    while (n_eval < max_iter) {
        if (n_eval == 2 && subfan > 0) {
            /* the plain rule's third angle, around which the sub-fan refines */
            const double den = cur.m - prev.m;
            double c3 = (den != 0.0) ? cur.theta - cur.m * (cur.theta - prev.theta) / den : NAN;
            if (!(isfinite(c3) && c3 > fmin(B.ta, B.tb) && c3 < fmax(B.ta, B.tb)))
                c3 = (B.ta * B.fb - B.tb * B.fa) / (B.fb - B.fa);
            Eval s0;
            memset(&s0, 0, sizeof s0);
            double th3;
            if (subfan_refine(F, R, xe, phi_e, psi_r, fan_ds, subfan, c3, &B, &th3, &s0)) {
                next = th3;
                prev = s0;
                cur = s0;
            } else {
                next = c3;
            }
        } else if (n_eval > 0) {
            next = NAN;
            /* R13: the fan model through the first trace (offset a), then through both (tilt b) */
            if (nw && n_eval <= 2 && !(cur.tr.flags & 3) && (n_eval == 1 || !(prev.tr.flags & 3))) {
                const double lo = fmin(B.ta, B.tb), hi = fmax(B.ta, B.tb);
                next = (n_eval == 1) ? r13_angle(tw, mw, nw, cur.theta, cur.m, 0.0, 0.0, 0, lo, hi)
                                     : r13_angle(tw, mw, nw, prev.theta, prev.m, cur.theta, cur.m, 1, lo, hi);
            }
            if (!isfinite(next)) {   /* no R13 angle: the R8 rule */
                if (n_eval == 1 && ok4 && !(cur.tr.flags & 3)) {
                    const double t5[5] = {cur.theta, t4[0], t4[1], t4[2], t4[3]};
                    const double m5[5] = {cur.m, m4[0], m4[1], m4[2], m4[3]};
                    next = inverse_poly_root(t5, m5, 5);
                } else {
                    double den = cur.m - prev.m;
                    next = (den != 0.0) ? cur.theta - cur.m * (cur.theta - prev.theta) / den : NAN;
                }
            }
            if (!(isfinite(next) && next > fmin(B.ta, B.tb) && next < fmax(B.ta, B.tb)))
                next = (B.ta * B.fb - B.tb * B.fa) / (B.fb - B.fa);
        }
        Eval e;
        evaluate(F, R, xe, xr, phi_e, psi_r, th_lo, th_hi, psi_at_lo, ds, next, &e);
        ++n_eval;
        if (n_eval == 1 || e.dist < best->dist) *best = e;
        if (e.dist <= tol) { conv = 1; break; }
        br_insert(&B, e.theta, e.m);
        prev = cur;
        cur = e;
    }
    *status = conv ? ORC_RAY_OK : (isinf(best->dist) ? ORC_RAY_STEPCAP : ORC_RAY_MAXITER);
    *n_eval_out = n_eval;
}

static int nthreads_of(int32_t n) {
#ifdef _OPENMP
    return n > 0 ? n : omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_num_threads(void) { return nthreads_of(0); }

int orc_field(const orc_grid* g, const double* c_mps, double* c, double* gx, double* gy, double* s) {
    Field F;
    int rc = field_make(&F, g, c_mps);
    if (rc) return rc;
    size_t n = (size_t)F.nx * F.ny;
    if (c) memcpy(c, F.c, n * sizeof(double));
    if (gx) memcpy(gx, F.gx, n * sizeof(double));
    if (gy) memcpy(gy, F.gy, n * sizeof(double));
    if (s) memcpy(s, F.s, n * sizeof(double));
    field_free(&F);
    return ORC_OK;
}

int orc_bspline_coef(const orc_grid* g, const double* f, double* a, int32_t transpose) {
    if (!g || !f || !a || g->nx < 3 || g->ny < 3) return ORC_EINVAL;
    return bspline_coef(g->nx, g->ny, f, a, transpose ? 1 : 0);
}

int orc_sample(const orc_grid* g, const double* c_mps, int32_t n, const double* xy, double* out) {
    Field F;
    int rc = field_make(&F, g, c_mps);
    if (rc) return rc;
    for (int32_t k = 0; k < n; ++k) sample(&F, xy[2 * k], xy[2 * k + 1], out + 4 * k);
    field_free(&F);
    return ORC_OK;
}

int orc_march(const orc_grid* g, const double* c_mps, double x, double y, double theta,
              double ds, int32_t n_steps, double* xy_out) {
    Field F;
    int rc = field_make(&F, g, c_mps);
    if (rc) return rc;
    double st[4] = {x, y, cos(theta), sin(theta)}, nx[4];
    xy_out[0] = x; xy_out[1] = y;
    for (int32_t k = 1; k <= n_steps; ++k) {
        rk4(&F, st, ds, nx);
        memcpy(st, nx, sizeof(st));
        xy_out[2 * k] = st[0];
        xy_out[2 * k + 1] = st[1];
    }
    field_free(&F);
    return ORC_OK;
}

int orc_trace(const orc_grid* g, const double* c_mps, double R, double xe, double ye,
              double xr, double yr, double theta, double ds, int64_t cap, double* pts,
              double* alpha, int64_t* n_pts, double* out6, int32_t* flags) {
    if (!ring_ok(g, R, ds)) return ORC_EINVAL;
    Field F;
    int rc = field_make(&F, g, c_mps);
    if (rc) return rc;
    TraceRes res;
    trace(&F, R, xe, ye, xr, yr, theta, ds, pts, alpha, cap, &res);
    if (n_pts) *n_pts = res.n_pts;
    if (out6) {
        out6[0] = res.T; out6[1] = res.hit[0]; out6[2] = res.hit[1];
        out6[3] = res.dir[0]; out6[4] = res.dir[1]; out6[5] = res.dsp;
    }
    if (flags) *flags = res.flags;
    field_free(&F);
    return ORC_OK;
}

static int check_common(const orc_grid* g, int32_t n_tx, const double* tx, double R, double ds,
                        int32_t n_pairs, const int32_t* pairs) {
    if (!g || !tx || n_tx < 2 || n_pairs < 0 || !ring_ok(g, R, ds)) return ORC_EINVAL;
    if (!pairs && (int64_t)n_pairs != (int64_t)n_tx * (n_tx - 1)) return ORC_EINVAL;
    for (int32_t t = 0; t < n_tx; ++t)
        if (!on_ring(tx + 2 * t, R)) return ORC_EINVAL;
    return ORC_OK;
}

int orc_link(const orc_grid* g, const double* c_mps, int32_t n_tx, const double* tx,
             double R, int32_t n_pairs, const int32_t* pairs, double ds, double tol,
             int32_t max_iter, int32_t fan_rays, double fan_ds, int32_t subfan, double* theta_io, double* tof,
             double* hit_xy, int32_t* status, int32_t* iters, int32_t nthreads) {
    int rc = check_common(g, n_tx, tx, R, ds, n_pairs, pairs);
    if (rc) return rc;
    if (!theta_io || !(tol > 0) || fan_rays == 1 || fan_rays < 0) return ORC_EINVAL;
    if (subfan < 0 || subfan > ORC_SUBFAN_MAX) return ORC_EINVAL;
    if (fan_ds == 0.0) fan_ds = ds;
    if (!(fan_ds > 0) || !isfinite(fan_ds) || (fan_rays > 0 && !ring_ok(g, R, fan_ds))) return ORC_EINVAL;
    Field F;
    rc = field_make(&F, g, c_mps);
    if (rc) return rc;
    double* fan = NULL;
    if (fan_rays > 0) {
        fan = malloc((size_t)n_tx * fan_rays * sizeof(double));
        if (!fan) { field_free(&F); return ORC_ENOMEM; }
        char* need = calloc((size_t)n_tx, 1);
        for (int32_t k = 0; k < n_pairs; ++k) {
            int e, r;
            if (pair_of(n_tx, pairs, k, &e, &r) && isnan(theta_io[k])) need[e] = 1;
        }
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads_of(nthreads))
        for (int32_t t = 0; t < n_tx; ++t)
            if (need[t]) fan_for_emitter(&F, R, tx + 2 * t, ds, fan_ds, fan_rays, fan + (size_t)t * fan_rays);
        free(need);
    }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads_of(nthreads)) reduction(| : bad)
    for (int32_t k = 0; k < n_pairs; ++k) {
        int e, r;
        if (!pair_of(n_tx, pairs, k, &e, &r)) {
            bad = 1;
            if (status) status[k] = ORC_RAY_BADINPUT;
            continue;
        }
        Eval best;
        memset(&best, 0, sizeof(best));
        int st, ne;
        if (fan && isnan(theta_io[k]))
            link_pair_fan(&F, R, tx + 2 * e, tx + 2 * r, ds, tol, max_iter, fan + (size_t)e * fan_rays, fan_rays,
                          fan_ds, subfan, &best, &st, &ne);
        else
            link_pair(&F, R, tx + 2 * e, tx + 2 * r, ds, tol, max_iter, theta_io[k], &best, &st, &ne);
        theta_io[k] = best.theta;
        if (tof) tof[k] = best.tr.T;
        if (hit_xy) { hit_xy[2 * k] = best.tr.hit[0]; hit_xy[2 * k + 1] = best.tr.hit[1]; }
        if (status) status[k] = st;
        if (iters) iters[k] = ne;
    }
    free(fan);
    field_free(&F);
    return bad ? ORC_EINVAL : ORC_OK;
}

int orc_tof(const orc_grid* g, const double* c_mps, int32_t n_tx, const double* tx,
            double R, int32_t n_pairs, const int32_t* pairs, double ds, const double* theta,
            double* tof, double* hit_xy, int32_t nthreads) {
    int rc = check_common(g, n_tx, tx, R, ds, n_pairs, pairs);
    if (rc) return rc;
    Field F;
    rc = field_make(&F, g, c_mps);
    if (rc) return rc;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads_of(nthreads)) reduction(| : bad)
    for (int32_t k = 0; k < n_pairs; ++k) {
        int e, r;
        if (!pair_of(n_tx, pairs, k, &e, &r)) { bad = 1; continue; }
        TraceRes res;
        trace(&F, R, tx[2 * e], tx[2 * e + 1], tx[2 * r], tx[2 * r + 1], theta[k], ds, NULL, NULL, 0,
              &res);
        if (tof) tof[k] = res.T;
        if (hit_xy) { hit_xy[2 * k] = res.hit[0]; hit_xy[2 * k + 1] = res.hit[1]; }
    }
    field_free(&F);
    return bad ? ORC_EINVAL : ORC_OK;
}

/* One row of L: (node, weight) entries of every sample point, sorted by node
 * and merged. Returns the entry count; ent holds 16 * n_pts slots. */
typedef struct { int64_t node; double w; } Entry;

static int cmp_entry(const void* a, const void* b) {
    int64_t x = ((const Entry*)a)->node, y = ((const Entry*)b)->node;
    return (x > y) - (x < y);
}

static int64_t build_row(const Field* F, const double* pts, const double* alpha, int64_t n_pts,
                         Entry* ent) {
    int64_t n = 0;
    for (int64_t m = 0; m < n_pts; ++m) {
        Stencil S;
        stencil_at(F, pts[2 * m], pts[2 * m + 1], &S);
        for (int q = 0; q < S.n; ++q) { ent[n].node = (int64_t)S.k[q]; ent[n].w = alpha[m] * S.w[q]; ++n; }
    }
    qsort(ent, (size_t)n, sizeof(Entry), cmp_entry);
    int64_t out = 0;
    for (int64_t t = 0; t < n; ++t) {
        if (out > 0 && ent[out - 1].node == ent[t].node) ent[out - 1].w += ent[t].w;
        else ent[out++] = ent[t];
    }
    return out;
}

int64_t orc_path_matrix(const orc_grid* g, const double* c_mps, int32_t n_tx, const double* tx,
                        double R, int32_t n_pairs, const int32_t* pairs, double ds,
                        const double* theta, int64_t* row_ptr, int32_t* col, double* val,
                        int64_t cap, int32_t nthreads) {
    if (check_common(g, n_tx, tx, R, ds, n_pairs, pairs) || !theta || !row_ptr) return -1;
    Field F;
    if (field_make(&F, g, c_mps)) return -1;
    const int64_t pcap = step_cap(R, ds) + 2;
    int64_t* counts = calloc((size_t)n_pairs + 1, sizeof(int64_t));
    int bad = 0;
    /* pass 1: row lengths */
#pragma omp parallel num_threads(nthreads_of(nthreads)) reduction(| : bad)
    {
        double* pts = malloc((size_t)pcap * 2 * sizeof(double));
        double* alpha = malloc((size_t)pcap * sizeof(double));
        Entry* ent = malloc((size_t)pcap * 16 * sizeof(Entry));
#pragma omp for schedule(dynamic, 8)
        for (int32_t k = 0; k < n_pairs; ++k) {
            int e, r;
            if (!pair_of(n_tx, pairs, k, &e, &r)) { bad = 1; continue; }
            TraceRes res;
            trace(&F, R, tx[2 * e], tx[2 * e + 1], tx[2 * r], tx[2 * r + 1], theta[k], ds, pts,
                  alpha, pcap, &res);
            counts[k] = build_row(&F, pts, alpha, res.n_pts, ent);
        }
        free(pts); free(alpha); free(ent);
    }
    row_ptr[0] = 0;
    for (int32_t k = 0; k < n_pairs; ++k) row_ptr[k + 1] = row_ptr[k] + counts[k];
    int64_t nnz = row_ptr[n_pairs];
    free(counts);
    if (bad) { field_free(&F); return -1; }
    if (!col || !val || cap < nnz) { field_free(&F); return nnz; }
    /* pass 2: fill */
#pragma omp parallel num_threads(nthreads_of(nthreads))
    {
        double* pts = malloc((size_t)pcap * 2 * sizeof(double));
        double* alpha = malloc((size_t)pcap * sizeof(double));
        Entry* ent = malloc((size_t)pcap * 16 * sizeof(Entry));
#pragma omp for schedule(dynamic, 8)
        for (int32_t k = 0; k < n_pairs; ++k) {
            int e, r;
            pair_of(n_tx, pairs, k, &e, &r);
            TraceRes res;
            trace(&F, R, tx[2 * e], tx[2 * e + 1], tx[2 * r], tx[2 * r + 1], theta[k], ds, pts,
                  alpha, pcap, &res);
            int64_t n = build_row(&F, pts, alpha, res.n_pts, ent);
            for (int64_t t = 0; t < n; ++t) {
                col[row_ptr[k] + t] = (int32_t)ent[t].node;
                val[row_ptr[k] + t] = ent[t].w;
            }
        }
        free(pts); free(alpha); free(ent);
    }
    field_free(&F);
    return nnz;
}

int orc_adjoint(const orc_grid* g, const double* c_mps, int32_t n_tx, const double* tx,
                double R, int32_t n_pairs, const int32_t* pairs, double ds, const double* theta,
                const double* g_tof, double* g_c, int32_t nthreads) {
    int rc = check_common(g, n_tx, tx, R, ds, n_pairs, pairs);
    if (rc) return rc;
    if (!theta || !g_tof || !g_c) return ORC_EINVAL;
    Field F;
    rc = field_make(&F, g, c_mps);
    if (rc) return rc;
    const size_t nn = (size_t)F.nx * F.ny;
    const int64_t pcap = step_cap(R, ds) + 2;
    const int nt = nthreads_of(nthreads);
    double* acc = calloc((size_t)nt * nn, sizeof(double));
    if (!acc) { field_free(&F); return ORC_ENOMEM; }
    int bad = 0;
#pragma omp parallel num_threads(nt) reduction(| : bad)
    {
#ifdef _OPENMP
        double* gs = acc + (size_t)omp_get_thread_num() * nn;
#else
        double* gs = acc;
#endif
        double* pts = malloc((size_t)pcap * 2 * sizeof(double));
        double* alpha = malloc((size_t)pcap * sizeof(double));
#pragma omp for schedule(dynamic, 8)
        for (int32_t k = 0; k < n_pairs; ++k) {
            int e, r;
            if (!pair_of(n_tx, pairs, k, &e, &r)) { bad = 1; continue; }
            TraceRes res;
            trace(&F, R, tx[2 * e], tx[2 * e + 1], tx[2 * r], tx[2 * r + 1], theta[k], ds, pts,
                  alpha, pcap, &res);
            /* (L^T g)_j = sum_i g_i L_ij with L_ij = sum_m alpha_m phi_j(x_m) */
            for (int64_t m = 0; m < res.n_pts; ++m) {
                Stencil S;
                stencil_at(&F, pts[2 * m], pts[2 * m + 1], &S);
                for (int q = 0; q < S.n; ++q) gs[S.k[q]] += g_tof[k] * alpha[m] * S.w[q];
            }
        }
        free(pts); free(alpha);
    }
    for (size_t j = 0; j < nn; ++j) {
        double sum = 0.0;
        for (int t = 0; t < nt; ++t) sum += acc[(size_t)t * nn + j];
        acc[j] = sum;
    }
    /* S3: T = L (P^-1 s) for the B-spline, so d/ds = P^-T (L^T g) */
    if (g_interp == 1 && bspline_coef(F.nx, F.ny, acc, acc, 1)) bad = 1;
    for (size_t j = 0; j < nn; ++j) {
        /* s = 1000 / c_mps (us/mm)  =>  ds/dc = -1000 / c_mps^2 */
        g_c[j] = -1000.0 * acc[j] / (c_mps[j] * c_mps[j]);
    }
    free(acc);
    field_free(&F);
    return bad ? ORC_EINVAL : ORC_OK;
}
