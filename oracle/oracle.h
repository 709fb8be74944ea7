/*
 * FP64 CPU oracle for two-point ray tracing in a gridded 2D sound-speed image.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls
 * this code: only the tests, the smoke check and the benchmark's CPU baseline
 * do. It shares no code, header, table or helper with the CUDA library.
 *
 * The oracle follows the paper (arXiv:2511.18511) step by step:
 *   - the field and its gradient live on grid nodes and are sampled off-grid by
 *     bilinear interpolation, the gradient being interpolated from grid values
 *     (Sec. 3.3.1, "Bilinear interpolation"), or optionally by a cubic B-spline
 *     whose control points sit at the nodes, with the analytic gradient
 *     (Sec. 3.3.1, "Cubic B-spline interpolation");
 *   - rays evolve position x and unit direction d from the sound speed and its
 *     gradient (Sec. 3.2.3; the eikonal/Fermat model of the Appendix), marched
 *     with classic RK4 at a fixed step ds;
 *   - the shooting method links each emitter-receiver pair by a root search on
 *     the launch angle for the boundary-interception misfit (Sec. 3.4, Secant
 *     default with Regula-Falsi safeguard);
 *   - the travel time is the trapezoid line integral of slowness with the last
 *     point replaced by the boundary interception (Sec. 4.2, acoustic-length
 *     trapezoid rule with the shortened last step ds');
 *   - the system-matrix row of a pair holds interpolation-weighted path
 *     lengths (Sec. 3.1.1), and the adjoint is its transpose.
 *
 * Units: mm, us, mm/us inside; sound speed is passed in m/s (1 m/s = 1e-3
 * mm/us), travel times come back in us, gradients per (m/s).
 * Grid node (i, j) sits at (x0 + i h, y0 + j h), row-major index j*nx + i.
 */
#ifndef RT_ORACLE_H
#define RT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { int32_t nx, ny; double h, x0, y0; } orc_grid;

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2 };
/* per-ray status */
enum { ORC_RAY_OK = 0, ORC_RAY_MAXITER = 1, ORC_RAY_STEPCAP = 2, ORC_RAY_BADINPUT = 4 };

/* Nodal field in mm/us units: c, dc/dx, dc/dy (central differences inside,
 * one-sided at the edges) and slowness s = 1/c. */
int orc_field(const orc_grid* g, const double* c_mps, double* c, double* gx, double* gy, double* s);

/* Samples of (c, dc/dx, dc/dy, s) at n points xy[2n] by the current
 * interpolator; out[4n]. */
int orc_sample(const orc_grid* g, const double* c_mps, int32_t n, const double* xy, double* out);

/* n_steps fixed RK4 steps of size ds from (x, y) at angle theta; writes the
 * n_steps+1 positions to xy_out[2(n_steps+1)]. */
int orc_march(const orc_grid* g, const double* c_mps, double x, double y, double theta,
              double ds, int32_t n_steps, double* xy_out);

/* One trace from (xe, ye) at angle theta until the first boundary crossing of
 * the circle |x| = R, landing exactly on it. out6 = {T, hit_x, hit_y, d_x, d_y, ds'};
 * T includes the endpoint correction toward (xr, yr). If pts/alpha are given
 * (capacity cap) the sample points and their trapezoid weights are written and
 * *n_pts is set. *flags: bit0 step cap hit, bit1 ray left outward at once. */
int orc_trace(const orc_grid* g, const double* c_mps, double R, double xe, double ye,
              double xr, double yr, double theta, double ds, int64_t cap, double* pts,
              double* alpha, int64_t* n_pts, double* out6, int32_t* flags);

/* Link every pair (pairs[2k], pairs[2k+1]) or, with pairs == NULL, all e != r
 * emitter-major. theta_io: NaN = cold start, else warm start; on return the
 * linked angle. Cold starts use the straight line to the receiver when
 * fan_rays == 0, else a fan of fan_rays (>= 2) rays per emitter predicts the
 * first angle and a bracket; the fan's rays are traced at step fan_ds (0 = ds;
 * their launch angles follow ds). subfan (0..ORC_SUBFAN_MAX, fan starts only):
 * after a second missed trace, subfan rays at fan_ds inside the bracket refine
 * it before the third (reading R12). Outputs may be NULL. */
#define ORC_SUBFAN_MAX 32
int orc_link(const orc_grid* g, const double* c_mps, int32_t n_tx, const double* tx,
             double R, int32_t n_pairs, const int32_t* pairs, double ds, double tol,
             int32_t max_iter, int32_t fan_rays, double fan_ds, int32_t subfan, double* theta_io, double* tof,
             double* hit_xy, int32_t* status, int32_t* iters, int32_t nthreads);

/* R12 sub-fan pieces, for tests: the M ray angles inside a bracket (ta, tb),
 * and the prediction from a sequence of n (angle, misfit, place) entries
 * (bracket end of negative misfit at place 0, the sub-fan rays that reached
 * the ring at their ray index q, the other bracket end at M + 1) around c3,
 * the plain rule's third angle, for ring radius R: out7 = {third
 * angle, new ta, new tb, secant start angle and misfit, 1 when the new
 * bracket changes sign, 1 when refined (else the angle is c3 and the bracket
 * the sequence's ends)}. */
int orc_subfan_angles(double ta, double tb, int32_t M, double* theta);
int orc_subfan_predict(int32_t n, const double* st, const double* sm, const int32_t* pos, double c3, double R,
                       double* out7);

/* Travel time (and hit) of every pair at the given angles, no linking. */
int orc_tof(const orc_grid* g, const double* c_mps, int32_t n_tx, const double* tx,
            double R, int32_t n_pairs, const int32_t* pairs, double ds, const double* theta,
            double* tof, double* hit_xy, int32_t nthreads);

/* Explicit CSR system matrix L (rows = pairs, cols = nodes), T = L s; with
 * the B-spline the columns are the slowness spline's control coefficients,
 * T = L a_s with a_s = orc_bspline_coef(s). Returns nnz (>= 0) or -1 on
 * error. With col == NULL only counts. Rows may repeat a column. */
int64_t orc_path_matrix(const orc_grid* g, const double* c_mps, int32_t n_tx, const double* tx,
                        double R, int32_t n_pairs, const int32_t* pairs, double ds,
                        const double* theta, int64_t* row_ptr, int32_t* col, double* val,
                        int64_t cap, int32_t nthreads);

/* Adjoint: g_c[node] = d(sum_i g_tof[i] T_i)/d c_node in us/(m/s) with the
 * rays frozen at theta, i.e. -(L^T g)_j * 1000 / c_j^2 (B-spline:
 * -(P^-T L^T g)_j * 1000 / c_j^2). */
int orc_adjoint(const orc_grid* g, const double* c_mps, int32_t n_tx, const double* tx,
                double R, int32_t n_pairs, const int32_t* pairs, double ds, const double* theta,
                const double* g_tof, double* g_c, int32_t nthreads);

int orc_num_threads(void);

/* Integrator of every later trace (process-wide): 0 = classic RK4 (default),
 * 1 = Heun's second-order Runge-Kutta. Returns ORC_EINVAL for other values. */
int orc_set_integrator(int32_t k);

/* Interpolator of every later sample, trace, matrix row and adjoint
 * (process-wide): 0 = bilinear with interpolated nodal gradient (default),
 * 1 = interpolating cubic B-spline with control points at the nodes and
 * analytic gradient (Sec. 3.3.1). Returns ORC_EINVAL for other values. */
int orc_set_interpolator(int32_t k);
int orc_get_interpolator(void);
int orc_get_integrator(void);

/* Linking rule of every later fan-started orc_link (process-wide): 0 = R8
 * (default), 1 = R13, the fan model corrected through the traces for the
 * second and third angles. Returns ORC_EINVAL for other values. */
int orc_set_link_rule(int32_t k);
int orc_get_link_rule(void);

/* R13's angle from the fan rays (t[q], m[q]), q < n <= 8: the root in (lo, hi)
 * of their interpolating polynomial moved onto the trace (x1, m1) by an
 * offset, or with two = 1 onto both traces (x1, m1), (x2, m2) by an offset and
 * a tilt; *out = NAN when the moved polynomial does not change sign there. */
int orc_r13_angle(const double* t, const double* m, int32_t n, double x1, double m1, double x2, double m2,
                  int32_t two, double lo, double hi, double* out);

/* Control coefficients a = P^-1 f of the interpolating cubic B-spline of the
 * nodal field f[ny*nx] (mirror boundary; P is the spline's value at the nodes,
 * one tridiagonal (1, 4, 1)/6 factor per axis), or a = P^-T f with transpose.
 * a may alias f. */
int orc_bspline_coef(const orc_grid* g, const double* f, double* a, int32_t transpose);

/* ---- ray-Born (born.c) ------------------------------------------------ */

/* Fan angles of transducer (xe, ye): theta_k = a_min + k * step, k < K. */
int orc_fan_angles(double xe, double ye, double R, double ds, int32_t K, double* a_min, double* step);

/* One fan ray with its paraxial ray; per sample point 9 values
 * (x, y, dx, dy, T, Q, P, c, s) into rec9 (capacity cap points);
 * *n_out = the number of points (may exceed cap). */
int orc_fan_ray(const orc_grid* g, const double* c_mps, double R, double xe, double ye, double theta,
                double ds, int64_t cap, double* rec9, int64_t* n_out);

/* First-arrival travel-time and amplitude maps of every transducer from a
 * fan of K rays each: T, A [n_tx][ny*nx] (T = +inf, A = 0 where unreached);
 * A from the candidate of least T + eta (b/h)^2, b its distance to the ray. */
int orc_fan_maps(const orc_grid* g, const double* c_mps, int32_t n_tx, const double* tx, double R,
                 double ds, int32_t K, double eta, double* T, double* A, int32_t nthreads);

/* Born map: d[f][q] = omega^2 h^2 sum_{|x| < R} E_e E_r dc (complex, interleaved)
 * for the listed pairs q = (e, r), or all n_tx x n_tx with pairs == NULL. */
int orc_born_apply(const orc_grid* g, double R, int32_t n_tx, const double* T, const double* A,
                   int32_t n_freq, const double* f_mhz, const double* dc, int32_t n_pairs,
                   const int32_t* pairs, double* d_out, int32_t nthreads);

/* Its adjoint: dc[x] from d[n_freq][n_tx][n_tx] (complex, interleaved). */
int orc_born_adjoint(const orc_grid* g, double R, int32_t n_tx, const double* T, const double* A,
                     int32_t n_freq, const double* f_mhz, const double* d_in, double* dc_out,
                     int32_t nthreads);

/* With absorption (the Appendix's alpha = alpha0 omega^y): alpha0 [ny*nx] in
 * Np (rad/s)^-y m^-1 (>= 0; NULL = none) gives, besides T and A, the path
 * integral Lam [n_tx][ny*nx] = int alpha0 ds (ds in m) of the ray that
 * supplies A (0 where unreached; Lam may be NULL). */
int orc_fan_maps_abs(const orc_grid* g, const double* c_mps, const double* alpha0, int32_t n_tx,
                     const double* tx, double R, double ds, int32_t K, double eta, double* T, double* A,
                     double* Lam, int32_t nthreads);

/* Born map and adjoint with E_t = A_t exp(-omega_s^y Lam_t) exp(i omega T_t),
 * omega_s = 2 pi f 1e6 rad/s, y >= 0 (Lam NULL: no absorption). */
int orc_born_apply_abs(const orc_grid* g, double R, int32_t n_tx, const double* T, const double* A,
                       const double* Lam, double y, int32_t n_freq, const double* f_mhz, const double* dc,
                       int32_t n_pairs, const int32_t* pairs, double* d_out, int32_t nthreads);
int orc_born_adjoint_abs(const orc_grid* g, double R, int32_t n_tx, const double* T, const double* A,
                         const double* Lam, double y, int32_t n_freq, const double* f_mhz, const double* d_in,
                         double* dc_out, int32_t nthreads);

#ifdef __cplusplus
}
#endif
#endif
