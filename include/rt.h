/*
 * rt.h — C ABI of the GB300-native two-point ray-tracing library
 * (libraytof.so): travel times, their adjoint and the ray-Born operator for
 * ultrasound sound-speed tomography on a 2D grid with a transducer ring,
 * following arXiv:2511.18511.
 *
 * Conventions shared by every call
 * --------------------------------
 * Units: lengths in mm, sound speed in m/s (converted internally to mm/us),
 * travel times in us, frequencies in MHz.
 * Grid: node (i, j), i along x, sits at (x0_mm + i*h_mm, y0_mm + j*h_mm) and
 * is stored row-major at index j*nx + i. The field is sampled off-grid by
 * bilinear interpolation of nodal values, its gradient by bilinear
 * interpolation of central-difference nodal gradients (paper Sec. 3.3.1).
 * Ring: transducer k at tx_xy_mm[2k], tx_xy_mm[2k+1], all on the circle of
 * radius ring_radius_mm centred on (0, 0); the circle plus one step and one
 * cell must lie inside the grid. A pair (e, r) is an emitter-receiver pair
 * (paper Sec. 1: one element fires, the others receive); pairs == NULL means
 * all e != r in emitter-major order (pair k = e*(N-1) + r - (r > e)); n_pairs == 0
 * is a valid empty call.
 * Memory: every array argument is DEVICE memory owned by the caller unless a
 * comment says "host". The library allocates only inside an rt_ctx
 * (workspace that grows on demand and is reused; rt_ctx_reserve sizes it
 * ahead of time). Output arrays are overwritten.
 * Streams: work is enqueued asynchronously on `stream` (a cudaStream_t; NULL
 * = legacy default stream); a call returns once the work is enqueued.
 * Errors: calls return RT_OK or an RT_E* code and never throw. Argument
 * errors are detected on the host before anything is enqueued; the message
 * is available from rt_last_error. Per-pair outcomes are reported in the
 * status arrays (RT_RAY_*), their counts by rt_status_counts.
 * Threads: one rt_ctx must not be used by two host threads at once.
 */
#ifndef RAYTOF_RT_H
#define RAYTOF_RT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RT_ABI_VERSION 4   /* 2: rt_options.interpolator, rt_bspline_coef, rtborn_*_abs;
                              3: rt_options.fan_ds_mm; 4: rt_options.subfan_rays */
#define RT_SUBFAN_MAX 32

enum rt_code {
    RT_OK = 0,
    RT_EINVAL = 1,    /* bad argument: size, pointer, ring outside grid, option */
    RT_ECUDA = 2,     /* a CUDA runtime call failed (message in rt_last_error) */
    RT_ENOCONV = 3,   /* returned only by rt_status_counts: some pairs did not link */
    RT_ETIMEOUT = 4,  /* a bounded device-side wait expired */
    RT_ENOMEM = 5     /* workspace allocation failed, or capacity too small */
};

/* Per-pair status written by rt_link (and the batch call). */
enum rt_ray_status {
    RT_RAY_OK = 0,        /* |x_hit - x_r| <= tol */
    RT_RAY_MAXITER = 1,   /* max_iter traces without reaching tol (closest ray kept) */
    RT_RAY_STEPCAP = 2,   /* no trace reached the ring within ceil(8R/ds) steps */
    /* 3 (a failed bracket) is never written: the two ends of the inward launch
       interval hit the ring on either side of every receiver, so the linking
       always holds a sign-changing bracket */
    RT_RAY_BADINPUT = 4,  /* invalid pair, transducer off the ring, or c <= 0 / NaN */
};

enum rt_precision {
    RT_FP64 = 0,       /* everything in FP64 */
    RT_FP32_COMP = 1   /* FP32 marching and interpolation with cell-local positions,
                          a compensated (double-float) direction and Kahan travel-time
                          sums; FP64 linking updates, landing and endpoint */
};

/* Ray integrator (paper Sec. 3.2.3 lists Heun's second-order Runge-Kutta as
 * its default; classic RK4 is this library's default). */
enum rt_integrator {
    RT_RK4 = 0,        /* classic fourth-order Runge-Kutta */
    RT_HEUN = 1        /* Heun's second-order Runge-Kutta: slopes at the start and
                          at the Euler end point, averaged */
};

/* Field sampler (paper Sec. 3.3.1 offers both; bilinear is its ToF default). */
enum rt_interpolator {
    RT_BILINEAR = 0,   /* c, grad c (central differences at the nodes) and s = 1/c
                          interpolated from the four vertices of the enclosing cell */
    RT_BSPLINE = 1     /* interpolating cubic B-spline: control coefficients, one per
                          node, solve (a[i-1] + 4 a[i] + a[i+1])/6 = f[i] per axis with
                          the mirror extension a[-1] = a[1], a[n] = a[n-2]; c and its
                          analytic gradient from the spline of c, s from the spline
                          of the nodal s; 4 x 4 coefficients per sample */
};

typedef struct {
    int32_t nx, ny;      /* nodes per axis, >= 3 */
    double h_mm;         /* node spacing */
    double x0_mm, y0_mm; /* position of node (0, 0) */
} rt_grid;

typedef struct {
    int32_t precision;   /* enum rt_precision */
    int32_t max_iter;    /* traces per pair in rt_link, >= 2 (30 is the usual) */
    double ds_mm;        /* fixed RK4 step length > 0 */
    double tol_mm;       /* linking tolerance on |x_hit - x_r| > 0 */
    int32_t fan_rays;    /* cold starts: 0 = straight line to the receiver (paper
                            Sec. 3.4.1) with a near-tangent orientation probe; K >= 2 =
                            a fan of K rays per emitter predicts a bracket, the
                            first angle (inverse interpolation through the eight,
                            else four, fan rays around the root) and, when the
                            first trace misses, the second (inverse quartic through
                            that trace and four fan rays); 256 is the binding's
                            default, 768 suits the 512-element ring at 95 mm;
                            ignored by the calls that take fixed angles */
    int32_t block_threads; /* rt_batch_run only: rays (threads) per block of the
                            persistent kernel, 0 (= 128), 64, 128 or 256 */
    int32_t step_unroll;   /* rt_batch_run only: RK4 steps a ray takes between
                            work-queue checks, 0 (= 16), 1 or 16 */
    int32_t blocks_per_sm; /* rt_batch_run only: resident blocks per SM the kernel
                            variant is compiled for (fewer registers, more warps),
                            0 = 512 / block_threads. FP32 variants (threads, steps,
                            blocks): (64,16,8) (64,16,12) (128,16,4) (128,16,5)
                            (128,16,6) (128,1,5) (256,16,2) (256,16,3); FP64:
                            (128,16,1) */
    int32_t integrator;    /* enum rt_integrator: the ray stepper of every trace of
                            the ToF calls and of the rtborn_maps fans */
    int32_t interpolator;  /* enum rt_interpolator: the field sampler of rt_link,
                            rt_tof_forward, rt_tof_adjoint, rt_path_matrix and
                            rtborn_maps (rt_batch_run and rt_tof_forward_noalloc
                            require RT_BILINEAR) */
    double fan_ds_mm;      /* step of the fan start's rays (rt_link, rt_batch_run),
                            0 = ds_mm. The fan only predicts first angles and
                            brackets: its launch angles follow ds_mm and every
                            linking trace uses ds_mm, so a coarser fan (e.g. h/2)
                            links the same rays in about as many traces for a
                            fraction of the fan's cost. With fan_rays >= 2 the
                            ring plus max(ds_mm, fan_ds_mm) and one cell must lie
                            inside the grid. */
    int32_t subfan_rays;   /* rt_link, rt_link_rows: 0 = off; M in [1, RT_SUBFAN_MAX]:
                            when the second trace of a fan-started pair misses, M
                            rays at fan_ds_mm evenly spaced inside its bracket
                            predict the third angle (inverse cubic through the four
                            around the root, else Regula Falsi in the narrowed
                            bracket; reading R12, the oracle's subfan) and the link
                            runs in rounds: every pair's first two traces in one
                            persistent launch, the sub-fan of the pairs still
                            unlinked, then their remaining traces, spread over
                            all warps. Only predictions change: the linked rays
                            stay those of the straight start. On the 1024^2 /
                            512-ring breast workload the rounds cost more than
                            they save (63.7 against 52.7 ms with 8 rays): the
                            last round's chains of up to four more traces run
                            after the bulk instead of beside it. An experimental option: on the fish-eye lens with
                            M = 32, 3 of 65,280 near-tangent pairs (adjacent
                            transducers, 4-6 FP32 traces where the oracle needs 2)
                            end at max_iter, the narrowed bracket holding a jump
                            of the misfit (rays that stop reaching the ring)
                            instead of the root; M = 8 and 16 link every pair
                            there. Workspace: about 0.53 KB + 8 M bytes per pair.
                            RT_FP32_COMP and RT_BILINEAR only; rt_batch_run
                            requires 0. */
} rt_options;

/* One ToF problem: grid, sound speed and ring (paper Sec. 3.1.1: the system
 * matrix maps the N_n grid values to the N_e*N_r pair travel times). */
typedef struct {
    rt_grid grid;
    const double* c_mps;      /* device [ny*nx], sound speed > 0 */
    int32_t n_tx;             /* transducers, >= 2 */
    const double* tx_xy_mm;   /* device [2*n_tx] */
    double ring_radius_mm;
    int32_t n_pairs;          /* number of pairs; n_tx*(n_tx-1) when pairs == NULL */
    const int32_t* pairs;     /* device [2*n_pairs] (e, r), or NULL */
} rt_problem;

typedef struct rt_ctx rt_ctx;

/* Library ABI version (RT_ABI_VERSION of the build). */
int rt_version(void);

/* Create a context bound to CUDA device `device`; *out receives it. */
int rt_ctx_create(rt_ctx** out, int device);
/* Free the context and its workspace (NULL is ignored). */
void rt_ctx_destroy(rt_ctx* ctx);
/* Last error message of this context ("" if none); valid until the next call. */
const char* rt_last_error(const rt_ctx* ctx);
/* Pre-size the workspace for grids of up to max_nodes nodes, so that later
 * calls allocate nothing (needed before capturing calls in a CUDA graph). */
int rt_ctx_reserve(rt_ctx* ctx, int64_t max_nodes);

/*
 * rt_link — shooting-method ray linking with the travel time fused in.
 * Paper Sec. 3.4 (ray linking: the launch direction is adjusted until the
 * misfit between the ray's boundary interception and the receiver centre,
 * parameterised by angle, vanishes; Secant default, Regula Falsi), Sec. 3.2.3
 * (rays evolve x and unit d from the sound speed and its gradient; RK4 at a
 * fixed step here), Sec. 4.2 (trapezoid travel time with the last point
 * replaced by the interception, shortened last step), Sec. 3.4.1 (first
 * linearisation starts from straight rays, later ones warm-start from the
 * previous angles).
 *   theta_io  [n_pairs] launch angle (rad, from +x). In: NaN = cold start
 *             (straight line, or the fan prediction when opt->fan_rays >= 2),
 *             else warm start. Out: angle of the linked ray (the traced ray
 *             closest to the receiver).
 *   tof_us    [n_pairs] travel time of the linked ray (or NULL).
 *   hit_xy_mm [2*n_pairs] boundary interception of the linked ray (or NULL).
 *   status    [n_pairs] enum rt_ray_status (or NULL).
 *   iters     [n_pairs] traces used (or NULL).
 * Status counts of this call can be read with rt_status_counts.
 */
int rt_link(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, double* theta_io,
            double* tof_us, double* hit_xy_mm, int32_t* status, int32_t* iters, void* stream);

/*
 * rt_tof_forward — travel time of every pair for fixed launch angles (one
 * trace each, no linking): the forward ToF operator at the linked rays
 * (paper Sec. 3.2.1, accumulated travel time; Sec. 4.2 quadrature).
 *   theta     [n_pairs] launch angles.
 *   tof_us    [n_pairs] out; hit_xy_mm [2*n_pairs] out (or NULL).
 */
int rt_tof_forward(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt,
                   const double* theta, double* tof_us, double* hit_xy_mm, void* stream);

/*
 * rt_tof_adjoint — transpose of the system matrix applied to travel-time
 * weights, chained to the sound speed (paper Sec. 3.1.1: each row holds the
 * interpolation-weighted path lengths of a pair's ray; Fermat keeps the rays
 * frozen at the linked angles):
 *   g_c[j] = sum_i w_i * dT_i/dc_j = -(1000 / c_j^2) * sum_i w_i L_ij
 * with w_i = g_tof[i] - (tof_ref ? tof_ref[i] : 0). With g_tof = T and
 * tof_ref = measured times this is the gradient of 0.5*||T - T_ref||^2.
 *   theta [n_pairs], g_tof [n_pairs], tof_ref [n_pairs] or NULL,
 *   g_c   [ny*nx] out, in us/(m/s), FP64 (accumulated with FP64 atomics).
 * With RT_BSPLINE the sum runs over the rows of the coefficient matrix and is
 * mapped to the nodes by the transposed prefilter: -(1000/c^2) P^-T L^T w.
 */
int rt_tof_adjoint(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt,
                   const double* theta, const double* g_tof, const double* tof_ref,
                   double* g_c, void* stream);

/*
 * Recorded rows of the system matrix (paper Sec. 3.1.1: each row holds the
 * interpolation-weighted path lengths of a pair's ray; "because of its
 * sparsity, it can be computed and stored explicitly"). rt_link_rows writes
 * them while it links, from the very traces it links with, so that
 * rt_tof_adjoint_rows applies the transpose without tracing the rays again.
 *
 * rt_run: one run of consecutive sample points of a ray inside one cell: the
 * index j*nx + i of the cell's lower-left node and the run's weights of the
 * nodes (i, j), (i+1, j), (i, j+1), (i+1, j+1): the sums over its points of
 * trapezoid weight x bilinear weight (mm), in FP32.
 * rt_rows: caller-owned device storage; pair k's runs at runs[k*cap ..
 * k*cap + len[k]) in the order the ray visits the cells; len[k] = -1 where no
 * row is recorded (the pair did not link to tol, or its ray visited more than
 * cap cells); rt_tof_adjoint_rows traces those pairs again.
 */
typedef struct {
    int32_t node;
    float w00, w10, w01, w11;
} rt_run;

typedef struct {
    rt_run* runs;      /* device [n_pairs * cap] */
    int32_t* len;      /* device [n_pairs] */
    int32_t cap;       /* runs per pair, >= 1 */
} rt_rows;

/* rt_rows_cap — runs per pair that hold every linked ray of the problem with
 * room to spare: 1.15 x the cells a straight diameter crosses diagonally, plus
 * 16, rounded up to a multiple of 4 (1564 for a 95 mm ring on a 0.2 mm grid:
 * 8.2 GB of runs for 261,632 pairs); rays that visit more cells are traced
 * again by rt_tof_adjoint_rows. With a multiple of 4 and a 16-byte aligned
 * runs array every row starts on a 16-byte boundary, which lets
 * rt_tof_adjoint_rows read the rows with 16-byte loads (any other capacity
 * works, with narrower loads). Returns 0 for an invalid problem. */
int32_t rt_rows_cap(const rt_problem* prob);

/*
 * rt_link_rows — rt_link (same arguments and results) that also records, for
 * every pair that links to tol, the row of its linked ray into `rows`. Every
 * trace of a pair records into the pair's slot, so the slot holds the last
 * trace, which is the linked one. RT_FP32_COMP and RT_BILINEAR only
 * (RT_EINVAL otherwise). Writes about 20 bytes per cell a trace visits.
 */
int rt_link_rows(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, double* theta_io,
                 double* tof_us, double* hit_xy_mm, int32_t* status, int32_t* iters, const rt_rows* rows,
                 void* stream);

/*
 * rt_tof_adjoint_rows — rt_tof_adjoint from recorded rows: g_c as written by
 * rt_tof_adjoint with the same theta, g_tof and tof_ref, for rows recorded by
 * rt_link_rows on the same problem and options whose linked angles are theta
 * (pairs without a row are traced again at theta). Each run's four weights
 * are scaled by w_i in FP32 and added to FP64 accumulators, the arithmetic of
 * rt_tof_adjoint, so the two agree up to the order of the FP64 sums. A warp
 * per pair reads its row (coalesced). RT_FP32_COMP and RT_BILINEAR only.
 */
int rt_tof_adjoint_rows(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, const rt_rows* rows,
                        const double* theta, const double* g_tof, const double* tof_ref, double* g_c,
                        void* stream);

/*
 * rt_path_matrix — the explicit sparse system matrix (paper Sec. 3.1.1,
 * "because of its sparsity, it can be computed and stored explicitly"):
 * row i = pair i, column j = node j, L_ij = sum over the ray's sample points
 * of (trapezoid weight * bilinear weight of node j), so that T = L s with
 * s = 1000/c (us/mm). CSR with one group of 4 entries per cell the ray visits;
 * a node shared by two visits appears twice (entries sum; column order is the
 * ray's order, not sorted). With RT_BSPLINE, column j is the slowness spline's
 * control coefficient at node j and L_ij sums (trapezoid weight * B-spline
 * basis weight), 16 entries per cell visit, so that T = L a_s with
 * a_s = rt_bspline_coef(s).
 *   row_ptr   [n_pairs+1] int64 out (always written).
 *   col, val  [capacity] out; filled only when capacity >= nnz.
 *   nnz_out   HOST int64 out: number of entries. The call synchronises the
 *             stream to read it; RT_ENOMEM if capacity < nnz (row_ptr valid).
 */
int rt_path_matrix(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt,
                   const double* theta, int64_t* row_ptr, int32_t* col, double* val,
                   int64_t capacity, int64_t* nnz_out, void* stream);

/*
 * rt_status_counts — synchronises `stream` and copies the per-status pair
 * counts of the last rt_link on this context: counts[s] for s = 0..7 (HOST
 * array), plus counts[7] = total RK4 steps taken by that call. Returns RT_OK
 * when every pair linked, RT_ENOCONV otherwise.
 */
int rt_status_counts(rt_ctx* ctx, int64_t counts[8], void* stream);

/*
 * rt_bspline_coef — control coefficients of the interpolating cubic B-spline
 * of a nodal field (paper Sec. 3.3.1, the spline defined by control points at
 * the grid nodes): a = P^-1 f, P = B_y (x) B_x the spline's values at the nodes,
 * B the (1, 4, 1)/6 tridiagonal matrix of one axis with the mirror extension;
 * with transpose != 0, a = P^-T f (the adjoint's map back to the nodes).
 * Recursive filtering along x, then y, in FP64.
 *   f, a   device [ny*nx] FP64; a == f filters in place (no partial overlap).
 * Errors: RT_EINVAL for nx or ny < 3 or null pointers.
 */
int rt_bspline_coef(rt_ctx* ctx, int32_t nx, int32_t ny, const double* f, double* a, int32_t transpose,
                    void* stream);

/*
 * rt_csr_matvec / rt_csr_rmatvec — products with a system matrix L written by
 * rt_path_matrix (paper Sec. 3.1.1: the sparse matrix of interpolation-weighted
 * path lengths, stored explicitly), for inversion steps that apply the matrix
 * of one linearisation repeatedly at fixed rays (SART, conjugate gradients).
 *   n_rows    rows of L (pairs); n_cols columns (grid nodes, ny*nx).
 *   row_ptr   [n_rows+1] int64, col [nnz] int32, val [nnz] double (device),
 *             as rt_path_matrix writes them; entries whose column lies outside
 *             [0, n_cols) are skipped.
 *   matvec:   y[n_rows] = L x, x [n_cols].
 *   rmatvec:  y[n_cols] = L^T w, w [n_rows]; y is overwritten (FP64 atomics,
 *             so the summation order, and the last bits, vary between calls).
 */
int rt_csr_matvec(rt_ctx* ctx, int32_t n_rows, int32_t n_cols, const int64_t* row_ptr, const int32_t* col,
                  const double* val, const double* x, double* y, void* stream);
int rt_csr_rmatvec(rt_ctx* ctx, int32_t n_rows, int32_t n_cols, const int64_t* row_ptr, const int32_t* col,
                   const double* val, const double* w, double* y, void* stream);

/* One problem of a batch: geometry plus its own outputs (device memory). */
typedef struct {
    rt_problem prob;
    double* theta_io;       /* [n_pairs] in/out, as for rt_link (NaN = cold start) */
    double* tof_us;         /* [n_pairs] out */
    double* hit_xy_mm;      /* [2*n_pairs] out or NULL */
    int32_t* status;        /* [n_pairs] out or NULL */
    int32_t* iters;         /* [n_pairs] out or NULL */
    const double* tof_ref;  /* [n_pairs] measured times, or NULL for no adjoint */
    double* g_c;            /* [ny*nx] out when tof_ref is given: gradient of
                               0.5*||T - tof_ref||^2 w.r.t. c, us^2/(m/s) */
} rt_instance;

/*
 * rt_batch_run — rt_link plus, for instances with tof_ref, the adjoint of the
 * L2 misfit (rt_tof_adjoint with g_tof = T), for n_inst problems of different
 * grids and rings in ONE persistent launch over all their pairs (longest rings
 * first, longest chords first within a ring). Each pair is linked (paper
 * Sec. 3.4) and then retraced by the same lane with its adjoint weight
 * T - T_ref (Sec. 3.1.1), so forward and adjoint share one launch.
 *   inst   HOST array of n_inst descriptors (read during the call).
 * Every per-instance output is as for rt_link / rt_tof_adjoint; status counts
 * (summed over instances) are read with rt_status_counts. The call sizes the
 * context's batch workspace on first use: make one call outside stream
 * capture, after which the same batch (sizes unchanged) can be captured into
 * a CUDA graph and replayed (the instance descriptors travel as a kernel
 * parameter, so a captured launch keeps the descriptors of the call that was
 * captured).
 */
int rt_batch_run(rt_ctx* ctx, int32_t n_inst, const rt_instance* inst, const rt_options* opt, void* stream);

/*
 * rt_tof_forward_noalloc — the same travel times and interceptions as
 * rt_tof_forward, for callers that cannot allocate device memory when they
 * need them: a host that routes all device memory through its own pool, a
 * loop that must not allocate once it runs, or a plugin that only receives
 * input and output buffers. The paper has no counterpart; this is a service
 * of the library.
 * It takes no rt_ctx and calls no allocator (cudaMalloc, cudaFree or any
 * allocating library routine). The packed field lives in a fixed device array
 * of 16 MiB inside the library, which every GPU that loads the library keeps
 * until the process exits: grids of up to 16 MiB / 64 B = 262,144 cells
 * (e.g. 513 x 513 nodes) in RT_FP32_COMP and 131,072 cells in RT_FP64;
 * larger grids return RT_ENOMEM without enqueueing anything.
 * The first call on a device looks up that array's device address with the
 * device current (make that first call before any stream capture). All calls
 * share the one array, which keeps the last call's contents: calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller. The first calls on one device may come from
 * several host threads at once. `stream` (NULL = the legacy default stream)
 * must belong to the current device; a stream of another device returns
 * RT_EINVAL. Arguments and outputs are as for rt_tof_forward, except that only
 * opt->interpolator = RT_BILINEAR is served (RT_BSPLINE returns RT_EINVAL:
 * its packed field and coefficient workspace do not fit the fixed array) and
 * opt->fan_rays is ignored. Returns RT_OK, RT_EINVAL (bad argument),
 * RT_ENOMEM (grid too large) or RT_ECUDA; there is no error message.
 */
int rt_tof_forward_noalloc(const rt_problem* prob, const rt_options* opt, const double* theta,
                           double* tof_us, double* hit_xy_mm, void* stream);


/* ------------------------------------------------------------------ ray-Born
 * The ray-Born operator of arXiv:2511.18511 (Sec. 3.5 and the Appendix): the
 * Green's function from transducer t to a point x is g = A_t(x) exp(i omega
 * T_t(x)), with the phase from the eikonal (travel time along rays) and the
 * geometric amplitude from the transport equation through the ray Jacobian,
 * which a paraxial ray traced with each ray supplies (Sec. 3.5, default). The
 * backward Green's functions of the receivers are the same per-transducer maps
 * (reciprocity). The *_abs variants add absorption (Appendix: wavenumber
 * k + i alpha, alpha = alpha0 omega^y, A = A_geom A_abs with A_abs accumulated
 * along the ray); the plain calls are the *_abs calls without it (A_abs = 1).
 */

/* Penalty (us) of the squared distance to the ray, in grid steps, in the
 * amplitude choice of rtborn_maps. */
#define RTBORN_ETA_US 1e-2f

/* Contraction arithmetic of rtborn_apply / rtborn_adjoint (complex64 in and
 * out). Both are this library's kernels. */
enum rtborn_gemm {
    RTBORN_GEMM_FP32 = 0,    /* FP32 multiply-add on the CUDA cores: E and W formed
                                in workspace (2 x 8 n_tx n_in bytes), then a tiled
                                complex GEMM per frequency */
    RTBORN_GEMM_TF32X3 = 1   /* tensor cores (tcgen05, kind::tf32, accumulators in
                                tensor memory): every operand value split into two
                                TF32 terms, hi = tf32(v), lo = tf32(v - hi), and each
                                product formed as hi*hi + hi*lo + lo*hi (~2^-21
                                relative error per product, FP32 accumulation); E is
                                formed inside the kernels from the maps, d's symmetry
                                d[e][r] = d[r][e] halves the work (only blocks of
                                128 x 128 transducers with e-block <= r-block are
                                contracted). The default. */
};

/*
 * rtborn_maps — first-arrival travel-time and amplitude maps of every
 * transducer, from a fan of fan_rays rays per transducer at evenly spaced
 * angles over the inward half-plane (tangents excluded by a margin ds/R).
 * Each ray is marched with RK4 (or Heun's RK2, opt->integrator) at the fixed
 * step opt->ds_mm (<= h) together
 * with its paraxial ray (Q, P): dQ/ds = c P, dP/ds = -(c_nn/c^2) Q, Q(0) = 0,
 * P(0) = 1/c_t, c_nn the second derivative of c across the ray (central
 * second differences interpolated bilinearly); the travel time by the
 * trapezoid rule over the interpolated slowness; A = sqrt(c/(c_t max(|Q|, h))).
 * Every sample point offers each node of the 3 x 3 block around its nearest
 * node whose foot on the ray lies within half a step (a = d.D in [-ds/2, ds/2),
 * D = node - point, b = n.D) the second-order ray-centred extrapolation from
 * that foot, T + s a + (P/Q_f)/2 b^2 with Q_f = Q + a c P (|Q_f| clamped to
 * >= h where P/Q_f < 0), and A from Q_f. A node's time is its earliest
 * candidate (first arrival); its amplitude is that of the candidate of least
 * T + RTBORN_ETA_US (b/h)^2 (then the smaller A), i.e. of the ray passing
 * closest to the node; as the first-arrival branch passes within h/2 of every
 * node it reaches, another branch supplies A only if it arrives within
 * RTBORN_ETA_US / 4 of the first.
 *   prob      grid, c_mps, n_tx, tx_xy_mm, ring_radius_mm (pairs ignored).
 *   opt       precision must be RT_FP32_COMP; ds_mm in (0, h]; blocks_per_sm
 *             picks the fan kernel variant (resident 128-thread blocks per SM
 *             it is compiled for): 0 (= 6, or 5 with absorption), 4, 5, 6 or 8;
 *             interpolator RT_BSPLINE takes c, its gradient and its Hessian
 *             from the interpolating cubic B-spline of c (analytic derivatives;
 *             the paper's choice for ray-Born, Sec. 3.3.1) and s from the spline
 *             of s, instead of the bilinear central differences; others ignored.
 *   fan_rays  rays per fan in [2, 2^20]; about 4 pi R / h covers the far side
 *             of the ring at one ray per half grid step.
 *   T_out     [n_tx][ny*nx] float out, us; +inf where no ray arrives.
 *   A_out     [n_tx][ny*nx] float out, amplitude (mm^-1/2); 0 where none.
 * Workspace: 12 bytes per map entry (n_tx * nx * ny) plus 32 bytes per node.
 * rt_status_counts afterwards reports counts[7] = RK4 steps of the fans
 * (counts[0..6] = 0).
 * A sound speed <= 0 or NaN anywhere leaves every entry unreached.
 */
int rtborn_maps(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, int32_t fan_rays,
                float* T_out, float* A_out, void* stream);

/*
 * rtborn_apply — the linearised Born map (Appendix: Helmholtz model with the
 * ray Green's functions; scattered data from a sound-speed perturbation):
 *   d[f][e][r] = omega_f^2 h^2 sum_{|x_n| < R} E_e(x_n) E_r(x_n) dc(x_n), e != r,
 *   d[f][e][e] = 0,  E_t = A_t exp(i omega_f T_t) (0 where T_t = inf),
 * omega_f = 2 pi f_mhz[f] rad/us, over the grid nodes strictly inside the ring
 * of radius ring_radius_mm. The physical prefactors of the scattering
 * potential (-2/c^3 and the source spectrum) are left to the caller.
 *   T, A      [n_tx][ny*nx] maps as written by rtborn_maps.
 *   f_mhz     HOST [n_freq] frequencies (MHz).
 *   dc_mps    [ny*nx] float perturbation (m/s).
 *   gemm_mode enum rtborn_gemm.
 *   d_out     [n_freq][n_tx][n_tx] complex64 out, interleaved (re, im) floats.
 * The first call for a grid and ring builds the list of inside nodes on the
 * host and synchronises the stream once. Workspace (reused over calls):
 * RTBORN_GEMM_TF32X3 128 KB per frequency and 128 x 128 block pair (10 MB
 * for 512 transducers and 8 frequencies); RTBORN_GEMM_FP32 2 x 8 bytes x
 * n_tx x (inside nodes). A tensor-core launch whose bounded device wait
 * expires (2 s without progress) writes NaN to every output of the call
 * instead of hanging.
 */
int rtborn_apply(rt_ctx* ctx, const rt_grid* grid, double ring_radius_mm, int32_t n_tx, const float* T,
                 const float* A, int32_t n_freq, const double* f_mhz, const float* dc_mps,
                 int32_t gemm_mode, float* d_out, void* stream);

/*
 * rtborn_adjoint — the adjoint of rtborn_apply under Re<a, b> = Re sum
 * conj(a) b on the data and the plain dot product on dc:
 *   dc_out[x] = Re sum_f omega_f^2 h^2 sum_{e != r} conj(E_e(x) E_r(x)) d[f][e][r]
 * for nodes inside the ring, 0 elsewhere (the diagonal of d is ignored).
 *   d_in      [n_freq][n_tx][n_tx] complex64, interleaved.
 *   dc_out    [ny*nx] float out.
 * Only the symmetric part of d contributes (E_e E_r is symmetric in e, r).
 * Workspace with RTBORN_GEMM_TF32X3: 512 KB per frequency and 128 x 128
 * block pair (the split, pre-swizzled operand tiles of d; 40 MB for 512
 * transducers and 8 frequencies) plus 4 bytes per inside node and frequency.
 * Other arguments as for rtborn_apply.
 */
int rtborn_adjoint(rt_ctx* ctx, const rt_grid* grid, double ring_radius_mm, int32_t n_tx, const float* T,
                   const float* A, int32_t n_freq, const double* f_mhz, const float* d_in,
                   int32_t gemm_mode, float* dc_out, void* stream);

/*
 * rtborn_maps_abs — rtborn_maps plus the absorption path integral of every
 * map entry: each fan ray also carries Lambda = int alpha0 ds (ds in metres;
 * trapezoid rule over the bilinearly interpolated alpha0, Kahan-summed); a
 * node's candidate is Lambda + alpha0 a from its foot (first order along the
 * ray), and the node keeps the Lambda of the candidate that supplies A (the
 * same least score; an exact tie of scores may pair A and Lambda of different
 * rays).
 *   alpha0    device [ny*nx] double, Np (rad/s)^-y m^-1, >= 0 (a negative or
 *             NaN value leaves every entry unreached, like a bad c); NULL =
 *             no absorption (then L_out is not written and may be NULL).
 *   L_out     [n_tx][ny*nx] float out, Np (rad/s)^-y; 0 where unreached.
 * Workspace: 20 bytes per map entry with alpha0 (12 without).
 */
int rtborn_maps_abs(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, int32_t fan_rays,
                    const double* alpha0, float* T_out, float* A_out, float* L_out, void* stream);

/*
 * rtborn_apply_abs / rtborn_adjoint_abs — rtborn_apply / rtborn_adjoint with
 * E_t = A_t exp(-omega_s^y L_t) exp(i omega T_t), omega_s = 2 pi f 1e6 rad/s.
 *   L         [n_tx][ny*nx] float, as written by rtborn_maps_abs; NULL = none.
 *   y         power-law exponent in [0, 3] (soft tissue 1 < y <= 1.5); with L,
 *             every frequency must be >= 0 and omega_s^y finite in FP32.
 * Other arguments and errors as for rtborn_apply / rtborn_adjoint.
 */
int rtborn_apply_abs(rt_ctx* ctx, const rt_grid* grid, double ring_radius_mm, int32_t n_tx, const float* T,
                     const float* A, const float* L, double y, int32_t n_freq, const double* f_mhz,
                     const float* dc_mps, int32_t gemm_mode, float* d_out, void* stream);
int rtborn_adjoint_abs(rt_ctx* ctx, const rt_grid* grid, double ring_radius_mm, int32_t n_tx, const float* T,
                       const float* A, const float* L, double y, int32_t n_freq, const double* f_mhz,
                       const float* d_in, int32_t gemm_mode, float* dc_out, void* stream);

/* ------------------------------------------------------- measurement service
 * Microbenchmarks of the hardware rates that the kernels above are measured
 * against (the paper reports no timing and has no counterpart). Each call
 * enqueues one kernel of `blocks` x 256 threads on `stream`; the caller times
 * it with events on that stream and divides the work stated here by the time.
 * Every pointer is device memory; `sink` receives one value per thread
 * (blocks * 256 elements of the stated type) so that no work is elided.
 * Returns RT_OK, RT_EINVAL (bad argument, nothing enqueued) or RT_ECUDA.
 *
 * rt_peak_fma — dtype 0: FP32, 1: FP64 (sink of that type); iters a positive
 *   multiple of 8; 8 independent fused multiply-add chains per thread and
 *   iteration: FLOPs = blocks * 256 * iters * 16.
 * rt_peak_gather — iters x 8 random 16-byte loads per thread from buf
 *   (n_vec float4, n_vec a power of two <= 2^28; 16 MiB = 2^20 float4 stays
 *   resident in L2): useful bytes = blocks * 256 * iters * 128.
 * rt_peak_read — `passes` coalesced sweeps of the whole grid over buf (n_vec
 *   float4): bytes = passes * n_vec * 16.
 */
int rt_peak_fma(int32_t dtype, int32_t blocks, int32_t iters, void* sink, void* stream);
int rt_peak_gather(const void* buf, int64_t n_vec, int32_t blocks, int32_t iters, float* sink, void* stream);
int rt_peak_read(const void* buf, int64_t n_vec, int32_t blocks, int32_t passes, float* sink, void* stream);

/*
 * rt_wait_selftest — exercises the bounded device wait that the tensor-core
 * Born kernels use on every pipeline barrier (wait for a barrier phase for at
 * most a limit of global time, then record an error code and return instead
 * of hanging). One block initialises a shared-memory barrier expecting one
 * arrival; with arrive != 0 a thread arrives, otherwise nothing does; the
 * thread then waits on it for at most limit_ns (1e3 .. 2e9 ns). *err (device
 * int32) receives 0 when the phase completed and 199 when the wait gave up.
 * Enqueues one kernel on `stream`; the caller synchronises and reads *err.
 * Returns RT_OK, RT_EINVAL (bad argument, nothing enqueued) or RT_ECUDA.
 */
int rt_wait_selftest(int64_t limit_ns, int32_t arrive, int32_t* err, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RAYTOF_RT_H */
