// rt_internal.h — host-side declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/rt.h"

struct rt_ctx {
    int device = 0;
    std::string err;
    void* field = nullptr;          // packed cells (bilinear or bicubic coefficients)
    size_t field_bytes = 0;
    double* bs_coef = nullptr;      // [2][ny*nx] B-spline coefficients of c and s
    size_t bs_coef_bytes = 0;
    unsigned long long* counters = nullptr;   // [8]: per-status counts, [7] RK4 steps
    int* dflag = nullptr;           // [1]: set by the pack kernel when c <= 0 or NaN
    int* queue = nullptr;           // [1]: work-queue head of the persistent linking kernel
    double* fan = nullptr;          // [n_tx * fan_rays] interception angles of the emitter fans
    int* fan_need = nullptr;        // [n_tx] emitters with at least one cold-start pair
    size_t fan_cap = 0, need_cap = 0;
    void* link_ws = nullptr;        // link rounds with the R12 sub-fan (rt::LinkWork)
    size_t link_ws_bytes = 0;
    double* txphi = nullptr;        // [n_tx] polar angles of the transducers (NaN = off the ring)
    size_t txphi_cap = 0;
    // batch workspace (rt_batch_run): packed fields, fans, flags
    void* batch_ws = nullptr;
    size_t batch_ws_bytes = 0;
    void* scan_tmp = nullptr;       // prefix-sum workspace (path matrix)
    size_t scan_bytes = 0;
    cudaStream_t last_stream = nullptr;
    // ray-Born workspace (rtborn_*): packed field with Hessian, fan-map keys,
    // inside-ring node list, contraction workspace (partial sums, D' tiles;
    // E / W(V) of the SIMT path) and small buffers
    void* born_field = nullptr;
    size_t born_field_bytes = 0;
    void* born_bsf = nullptr;       // per-cell bicubics of c and s (B-spline fans)
    size_t born_bsf_bytes = 0;
    void* born_keys = nullptr;
    size_t born_keys_bytes = 0;
    int* born_idx = nullptr;
    size_t born_idx_bytes = 0;
    int born_idx_key[2] = {0, 0};
    double born_idx_geo[4] = {0, 0, 0, 0};
    int born_n_in = 0;
    void* born_E = nullptr;
    size_t born_E_bytes = 0;
    void* born_W = nullptr;
    size_t born_W_bytes = 0;
    void* born_aux = nullptr;
    size_t born_aux_bytes = 0;
    void* born_acc = nullptr;
    size_t born_acc_bytes = 0;
    void* born_err = nullptr;       // device word: a contraction kernel's bounded wait expired
    size_t born_err_bytes = 0;
};

namespace rt {

struct Geom;

// Fills a Geom for a validated problem; returns RT_OK or RT_EINVAL (message in ctx).
int make_geom(rt_ctx* ctx, const rt_problem* p, const rt_options* o, Geom* G);
// Records an error message on ctx (when not null) and returns code.
int set_error(rt_ctx* ctx, int code, const std::string& msg);
bool stream_capturing(cudaStream_t s);

// Kernel launchers (rt_ray.cu). All enqueue on `s` and return a cudaError_t;
// the field layout (and kernel variant) follows G.interp.
cudaError_t launch_pack(const rt_grid& g, const double* c_mps, void* field, int* dflag, int prec,
                        cudaStream_t s);
struct RowRec;
struct LinkState;
// Workspace of a link split into rounds with the R12 sub-fan (subfan rays per
// pair, > 0): two set-aside state arrays of n_pairs entries, the sub-fan
// misfits [n_pairs * subfan] and five int counters.
struct LinkWork {
    int subfan;
    LinkState* aside;
    double* sub;
    int* ctr;
};
size_t link_state_bytes();
// fan_ds: the fan's tracing step (0 = G.ds); its launch angles follow G.ds.
// rec: record the rows of the system matrix (FP32-compensated bilinear only).
// W (subfan > 0): link in rounds (two traces, the sub-fan, the rest).
cudaError_t launch_link(const Geom& G, const void* field, int prec, double tol, int max_iter,
                        double* theta, double* tof, double* hit, int32_t* status, int32_t* iters,
                        unsigned long long* counters, int* queue, int fan_rays, double fan_ds, double* fan,
                        int* fan_need, cudaStream_t s, const RowRec* rec = nullptr, const LinkWork* W = nullptr);
// adjoint from recorded rows (pairs without one traced again), then the chain rule
cudaError_t launch_adjoint_rows(const Geom& G, const void* field, const double* theta, const double* g_tof,
                                const double* tof_ref, const double* c_mps, const RowRec& rec, double* g_c,
                                cudaStream_t s);
cudaError_t launch_fan(const Geom& G, double fan_ds, const void* field, int prec, int fan_rays, const double* theta,
                       double* fan, int* fan_need, unsigned long long* counters, cudaStream_t s);
cudaError_t launch_tof(const Geom& G, const void* field, int prec, const double* theta, double* tof,
                       double* hit, cudaStream_t s);
cudaError_t launch_adjoint(const Geom& G, const void* field, int prec, const double* theta,
                           const double* g_tof, const double* tof_ref, const double* c_mps,
                           double* g_c, cudaStream_t s);
cudaError_t launch_rows(const Geom& G, const void* field, int prec, const double* theta,
                        int64_t* row_ptr, int32_t* col, double* val, bool fill, cudaStream_t s);
cudaError_t launch_tx_phi(const Geom& G, double* phi, cudaStream_t s);
// B-spline sampler (rt_bspline.cu): nodal c and s -> coefficients (coef [2][ny*nx])
// -> per-cell bicubics in `field`; the line filter of nf planes (transpose: P^-T).
cudaError_t launch_pack_bs(const rt_grid& g, const double* c_mps, double* coef, void* field, int* dflag, int prec,
                           cudaStream_t s);
cudaError_t launch_bs_filter(double* f, int nx, int ny, int nf, bool transpose, cudaStream_t s);
cudaError_t launch_scan(int64_t* row_ptr, int n, void* tmp, size_t* tmp_bytes, cudaStream_t s);

// bytes per packed cell for a precision and interpolator
size_t node_bytes(int prec, int interp = RT_BILINEAR);

// Born contractions (rt_born_tc.cu). Per-frequency constants: f = fh + fl
// (MHz), the absorption exponent factor wy = omega_s^y and the weight
// scale = omega^2 h^2.
struct BornFreq {
    float fh, fl, wy, scale;
};
constexpr int kBornFreqMax = 64;   // frequencies per contraction launch
struct BornTCJob {
    int n_tx, n_freq, n_in;           // n_freq <= kBornFreqMax
    long long nn;             // nodes per map
    const int* idx;           // inside-ring nodes, padded to a multiple of 128 (+128) with node 0
    const float* T;
    const float* A;
    const float* L;           // maps [n_tx][nn]; L NULL without absorption
    const float* dc;          // [nn] (apply only)
    const BornFreq* fq;       // HOST [n_freq], passed to the kernels as parameters
    int chunk;                // apply: K-tiles per accumulation run (0 = the default)
};
// workspace of the tensor-core apply (partial sums) and adjoint (D' tiles)
size_t born_tc_acc_bytes(int n_tx, int n_freq);
size_t born_tc_bd_bytes(int n_tx, int n_freq);
// apply: d [n_freq][n_tx][n_tx] complex64; adjoint: dc_out[idx[p]] (=, or +=
// with accumulate) for the inside nodes (part: [n_freq][n_in] floats of
// workspace); err: device word that a kernel whose bounded wait expired sets,
// after which the finishing kernel writes NaN to the outputs.
cudaError_t launch_born_apply_tc(int device, const BornTCJob& j, float* acc, float2* d, int* err, cudaStream_t s);
cudaError_t launch_born_adjoint_tc(int device, const BornTCJob& j, const float2* d, float* bd, float* part,
                                   float* dc_out, bool accumulate, int* err, cudaStream_t s);
// FP32 SIMT complex GEMM C(m, n) += sum_k A(m, k) B(n, k) (element strides; C pre-zeroed)
cudaError_t launch_cgemm(int M, int N, int K, const float2* A, long long sam, long long sak, const float2* B,
                         long long sbn, long long sbk, float2* C, long long scm, long long scn, int device,
                         cudaStream_t s);

}  // namespace rt
