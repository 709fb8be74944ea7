// rt_api.cu — the C ABI declared in include/rt.h: context, argument checks,
// workspace and kernel launches. No exception crosses the ABI.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "rt_internal.h"
#include "rt_link.cuh"
#include "rt_trace.cuh"

namespace {

int fail(rt_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_fail(rt_ctx* ctx, cudaError_t e, const char* where) {
    return fail(ctx, RT_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

// Grows the packed-field buffer; refuses to allocate while `s` is being captured.
int ensure_field(rt_ctx* ctx, size_t bytes, cudaStream_t s) {
    if (ctx->field_bytes >= bytes) return RT_OK;
    if (capturing(s)) return fail(ctx, RT_EINVAL, "workspace too small during stream capture: call rt_ctx_reserve first");
    if (ctx->field) cudaFree(ctx->field);
    ctx->field = nullptr;
    ctx->field_bytes = 0;
    cudaError_t e = cudaMalloc(&ctx->field, bytes);
    if (e != cudaSuccess) return fail(ctx, RT_ENOMEM, std::string("field workspace: ") + cudaGetErrorString(e));
    ctx->field_bytes = bytes;
    return RT_OK;
}

int set_device(rt_ctx* ctx) {
    cudaError_t e = cudaSetDevice(ctx->device);
    return e == cudaSuccess ? RT_OK : cuda_fail(ctx, e, "cudaSetDevice");
}

int check_options(rt_ctx* ctx, const rt_options* o, bool need_link) {
    if (!o) return fail(ctx, RT_EINVAL, "options pointer is NULL");
    if (o->precision != RT_FP64 && o->precision != RT_FP32_COMP) return fail(ctx, RT_EINVAL, "unknown precision");
    if (!(o->ds_mm > 0) || !std::isfinite(o->ds_mm)) return fail(ctx, RT_EINVAL, "ds_mm must be > 0");
    if (need_link && !(o->tol_mm > 0)) return fail(ctx, RT_EINVAL, "tol_mm must be > 0");
    if (need_link && o->max_iter < 2) return fail(ctx, RT_EINVAL, "max_iter must be >= 2");
    if (o->integrator != RT_RK4 && o->integrator != RT_HEUN) return fail(ctx, RT_EINVAL, "unknown integrator");
    if (o->interpolator != RT_BILINEAR && o->interpolator != RT_BSPLINE)
        return fail(ctx, RT_EINVAL, "unknown interpolator");
    return RT_OK;
}

// Validate, pack the field into the workspace and fill the launch geometry.
int prepare(rt_ctx* ctx, const rt_problem* p, const rt_options* o, bool need_link, cudaStream_t s,
            rt::Geom* G) {
    if (!ctx) return RT_EINVAL;
    ctx->err.clear();
    int rc = check_options(ctx, o, need_link);
    if (rc) return rc;
    rc = rt::make_geom(ctx, p, o, G);
    if (rc) return rc;
    rc = set_device(ctx);
    if (rc) return rc;
    const size_t bytes =
        rt::node_bytes(o->precision, o->interpolator) * (size_t)(p->grid.nx - 1) * (size_t)(p->grid.ny - 1);
    rc = ensure_field(ctx, bytes, s);
    if (rc) return rc;
    cudaError_t e;
    if (o->interpolator == RT_BSPLINE) {
        const size_t cb = 2 * sizeof(double) * (size_t)p->grid.nx * (size_t)p->grid.ny;
        if (ctx->bs_coef_bytes < cb) {
            if (capturing(s)) return fail(ctx, RT_EINVAL, "B-spline workspace too small during stream capture");
            if (ctx->bs_coef) cudaFree(ctx->bs_coef);
            ctx->bs_coef = nullptr;
            ctx->bs_coef_bytes = 0;
            if (cudaMalloc(&ctx->bs_coef, cb) != cudaSuccess) return fail(ctx, RT_ENOMEM, "B-spline workspace");
            ctx->bs_coef_bytes = cb;
        }
        e = rt::launch_pack_bs(p->grid, p->c_mps, ctx->bs_coef, ctx->field, ctx->dflag, o->precision, s);
    } else {
        e = rt::launch_pack(p->grid, p->c_mps, ctx->field, ctx->dflag, o->precision, s);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pack kernel");
    G->bad_field = ctx->dflag;
    // per-transducer polar angles (NaN = off the ring), read by every pair set-up
    const size_t phi_bytes = sizeof(double) * (size_t)p->n_tx;
    if (ctx->txphi_cap < phi_bytes) {
        if (capturing(s)) return fail(ctx, RT_EINVAL, "transducer table too small during stream capture");
        if (ctx->txphi) cudaFree(ctx->txphi);
        ctx->txphi = nullptr;
        ctx->txphi_cap = 0;
        if (cudaMalloc(&ctx->txphi, phi_bytes) != cudaSuccess) return fail(ctx, RT_ENOMEM, "transducer table");
        ctx->txphi_cap = phi_bytes;
    }
    e = rt::launch_tx_phi(*G, ctx->txphi, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "transducer table kernel");
    G->tx_phi = ctx->txphi;
    ctx->last_stream = s;
    return RT_OK;
}

// Fan workspace of a cold-start link (sized outside stream capture).
int ensure_fan(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, cudaStream_t s) {
    if (opt->fan_rays == 1 || opt->fan_rays < 0 || opt->fan_rays > 65536)
        return fail(ctx, RT_EINVAL, "fan_rays must be 0 or in [2, 65536]");
    if (opt->fan_rays < 2) return RT_OK;
    const size_t fan_bytes = sizeof(double) * (size_t)prob->n_tx * (size_t)opt->fan_rays;
    const size_t need_bytes = sizeof(int) * (size_t)prob->n_tx;
    if (ctx->fan_cap >= fan_bytes && ctx->need_cap >= need_bytes) return RT_OK;
    if (capturing(s)) return fail(ctx, RT_EINVAL, "fan workspace too small during stream capture");
    if (ctx->fan_cap < fan_bytes) {
        if (ctx->fan) cudaFree(ctx->fan);
        ctx->fan = nullptr;
        ctx->fan_cap = 0;
        if (cudaMalloc(&ctx->fan, fan_bytes) != cudaSuccess) return fail(ctx, RT_ENOMEM, "fan workspace");
        ctx->fan_cap = fan_bytes;
    }
    if (ctx->need_cap < need_bytes) {
        if (ctx->fan_need) cudaFree(ctx->fan_need);
        ctx->fan_need = nullptr;
        ctx->need_cap = 0;
        if (cudaMalloc(&ctx->fan_need, need_bytes) != cudaSuccess) return fail(ctx, RT_ENOMEM, "fan workspace");
        ctx->need_cap = need_bytes;
    }
    return RT_OK;
}

// Workspace of the R12 rounds (opt->subfan_rays > 0): the set-aside state
// array, the sub-fan misfits and the round counters, 256-byte aligned parts.
static int ensure_link_ws(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, cudaStream_t s,
                          rt::LinkWork* W) {
    W->subfan = 0;
    if (opt->subfan_rays < 0 || opt->subfan_rays > RT_SUBFAN_MAX)
        return fail(ctx, RT_EINVAL, "subfan_rays must be in [0, RT_SUBFAN_MAX]");
    if (opt->subfan_rays == 0 || prob->n_pairs == 0) return RT_OK;
    if (opt->precision != RT_FP32_COMP || opt->interpolator != RT_BILINEAR)
        return fail(ctx, RT_EINVAL, "subfan_rays needs RT_FP32_COMP and RT_BILINEAR");
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t np = (size_t)prob->n_pairs;
    const size_t st = al(rt::link_state_bytes() * np), sb = al(sizeof(double) * np * (size_t)opt->subfan_rays);
    const size_t need = st + sb + 256;
    if (ctx->link_ws_bytes < need) {
        if (capturing(s)) return fail(ctx, RT_EINVAL, "link workspace too small during stream capture");
        if (ctx->link_ws) cudaFree(ctx->link_ws);
        ctx->link_ws = nullptr;
        ctx->link_ws_bytes = 0;
        if (cudaMalloc(&ctx->link_ws, need) != cudaSuccess) return fail(ctx, RT_ENOMEM, "link workspace");
        ctx->link_ws_bytes = need;
    }
    char* b = (char*)ctx->link_ws;
    W->subfan = opt->subfan_rays;
    W->aside = (rt::LinkState*)b;
    W->sub = (double*)(b + st);
    W->ctr = (int*)(b + st + sb);
    return RT_OK;
}

}  // namespace

namespace rt {

int set_error(rt_ctx* ctx, int code, const std::string& msg) { return fail(ctx, code, msg); }
bool stream_capturing(cudaStream_t s) { return capturing(s); }

int make_geom(rt_ctx* ctx, const rt_problem* p, const rt_options* o, Geom* G) {
    if (!p) return fail(ctx, RT_EINVAL, "problem pointer is NULL");
    const rt_grid& g = p->grid;
    if (g.nx < 3 || g.ny < 3) return fail(ctx, RT_EINVAL, "grid must have at least 3 nodes per axis");
    if ((int64_t)g.nx * g.ny > (int64_t)INT32_MAX / 2) return fail(ctx, RT_EINVAL, "grid too large");
    if (!(g.h_mm > 0) || !std::isfinite(g.h_mm) || !std::isfinite(g.x0_mm) || !std::isfinite(g.y0_mm))
        return fail(ctx, RT_EINVAL, "grid spacing/origin invalid");
    if (!p->c_mps) return fail(ctx, RT_EINVAL, "c_mps is NULL");
    if (p->n_tx < 2 || !p->tx_xy_mm) return fail(ctx, RT_EINVAL, "need >= 2 transducers and their positions");
    if (p->n_pairs < 0) return fail(ctx, RT_EINVAL, "n_pairs < 0");
    if (!p->pairs && p->n_pairs != 0 && (int64_t)p->n_pairs != (int64_t)p->n_tx * (p->n_tx - 1))
        return fail(ctx, RT_EINVAL, "pairs == NULL requires n_pairs == n_tx*(n_tx-1)");
    const double R = p->ring_radius_mm;
    if (!(R > 0) || !std::isfinite(R)) return fail(ctx, RT_EINVAL, "ring radius must be > 0");
    if (!(o->fan_ds_mm >= 0.0) || !std::isfinite(o->fan_ds_mm))
        return fail(ctx, RT_EINVAL, "fan_ds_mm must be 0 (= ds_mm) or > 0");
    // the ring plus one step (of the march or, for the fan, of the fan) and one cell
    const double need = R + std::max(o->ds_mm, o->fan_rays >= 2 ? o->fan_ds_mm : 0.0) + g.h_mm;
    const double xl = g.x0_mm, xh = g.x0_mm + (g.nx - 1) * g.h_mm;
    const double yl = g.y0_mm, yh = g.y0_mm + (g.ny - 1) * g.h_mm;
    if (!(-need >= xl && need <= xh && -need >= yl && need <= yh))
        return fail(ctx, RT_EINVAL, "ring (plus one step and one cell) must lie inside the grid");
    const double Rc = R / g.h_mm;
    if (Rc * Rc > 1.0e8 || g.nx > 16384 || g.ny > 16384)
        return fail(ctx, RT_EINVAL, "ring or grid too large (at most 16384 nodes per axis)");
    G->nx = g.nx;
    G->ny = g.ny;
    G->h = g.h_mm;
    G->x0 = g.x0_mm;
    G->y0 = g.y0_mm;
    G->R = R;
    G->inv_R2 = 1.0 / (R * R);
    G->heun = o->integrator == RT_HEUN ? 1 : 0;
    G->interp = o->interpolator == RT_BSPLINE ? RT_BSPLINE : RT_BILINEAR;
    G->ds = o->ds_mm;
    const double ox = -g.x0_mm / g.h_mm, oy = -g.y0_mm / g.h_mm;
    G->Ox = (int)std::floor(ox);
    G->Oy = (int)std::floor(oy);
    G->oxf = ox - G->Ox;
    G->oyf = oy - G->Oy;
    const double R2 = Rc * Rc;
    G->Q = (long long)std::floor(R2);
    G->q = R2 - (double)G->Q;
    G->max_steps = (long long)std::ceil(8.0 * R / o->ds_mm);
    if (G->max_steps > (long long)INT32_MAX - 16) return fail(ctx, RT_EINVAL, "ring too large for the step length");
    G->max_steps_i = (int)G->max_steps;
    G->tx = p->tx_xy_mm;
    G->n_tx = p->n_tx;
    G->pairs = p->pairs;
    G->n_pairs = p->n_pairs;
    G->bad_field = nullptr;
    G->tx_phi = nullptr;
    if (G->Q > (long long)INT32_MAX / 2) return fail(ctx, RT_EINVAL, "ring too large in cells");
    G->Qi = (int)G->Q;
    G->Hf = (float)(o->ds_mm / g.h_mm);
    G->dsf = (float)o->ds_mm;
    G->Rcf = (float)Rc;
    G->oxff = (float)G->oxf;
    G->oyff = (float)G->oyf;
    G->qf = (float)G->q;
    return RT_OK;
}

}  // namespace rt

extern "C" {

int rt_version(void) { return RT_ABI_VERSION; }

int rt_ctx_create(rt_ctx** out, int device) {
    if (!out) return RT_EINVAL;
    *out = nullptr;
    rt_ctx* ctx = new (std::nothrow) rt_ctx();
    if (!ctx) return RT_ENOMEM;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->counters, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->dflag, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->queue, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->counters, 0, 8 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(ctx->dflag, 0, sizeof(int));
    if (e != cudaSuccess) {
        rt_ctx_destroy(ctx);
        return RT_ECUDA;
    }
    *out = ctx;
    return RT_OK;
}

void rt_ctx_destroy(rt_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->field) cudaFree(ctx->field);
    if (ctx->bs_coef) cudaFree(ctx->bs_coef);
    if (ctx->counters) cudaFree(ctx->counters);
    if (ctx->dflag) cudaFree(ctx->dflag);
    if (ctx->queue) cudaFree(ctx->queue);
    if (ctx->scan_tmp) cudaFree(ctx->scan_tmp);
    if (ctx->fan) cudaFree(ctx->fan);
    if (ctx->fan_need) cudaFree(ctx->fan_need);
    if (ctx->link_ws) cudaFree(ctx->link_ws);
    if (ctx->txphi) cudaFree(ctx->txphi);
    if (ctx->batch_ws) cudaFree(ctx->batch_ws);
    for (void* p : {ctx->born_field, ctx->born_bsf, ctx->born_keys, (void*)ctx->born_idx, ctx->born_E, ctx->born_W, ctx->born_aux,
                    ctx->born_acc, ctx->born_err})
        if (p) cudaFree(p);
    delete ctx;
}

const char* rt_last_error(const rt_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int rt_ctx_reserve(rt_ctx* ctx, int64_t max_nodes) {
    if (!ctx) return RT_EINVAL;
    ctx->err.clear();
    if (max_nodes < 0) return fail(ctx, RT_EINVAL, "max_nodes < 0");
    int rc = set_device(ctx);
    if (rc) return rc;
    return ensure_field(ctx, rt::node_bytes(RT_FP64) * (size_t)max_nodes, nullptr);
}

int rt_link(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, double* theta_io, double* tof_us,
            double* hit_xy_mm, int32_t* status, int32_t* iters, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx && !theta_io && prob && prob->n_pairs > 0) return fail(ctx, RT_EINVAL, "theta_io is NULL");
    rt::Geom G;
    int rc = prepare(ctx, prob, opt, true, s, &G);
    if (rc) return rc;
    rc = ensure_fan(ctx, prob, opt, s);
    if (rc) return rc;
    rt::LinkWork W;
    rc = ensure_link_ws(ctx, prob, opt, s, &W);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(ctx->counters, 0, 8 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "counter reset");
    e = rt::launch_link(G, ctx->field, opt->precision, opt->tol_mm, opt->max_iter, theta_io, tof_us, hit_xy_mm,
                        status, iters, ctx->counters, ctx->queue, opt->fan_rays, opt->fan_ds_mm, ctx->fan,
                        ctx->fan_need, s, nullptr, W.subfan ? &W : nullptr);
    return e == cudaSuccess ? RT_OK : cuda_fail(ctx, e, "link kernel");
}

int32_t rt_rows_cap(const rt_problem* prob) {
    if (!prob || !(prob->grid.h_mm > 0) || !(prob->ring_radius_mm > 0)) return 0;
    const double cells = 1.15 * std::sqrt(2.0) * 2.0 * prob->ring_radius_mm / prob->grid.h_mm + 16.0;
    if (!(cells < 1e9)) return 0;
    return ((int32_t)std::ceil(cells) + 3) & ~3;   // a multiple of 4: rows start on 16-byte boundaries
}

static int check_rows(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, const rt_rows* rows) {
    if (!opt) return fail(ctx, RT_EINVAL, "options pointer is NULL");
    if (opt->precision != RT_FP32_COMP || opt->interpolator != RT_BILINEAR)
        return fail(ctx, RT_EINVAL, "recorded rows need RT_FP32_COMP and RT_BILINEAR");
    if (!rows || rows->cap < 1 || (prob && prob->n_pairs > 0 && (!rows->runs || !rows->len)))
        return fail(ctx, RT_EINVAL, "rows: runs, len and cap >= 1 are required");
    return RT_OK;
}

int rt_link_rows(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, double* theta_io, double* tof_us,
                 double* hit_xy_mm, int32_t* status, int32_t* iters, const rt_rows* rows, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!ctx) return RT_EINVAL;
    int rc = check_rows(ctx, prob, opt, rows);
    if (rc) return rc;
    if (!theta_io && prob && prob->n_pairs > 0) return fail(ctx, RT_EINVAL, "theta_io is NULL");
    rt::Geom G;
    rc = prepare(ctx, prob, opt, true, s, &G);
    if (rc) return rc;
    rc = ensure_fan(ctx, prob, opt, s);
    if (rc) return rc;
    rt::LinkWork W;
    rc = ensure_link_ws(ctx, prob, opt, s, &W);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(ctx->counters, 0, 8 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "counter reset");
    const rt::RowRec rec{rows->runs, rows->len, rows->cap};
    e = rt::launch_link(G, ctx->field, opt->precision, opt->tol_mm, opt->max_iter, theta_io, tof_us, hit_xy_mm,
                        status, iters, ctx->counters, ctx->queue, opt->fan_rays, opt->fan_ds_mm, ctx->fan,
                        ctx->fan_need, s, &rec, W.subfan ? &W : nullptr);
    return e == cudaSuccess ? RT_OK : cuda_fail(ctx, e, "link kernel");
}

int rt_tof_adjoint_rows(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, const rt_rows* rows,
                        const double* theta, const double* g_tof, const double* tof_ref, double* g_c, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!ctx) return RT_EINVAL;
    int rc = check_rows(ctx, prob, opt, rows);
    if (rc) return rc;
    if (!g_c) return fail(ctx, RT_EINVAL, "g_c is required");
    if ((!theta || !g_tof) && prob && prob->n_pairs > 0) return fail(ctx, RT_EINVAL, "theta and g_tof are required");
    rt::Geom G;
    rc = prepare(ctx, prob, opt, false, s, &G);
    if (rc) return rc;
    const rt::RowRec rec{rows->runs, rows->len, rows->cap};
    cudaError_t e = rt::launch_adjoint_rows(G, ctx->field, theta, g_tof, tof_ref, prob->c_mps, rec, g_c, s);
    return e == cudaSuccess ? RT_OK : cuda_fail(ctx, e, "adjoint kernel");
}

int rt_tof_forward(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, const double* theta,
                   double* tof_us, double* hit_xy_mm, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx && (!theta || !tof_us) && prob && prob->n_pairs > 0)
        return fail(ctx, RT_EINVAL, "theta and tof_us are required");
    rt::Geom G;
    int rc = prepare(ctx, prob, opt, false, s, &G);
    if (rc) return rc;
    cudaError_t e = rt::launch_tof(G, ctx->field, opt->precision, theta, tof_us, hit_xy_mm, s);
    return e == cudaSuccess ? RT_OK : cuda_fail(ctx, e, "tof kernel");
}

int rt_tof_adjoint(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, const double* theta,
                   const double* g_tof, const double* tof_ref, double* g_c, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx && !g_c) return fail(ctx, RT_EINVAL, "g_c is required");
    if (ctx && (!theta || !g_tof) && prob && prob->n_pairs > 0)
        return fail(ctx, RT_EINVAL, "theta and g_tof are required");
    rt::Geom G;
    int rc = prepare(ctx, prob, opt, false, s, &G);
    if (rc) return rc;
    cudaError_t e =
        rt::launch_adjoint(G, ctx->field, opt->precision, theta, g_tof, tof_ref, prob->c_mps, g_c, s);
    return e == cudaSuccess ? RT_OK : cuda_fail(ctx, e, "adjoint kernel");
}

int rt_path_matrix(rt_ctx* ctx, const rt_problem* prob, const rt_options* opt, const double* theta,
                   int64_t* row_ptr, int32_t* col, double* val, int64_t capacity, int64_t* nnz_out,
                   void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx && (!row_ptr || !nnz_out)) return fail(ctx, RT_EINVAL, "row_ptr and nnz_out are required");
    if (ctx && !theta && prob && prob->n_pairs > 0) return fail(ctx, RT_EINVAL, "theta is required");
    rt::Geom G;
    int rc = prepare(ctx, prob, opt, false, s, &G);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "row_ptr reset");
    e = rt::launch_rows(G, ctx->field, opt->precision, theta, row_ptr, nullptr, nullptr, false, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "row count kernel");
    if (G.n_pairs > 0) {
        size_t need = 0;
        e = rt::launch_scan(row_ptr, G.n_pairs, nullptr, &need, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "scan size");
        if (ctx->scan_bytes < need) {
            if (ctx->scan_tmp) cudaFree(ctx->scan_tmp);
            ctx->scan_tmp = nullptr;
            ctx->scan_bytes = 0;
            e = cudaMalloc(&ctx->scan_tmp, need);
            if (e != cudaSuccess) return fail(ctx, RT_ENOMEM, "scan workspace");
            ctx->scan_bytes = need;
        }
        size_t have = ctx->scan_bytes;
        e = rt::launch_scan(row_ptr, G.n_pairs, ctx->scan_tmp, &have, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "scan");
    }
    int64_t nnz = 0;
    e = cudaMemcpyAsync(&nnz, row_ptr + G.n_pairs, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "nnz readback");
    *nnz_out = nnz;
    if (capacity < nnz || !col || !val) return fail(ctx, RT_ENOMEM, "capacity smaller than nnz (row_ptr is valid)");
    e = rt::launch_rows(G, ctx->field, opt->precision, theta, row_ptr, col, val, true, s);
    return e == cudaSuccess ? RT_OK : cuda_fail(ctx, e, "row fill kernel");
}

int rt_status_counts(rt_ctx* ctx, int64_t counts[8], void* stream) {
    if (!ctx || !counts) return RT_EINVAL;
    ctx->err.clear();
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->last_stream;
    unsigned long long h[8];
    cudaError_t e = cudaMemcpyAsync(h, ctx->counters, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status readback");
    for (int k = 0; k < 8; ++k) counts[k] = (int64_t)h[k];
    int64_t bad = 0;
    for (int k = 1; k < 7; ++k) bad += counts[k];
    return bad ? RT_ENOCONV : RT_OK;
}

}  // extern "C"
