"""GB300-native two-point ray tracing for ultrasound sound-speed tomography.

Python binding of ``libraytof.so`` (C ABI in ``include/rt.h``). Every array is
a CUDA torch tensor; the functions only marshal pointers and sizes, all work
runs in the library's kernels on the current torch stream. PyTorch supplies
device memory, streams and the autograd wrapper.

Units: mm, m/s, us (see ``include/rt.h``). Paper: arXiv:2511.18511.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional

import torch

from . import _lib as _L
from .phantoms import Grid

__all__ = ["Context", "Problem", "rt_link", "rt_link_rows", "rt_tof_adjoint_rows", "Rows", "rt_tof_forward", "rt_tof_adjoint", "rt_path_matrix",
           "rt_status_counts", "rt_batch_run", "BatchInstance", "ToF", "tof", "PRECISIONS",
           "BornMaps", "rtborn_maps", "rtborn_apply", "rtborn_adjoint", "Born", "born", "GEMM_MODES"]

PRECISIONS = {"fp64": _L.RT_FP64, "fp32c": _L.RT_FP32_COMP}
INTEGRATORS = {"rk4": 0, "heun": 1}
INTERPOLATORS = {"bilinear": 0, "bspline": 1}


class Context:
    """An ``rt_ctx`` on one CUDA device (workspace owner)."""

    def __init__(self, device: Optional[int] = None):
        self.lib = _L.load()
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = C.c_void_p()
        _L.check(None, self.lib.rt_ctx_create(C.byref(h), self.device))
        self.h = h

    def reserve(self, max_nodes: int):
        _L.check(self.h, self.lib.rt_ctx_reserve(self.h, int(max_nodes)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.rt_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_contexts: dict[int, Context] = {}


def default_context(device: Optional[int] = None) -> Context:
    d = torch.cuda.current_device() if device is None else int(device)
    if d not in _contexts:
        _contexts[d] = Context(d)
    return _contexts[d]


def _stream(stream) -> C.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev_f64(x, device) -> torch.Tensor:
    t = torch.as_tensor(x, dtype=torch.float64, device=device)
    return t.contiguous()


@dataclasses.dataclass
class Problem:
    """Grid + sound speed + ring (device tensors), the rt_problem of the ABI."""
    grid: Grid
    c: torch.Tensor                   # float64 [ny, nx] m/s, CUDA
    tx: torch.Tensor                  # float64 [N, 2] mm, CUDA
    ring_radius: float
    pairs: Optional[torch.Tensor] = None   # int32 [P, 2] or None = all e != r

    @staticmethod
    def create(grid: Grid, c, tx, ring_radius: float, pairs=None, device="cuda") -> "Problem":
        p = None if pairs is None else torch.as_tensor(pairs, dtype=torch.int32, device=device).contiguous()
        return Problem(grid, _dev_f64(c, device), _dev_f64(tx, device), float(ring_radius), p)

    @property
    def n_tx(self) -> int:
        return int(self.tx.shape[0])

    @property
    def n_pairs(self) -> int:
        return self.n_tx * (self.n_tx - 1) if self.pairs is None else int(self.pairs.shape[0])

    def struct(self, c: Optional[torch.Tensor] = None) -> _L.RtProblem:
        c = self.c if c is None else c
        if c.dtype != torch.float64 or not c.is_cuda or not c.is_contiguous():
            raise ValueError("c must be a contiguous float64 CUDA tensor")
        if c.numel() != self.grid.nx * self.grid.ny:
            raise ValueError("c has the wrong number of nodes")
        g = _L.RtGrid(self.grid.nx, self.grid.ny, self.grid.h, self.grid.x0, self.grid.y0)
        return _L.RtProblem(g, c.data_ptr(), self.n_tx, self.tx.data_ptr(), self.ring_radius,
                            self.n_pairs, None if self.pairs is None else self.pairs.data_ptr())


DEFAULT_FAN = 256


def _opts(ds, tol=1e-4, max_iter=30, precision="fp32c", fan_rays=DEFAULT_FAN, block_threads=0,
          step_unroll=0, blocks_per_sm=0, integrator="rk4", interpolator="bilinear", fan_ds=0.0,
          subfan_rays=0) -> _L.RtOptions:
    if precision not in PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
    if integrator not in INTEGRATORS:
        raise ValueError(f"integrator must be one of {sorted(INTEGRATORS)}")
    if interpolator not in INTERPOLATORS:
        raise ValueError(f"interpolator must be one of {sorted(INTERPOLATORS)}")
    return _L.RtOptions(PRECISIONS[precision], int(max_iter), float(ds), float(tol), int(fan_rays),
                        int(block_threads), int(step_unroll), int(blocks_per_sm), INTEGRATORS[integrator],
                        INTERPOLATORS[interpolator], float(fan_ds), int(subfan_rays))


def rt_link(prob: Problem, ds: float, tol: float = 1e-4, max_iter: int = 30, precision: str = "fp32c",
            theta0: Optional[torch.Tensor] = None, c: Optional[torch.Tensor] = None,
            ctx: Optional[Context] = None, stream=None, out: Optional[dict] = None,
            fan_rays: int = DEFAULT_FAN, integrator: str = "rk4", interpolator: str = "bilinear",
            fan_ds: float = 0.0, subfan_rays: int = 0) -> dict:
    """Link every pair (shooting method, paper Sec. 3.4) and return the linked
    angles, travel times (us), interceptions (mm), per-pair status and traces.
    Cold starts (theta0 None / NaN) use a fan of fan_rays rays per emitter, or
    the straight line to the receiver with fan_rays = 0; the fan's rays are
    traced at step fan_ds (0 = ds), their launch angles follow ds. integrator: "rk4" or
    "heun" (the paper's default stepper); interpolator: "bilinear" or "bspline"
    (the interpolating cubic B-spline, Sec. 3.3.1). subfan_rays > 0: link in
    rounds (every pair's first two traces, the sub-fan, the rest), with that many
    rays refining the third angle of a fan-started pair whose second trace
    missed."""
    ctx = ctx or default_context(prob.c.device.index)
    dev = prob.c.device
    n = prob.n_pairs
    if out is None:
        out = dict(theta=torch.empty(n, dtype=torch.float64, device=dev),
                   tof=torch.empty(n, dtype=torch.float64, device=dev),
                   hit=torch.empty((n, 2), dtype=torch.float64, device=dev),
                   status=torch.empty(n, dtype=torch.int32, device=dev),
                   iters=torch.empty(n, dtype=torch.int32, device=dev))
    if theta0 is None:
        out["theta"].fill_(float("nan"))
    else:
        out["theta"].copy_(theta0)
    ps = prob.struct(c)
    o = _opts(ds, tol, max_iter, precision, fan_rays, integrator=integrator, interpolator=interpolator, fan_ds=fan_ds,
              subfan_rays=subfan_rays)
    _L.check(ctx.h, ctx.lib.rt_link(ctx.h, C.byref(ps), C.byref(o), _ptr(out["theta"]), _ptr(out["tof"]),
                                    _ptr(out["hit"]), _ptr(out["status"]), _ptr(out["iters"]), _stream(stream)))
    return out


@dataclasses.dataclass
class Rows:
    """Recorded rows of the system matrix (rt_rows): per pair up to `cap` runs
    of 20 bytes (node index, four FP32 node weights) and the number recorded
    (-1 = none)."""
    runs: torch.Tensor               # int32 [n_pairs * cap * 5] (rt_run records)
    len: torch.Tensor                # int32 [n_pairs]
    cap: int

    @staticmethod
    def create(prob: Problem, cap: Optional[int] = None) -> "Rows":
        lib = _L.load()
        ps = prob.struct()
        cap = int(lib.rt_rows_cap(C.byref(ps))) if cap is None else int(cap)
        if cap < 1:
            raise ValueError("invalid problem for recorded rows")
        dev = prob.c.device
        return Rows(torch.empty(prob.n_pairs * cap * 5, dtype=torch.int32, device=dev),
                    torch.empty(prob.n_pairs, dtype=torch.int32, device=dev), cap)

    def struct(self) -> _L.RtRows:
        return _L.RtRows(self.runs.data_ptr(), self.len.data_ptr(), self.cap)


def rt_link_rows(prob: Problem, ds: float, rows: Rows, tol: float = 1e-4, max_iter: int = 30,
                 theta0: Optional[torch.Tensor] = None, c: Optional[torch.Tensor] = None,
                 ctx: Optional[Context] = None, stream=None, out: Optional[dict] = None,
                 fan_rays: int = DEFAULT_FAN, fan_ds: float = 0.0, subfan_rays: int = 0) -> dict:
    """rt_link (FP32-compensated, bilinear) that also records the rows of the
    linked rays into `rows` for rt_tof_adjoint_rows."""
    ctx = ctx or default_context(prob.c.device.index)
    dev = prob.c.device
    n = prob.n_pairs
    if out is None:
        out = dict(theta=torch.empty(n, dtype=torch.float64, device=dev),
                   tof=torch.empty(n, dtype=torch.float64, device=dev),
                   hit=torch.empty((n, 2), dtype=torch.float64, device=dev),
                   status=torch.empty(n, dtype=torch.int32, device=dev),
                   iters=torch.empty(n, dtype=torch.int32, device=dev))
    if theta0 is None:
        out["theta"].fill_(float("nan"))
    else:
        out["theta"].copy_(theta0)
    ps = prob.struct(c)
    o = _opts(ds, tol, max_iter, "fp32c", fan_rays, fan_ds=fan_ds, subfan_rays=subfan_rays)
    rs = rows.struct()
    _L.check(ctx.h, ctx.lib.rt_link_rows(ctx.h, C.byref(ps), C.byref(o), _ptr(out["theta"]), _ptr(out["tof"]),
                                         _ptr(out["hit"]), _ptr(out["status"]), _ptr(out["iters"]), C.byref(rs),
                                         _stream(stream)))
    return out


def rt_tof_adjoint_rows(prob: Problem, rows: Rows, theta: torch.Tensor, g_tof: torch.Tensor, ds: float,
                        tof_ref: Optional[torch.Tensor] = None, c: Optional[torch.Tensor] = None,
                        ctx: Optional[Context] = None, stream=None,
                        out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """rt_tof_adjoint from the rows recorded by rt_link_rows (same problem and
    options; theta = the linked angles)."""
    ctx = ctx or default_context(prob.c.device.index)
    cc = prob.c if c is None else c
    g = torch.empty_like(cc) if out is None else out
    ps = prob.struct(c)
    o = _opts(ds, precision="fp32c")
    rs = rows.struct()
    _L.check(ctx.h, ctx.lib.rt_tof_adjoint_rows(ctx.h, C.byref(ps), C.byref(o), C.byref(rs),
                                                _ptr(theta.contiguous()), _ptr(g_tof.contiguous()),
                                                _ptr(None if tof_ref is None else tof_ref.contiguous()), _ptr(g),
                                                _stream(stream)))
    return g


def rt_tof_forward(prob: Problem, theta: torch.Tensor, ds: float, precision: str = "fp32c",
                   c: Optional[torch.Tensor] = None, ctx: Optional[Context] = None, stream=None,
                   integrator: str = "rk4", interpolator: str = "bilinear"):
    """Travel time and interception of every pair at fixed launch angles."""
    ctx = ctx or default_context(prob.c.device.index)
    dev = prob.c.device
    tof_ = torch.empty(prob.n_pairs, dtype=torch.float64, device=dev)
    hit = torch.empty((prob.n_pairs, 2), dtype=torch.float64, device=dev)
    ps = prob.struct(c)
    o = _opts(ds, precision=precision, integrator=integrator, interpolator=interpolator)
    _L.check(ctx.h, ctx.lib.rt_tof_forward(ctx.h, C.byref(ps), C.byref(o), _ptr(theta.contiguous()), _ptr(tof_),
                                           _ptr(hit), _stream(stream)))
    return tof_, hit


def rt_tof_adjoint(prob: Problem, theta: torch.Tensor, g_tof: torch.Tensor, ds: float,
                   tof_ref: Optional[torch.Tensor] = None, precision: str = "fp32c",
                   c: Optional[torch.Tensor] = None, ctx: Optional[Context] = None, stream=None,
                   out: Optional[torch.Tensor] = None, integrator: str = "rk4",
                   interpolator: str = "bilinear") -> torch.Tensor:
    """g_c = sum_i (g_tof_i - tof_ref_i) dT_i/dc (us per m/s) with the rays
    frozen at theta: the transpose of the system matrix (paper Sec. 3.1.1)."""
    ctx = ctx or default_context(prob.c.device.index)
    cc = prob.c if c is None else c
    g = torch.empty_like(cc) if out is None else out
    ps = prob.struct(c)
    o = _opts(ds, precision=precision, integrator=integrator, interpolator=interpolator)
    _L.check(ctx.h, ctx.lib.rt_tof_adjoint(ctx.h, C.byref(ps), C.byref(o), _ptr(theta.contiguous()),
                                           _ptr(g_tof.contiguous()),
                                           _ptr(None if tof_ref is None else tof_ref.contiguous()),
                                           _ptr(g), _stream(stream)))
    return g


def rt_path_matrix(prob: Problem, theta: torch.Tensor, ds: float, precision: str = "fp32c",
                   ctx: Optional[Context] = None, stream=None, integrator: str = "rk4",
                   c: Optional[torch.Tensor] = None, interpolator: str = "bilinear"):
    """Explicit CSR system matrix (row_ptr int64, col int32, val float64) with
    T = L s, s = 1000/c; duplicate (row, col) entries sum. With the B-spline
    the columns are the slowness spline's coefficients: T = L bspline_coef(s)."""
    ctx = ctx or default_context(prob.c.device.index)
    dev = prob.c.device
    row_ptr = torch.empty(prob.n_pairs + 1, dtype=torch.int64, device=dev)
    nnz = C.c_int64(0)
    ps = prob.struct(c)
    o = _opts(ds, precision=precision, integrator=integrator, interpolator=interpolator)
    th = theta.contiguous()
    rc = ctx.lib.rt_path_matrix(ctx.h, C.byref(ps), C.byref(o), _ptr(th), _ptr(row_ptr), None, None, 0,
                                C.byref(nnz), _stream(stream))
    if rc not in (_L.RT_OK, _L.RT_ENOMEM):
        _L.check(ctx.h, rc)
    col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=dev)
    val = torch.empty(max(nnz.value, 1), dtype=torch.float64, device=dev)
    _L.check(ctx.h, ctx.lib.rt_path_matrix(ctx.h, C.byref(ps), C.byref(o), _ptr(th), _ptr(row_ptr), _ptr(col),
                                           _ptr(val), nnz.value, C.byref(nnz), _stream(stream)))
    return row_ptr, col[: nnz.value], val[: nnz.value]


def bspline_coef(f: torch.Tensor, transpose: bool = False, ctx: Optional[Context] = None, stream=None,
                 out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Control coefficients P^-1 f (P^-T f with transpose) of the interpolating
    cubic B-spline of a nodal field f [ny, nx] (float64 CUDA tensor)."""
    if f.dim() != 2 or f.dtype != torch.float64 or not f.is_cuda:
        raise ValueError("f must be a 2-D float64 CUDA tensor [ny, nx]")
    ctx = ctx or default_context(f.device.index)
    src = f.contiguous()
    a = torch.empty_like(src) if out is None else out
    _L.check(ctx.h, ctx.lib.rt_bspline_coef(ctx.h, src.shape[1], src.shape[0], _ptr(src), _ptr(a),
                                            int(bool(transpose)), _stream(stream)))
    return a


def csr_matvec(row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, x: torch.Tensor,
               ctx: Optional[Context] = None, stream=None, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """y = L x for a system matrix from rt_path_matrix (x: float64 [n_cols])."""
    ctx = ctx or default_context(x.device.index)
    n_rows = row_ptr.numel() - 1
    y = torch.empty(n_rows, dtype=torch.float64, device=x.device) if out is None else out
    _L.check(ctx.h, ctx.lib.rt_csr_matvec(ctx.h, n_rows, x.numel(), _ptr(row_ptr), _ptr(col), _ptr(val),
                                          _ptr(x.contiguous()), _ptr(y), _stream(stream)))
    return y


def csr_rmatvec(row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, w: torch.Tensor, n_cols: int,
                ctx: Optional[Context] = None, stream=None, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """y = L^T w for a system matrix from rt_path_matrix (w: float64 [n_rows])."""
    ctx = ctx or default_context(w.device.index)
    y = torch.empty(n_cols, dtype=torch.float64, device=w.device) if out is None else out
    _L.check(ctx.h, ctx.lib.rt_csr_rmatvec(ctx.h, row_ptr.numel() - 1, int(n_cols), _ptr(row_ptr), _ptr(col),
                                           _ptr(val), _ptr(w.contiguous()), _ptr(y), _stream(stream)))
    return y


def rt_status_counts(ctx: Optional[Context] = None, stream=None):
    """(all_linked, counts[8]) of the last rt_link on ctx; counts[7] = RK4 steps."""
    ctx = ctx or default_context()
    arr = (C.c_int64 * 8)()
    rc = ctx.lib.rt_status_counts(ctx.h, arr, _stream(stream))
    if rc not in (_L.RT_OK, _L.RT_ENOCONV):
        _L.check(ctx.h, rc)
    return rc == _L.RT_OK, list(arr)


class ToF(torch.autograd.Function):
    """T = ToF(c): linked travel times; backward = the adjoint scatter kernel."""

    @staticmethod
    def forward(fctx, c, prob: Problem, ds: float, tol: float, max_iter: int, precision: str, theta0,
                fan_rays: int = DEFAULT_FAN):
        r = rt_link(prob, ds, tol, max_iter, precision, theta0=theta0, c=c.detach().contiguous(),
                    fan_rays=fan_rays)
        fctx.prob, fctx.ds, fctx.precision = prob, ds, precision
        fctx.save_for_backward(c, r["theta"])
        fctx.link = r
        return r["tof"]

    @staticmethod
    def backward(fctx, g_tof):
        c, theta = fctx.saved_tensors
        g = rt_tof_adjoint(fctx.prob, theta, g_tof.contiguous(), fctx.ds, precision=fctx.precision,
                           c=c.detach().contiguous())
        return g, None, None, None, None, None, None, None


def tof(c: torch.Tensor, prob: Problem, ds: float, tol: float = 1e-4, max_iter: int = 30,
        precision: str = "fp32c", theta0: Optional[torch.Tensor] = None,
        fan_rays: int = DEFAULT_FAN) -> torch.Tensor:
    """Differentiable travel times of all pairs of ``prob`` for sound speed c."""
    return ToF.apply(c, prob, ds, tol, max_iter, precision, theta0, fan_rays)


@dataclasses.dataclass
class BatchInstance:
    """One problem of rt_batch_run with its outputs (device tensors)."""
    prob: Problem
    theta: torch.Tensor
    tof: torch.Tensor
    hit: torch.Tensor
    status: torch.Tensor
    iters: torch.Tensor
    tof_ref: Optional[torch.Tensor] = None
    g_c: Optional[torch.Tensor] = None

    @staticmethod
    def create(prob: Problem, tof_ref: Optional[torch.Tensor] = None) -> "BatchInstance":
        n, dev = prob.n_pairs, prob.c.device
        return BatchInstance(prob,
                             torch.full((n,), float("nan"), dtype=torch.float64, device=dev),
                             torch.empty(n, dtype=torch.float64, device=dev),
                             torch.empty((n, 2), dtype=torch.float64, device=dev),
                             torch.empty(n, dtype=torch.int32, device=dev),
                             torch.empty(n, dtype=torch.int32, device=dev),
                             None if tof_ref is None else tof_ref.contiguous(),
                             None if tof_ref is None else torch.empty_like(prob.c))

    def struct(self) -> _L.RtInstance:
        return _L.RtInstance(self.prob.struct(), self.theta.data_ptr(), self.tof.data_ptr(), self.hit.data_ptr(),
                             self.status.data_ptr(), self.iters.data_ptr(),
                             None if self.tof_ref is None else self.tof_ref.data_ptr(),
                             None if self.g_c is None else self.g_c.data_ptr())


def rt_batch_run(instances, ds: float, tol: float = 1e-4, max_iter: int = 30, precision: str = "fp32c",
                 fan_rays: int = DEFAULT_FAN, block_threads: int = 0, step_unroll: int = 0, fan_ds: float = 0.0,
                 blocks_per_sm: int = 0, ctx: Optional[Context] = None, stream=None,
                 reset_angles: bool = True, integrator: str = "rk4"):
    """Link (and, where tof_ref is set, adjoint-scatter) every pair of every
    instance in one persistent launch. reset_angles=True starts cold (NaN)."""
    ctx = ctx or default_context(instances[0].prob.c.device.index)
    if reset_angles:
        for b in instances:
            b.theta.fill_(float("nan"))
    arr = (_L.RtInstance * len(instances))(*[b.struct() for b in instances])
    o = _opts(ds, tol, max_iter, precision, fan_rays, block_threads, step_unroll, blocks_per_sm, integrator,
              fan_ds=fan_ds)
    _L.check(ctx.h, ctx.lib.rt_batch_run(ctx.h, len(instances), arr, C.byref(o), _stream(stream)))
    return instances


# ---------------------------------------------------------------- ray-Born

GEMM_MODES = {"fp32": _L.RTBORN_GEMM_FP32, "tf32x3": _L.RTBORN_GEMM_TF32X3}


@dataclasses.dataclass
class BornMaps:
    """Per-transducer first-arrival maps (device float32 [n_tx, ny, nx]):
    travel time T (us, +inf where no ray arrives) and amplitude A; with
    absorption also L, the path integral of alpha0 (Np (rad/s)^-y), and the
    power-law exponent y of alpha = alpha0 omega^y."""
    grid: Grid
    ring_radius: float
    T: torch.Tensor
    A: torch.Tensor
    L: Optional[torch.Tensor] = None
    y: float = 1.0

    @property
    def n_tx(self) -> int:
        return int(self.T.shape[0])

    def _grid_struct(self) -> _L.RtGrid:
        return _L.RtGrid(self.grid.nx, self.grid.ny, self.grid.h, self.grid.x0, self.grid.y0)


def rtborn_maps(prob: Problem, ds: float, fan_rays: int, c: Optional[torch.Tensor] = None,
                ctx: Optional[Context] = None, stream=None, out: Optional[BornMaps] = None,
                blocks_per_sm: int = 0, alpha0: Optional[torch.Tensor] = None, y: float = 1.0,
                interpolator: str = "bilinear", integrator: str = "rk4") -> BornMaps:
    """Travel-time and amplitude maps of every transducer from fans of
    fan_rays rays traced with their paraxial rays (paper Sec. 3.5).
    blocks_per_sm selects the fan kernel variant (0 = default). With alpha0
    (float64 CUDA [ny, nx], Np (rad/s)^-y m^-1) the maps also carry the
    absorption path integrals L and the exponent y (Appendix: alpha0 omega^y).
    interpolator "bspline" samples c, its gradient and Hessian, and s from the
    interpolating cubic B-spline (the paper's choice for ray-Born)."""
    ctx = ctx or default_context(prob.c.device.index)
    g = prob.grid
    shape = (prob.n_tx, g.ny, g.nx)
    dev = prob.c.device
    if out is None:
        out = BornMaps(g, prob.ring_radius, torch.empty(shape, dtype=torch.float32, device=dev),
                       torch.empty(shape, dtype=torch.float32, device=dev))
    if alpha0 is not None:
        alpha0 = alpha0.to(device=dev, dtype=torch.float64).contiguous()
        if alpha0.numel() != g.nx * g.ny:
            raise ValueError("alpha0 needs one value per node")
        if out.L is None:
            out.L = torch.empty(shape, dtype=torch.float32, device=dev)
        out.y = float(y)
    else:
        out.L = None
    o = _opts(ds, precision="fp32c", blocks_per_sm=blocks_per_sm, interpolator=interpolator, integrator=integrator)
    ps = prob.struct(c)
    _L.check(ctx.h, ctx.lib.rtborn_maps_abs(ctx.h, C.byref(ps), C.byref(o), int(fan_rays), _ptr(alpha0),
                                            _ptr(out.T), _ptr(out.A), _ptr(out.L), _stream(stream)))
    return out


def _freqs(f_mhz):
    f = [float(v) for v in f_mhz]
    return len(f), (C.c_double * max(len(f), 1))(*f)


def _check_maps(maps: BornMaps):
    for t in (maps.T, maps.A) + (() if maps.L is None else (maps.L,)):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("maps must be contiguous float32 CUDA tensors")
        if t.shape != (maps.n_tx, maps.grid.ny, maps.grid.nx):
            raise ValueError("maps have the wrong shape")


def rtborn_apply(maps: BornMaps, f_mhz, dc: torch.Tensor, gemm: str = "tf32x3", ctx: Optional[Context] = None,
                 stream=None, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Born data d[f, e, r] (complex64) of the perturbation dc (m/s, float32
    [ny, nx]) at frequencies f_mhz."""
    _check_maps(maps)
    ctx = ctx or default_context(maps.T.device.index)
    nf, fa = _freqs(f_mhz)
    dc = dc.to(torch.float32).contiguous()
    if dc.numel() != maps.grid.nx * maps.grid.ny or not dc.is_cuda:
        raise ValueError("dc must be a CUDA tensor with one value per node")
    if out is None:
        out = torch.empty((nf, maps.n_tx, maps.n_tx), dtype=torch.complex64, device=maps.T.device)
    g = maps._grid_struct()
    _L.check(ctx.h, ctx.lib.rtborn_apply_abs(ctx.h, C.byref(g), maps.ring_radius, maps.n_tx, _ptr(maps.T),
                                             _ptr(maps.A), _ptr(maps.L), float(maps.y), nf, fa, _ptr(dc),
                                             GEMM_MODES[gemm], _ptr(out), _stream(stream)))
    return out


def rtborn_adjoint(maps: BornMaps, f_mhz, d: torch.Tensor, gemm: str = "tf32x3", ctx: Optional[Context] = None,
                   stream=None, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Adjoint of rtborn_apply: float32 [ny, nx] from complex64 d[f, e, r]."""
    _check_maps(maps)
    ctx = ctx or default_context(maps.T.device.index)
    nf, fa = _freqs(f_mhz)
    d = d.to(torch.complex64).contiguous()
    if d.shape != (nf, maps.n_tx, maps.n_tx) or not d.is_cuda:
        raise ValueError("d must be a CUDA complex tensor [n_freq, n_tx, n_tx]")
    if out is None:
        out = torch.empty((maps.grid.ny, maps.grid.nx), dtype=torch.float32, device=maps.T.device)
    g = maps._grid_struct()
    _L.check(ctx.h, ctx.lib.rtborn_adjoint_abs(ctx.h, C.byref(g), maps.ring_radius, maps.n_tx, _ptr(maps.T),
                                               _ptr(maps.A), _ptr(maps.L), float(maps.y), nf, fa, _ptr(d),
                                               GEMM_MODES[gemm], _ptr(out), _stream(stream)))
    return out


class Born(torch.autograd.Function):
    """d = Born(dc): the linearised ray-Born map; backward = rtborn_adjoint
    (for a real input and complex output, the vector-Jacobian product is
    Re(F^H g))."""

    @staticmethod
    def forward(fctx, dc, maps: BornMaps, f_mhz, gemm: str):
        fctx.maps, fctx.f, fctx.gemm = maps, list(f_mhz), gemm
        return rtborn_apply(maps, f_mhz, dc.detach(), gemm=gemm)

    @staticmethod
    def backward(fctx, g):
        return rtborn_adjoint(fctx.maps, fctx.f, g, gemm=fctx.gemm), None, None, None


def born(dc: torch.Tensor, maps: BornMaps, f_mhz, gemm: str = "tf32x3") -> torch.Tensor:
    """Differentiable Born data of dc (float32 [ny, nx])."""
    return Born.apply(dc, maps, f_mhz, gemm)


def wait_selftest(limit_ns: int, arrive: bool, stream=None) -> tuple:
    """Runs the bounded device wait of the tensor-core kernels once on a
    barrier that completes (arrive) or never does; returns (error code, wall
    seconds): 0 when the phase completed, 199 when the wait gave up."""
    import time
    lib = _L.load()
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _L.check(None, lib.rt_wait_selftest(int(limit_ns), 1 if arrive else 0, _ptr(err), _stream(stream)))
    torch.cuda.synchronize()
    return int(err.item()), time.perf_counter() - t0
