"""FP64 CPU oracle for two-point ray tracing and ray-Born: ctypes wrapper
around oracle.c and born.c.

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it; the library never does. It shares no code
with the CUDA path. The C sources are compiled on first use (gcc, OpenMP,
``-ffp-contract=off`` so that x86 and Arm hosts round identically).

Every function takes plain numpy arrays in the library's units: lengths in mm,
sound speed in m/s, times in us.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "born.c")]
_HDR = os.path.join(_HERE, "oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

RAY_OK, RAY_MAXITER, RAY_STEPCAP, RAY_BADINPUT = 0, 1, 2, 4


def compile_to(out_path: str, sources=None) -> str:
    """gcc-compile the oracle sources (default: oracle.c and born.c) into a shared library."""
    sources = list(sources or _SRC)
    tmp = out_path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-I", _HERE, "-o", tmp] + sources + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out_path)
    return out_path


def build(force: bool = False) -> str:
    """Compile liboracle.so if missing or stale; returns its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + [_HDR])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    return compile_to(_LIB_PATH)


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("h", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)


def load(path: str):
    """Open an oracle shared library and declare its C signatures."""
    L = C.CDLL(path)
    G = C.POINTER(_Grid)
    L.orc_field.argtypes = [G, _dp, _dp, _dp, _dp, _dp]
    L.orc_sample.argtypes = [G, _dp, C.c_int32, _dp, _dp]
    L.orc_march.argtypes = [G, _dp, C.c_double, C.c_double, C.c_double, C.c_double,
                            C.c_int32, _dp]
    L.orc_trace.argtypes = [G, _dp, C.c_double, C.c_double, C.c_double, C.c_double,
                            C.c_double, C.c_double, C.c_double, C.c_int64, _dp, _dp,
                            _lp, _dp, _ip]
    L.orc_link.argtypes = [G, _dp, C.c_int32, _dp, C.c_double, C.c_int32, _ip,
                           C.c_double, C.c_double, C.c_int32, C.c_int32, C.c_double, C.c_int32, _dp, _dp, _dp, _ip,
                           _ip, C.c_int32]
    L.orc_subfan_angles.argtypes = [C.c_double, C.c_double, C.c_int32, _dp]
    L.orc_subfan_predict.argtypes = [C.c_int32, _dp, _dp, _ip, C.c_double, C.c_double, _dp]
    L.orc_tof.argtypes = [G, _dp, C.c_int32, _dp, C.c_double, C.c_int32, _ip, C.c_double,
                          _dp, _dp, _dp, C.c_int32]
    L.orc_path_matrix.argtypes = [G, _dp, C.c_int32, _dp, C.c_double, C.c_int32, _ip,
                                  C.c_double, _dp, _lp, _ip, _dp, C.c_int64, C.c_int32]
    L.orc_path_matrix.restype = C.c_int64
    L.orc_adjoint.argtypes = [G, _dp, C.c_int32, _dp, C.c_double, C.c_int32, _ip,
                              C.c_double, _dp, _dp, _dp, C.c_int32]
    L.orc_num_threads.argtypes = []
    L.orc_set_integrator.argtypes = [C.c_int32]
    L.orc_set_link_rule.argtypes = [C.c_int32]
    L.orc_r13_angle.argtypes = [_dp, _dp, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32,
                                C.c_double, C.c_double, _dp]
    L.orc_set_interpolator.argtypes = [C.c_int32]
    L.orc_bspline_coef.argtypes = [G, _dp, _dp, C.c_int32]
    L.orc_fan_angles.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32, _dp, _dp]
    L.orc_fan_ray.argtypes = [G, _dp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                              C.c_int64, _dp, _lp]
    L.orc_fan_maps.argtypes = [G, _dp, C.c_int32, _dp, C.c_double, C.c_double, C.c_int32, C.c_double,
                               _dp, _dp, C.c_int32]
    L.orc_born_apply.argtypes = [G, C.c_double, C.c_int32, _dp, _dp, C.c_int32, _dp, _dp, C.c_int32,
                                 _ip, _dp, C.c_int32]
    L.orc_born_adjoint.argtypes = [G, C.c_double, C.c_int32, _dp, _dp, C.c_int32, _dp, _dp, _dp,
                                   C.c_int32]
    L.orc_fan_maps_abs.argtypes = [G, _dp, _dp, C.c_int32, _dp, C.c_double, C.c_double, C.c_int32, C.c_double,
                                   _dp, _dp, _dp, C.c_int32]
    L.orc_born_apply_abs.argtypes = [G, C.c_double, C.c_int32, _dp, _dp, _dp, C.c_double, C.c_int32, _dp, _dp,
                                     C.c_int32, _ip, _dp, C.c_int32]
    L.orc_born_adjoint_abs.argtypes = [G, C.c_double, C.c_int32, _dp, _dp, _dp, C.c_double, C.c_int32, _dp, _dp,
                                       _dp, C.c_int32]
    return L


_current = None


def lib():
    """The library the functions below call (the built oracle unless overridden)."""
    global _lib
    with _lock:
        if _current is not None:
            return _current
        if _lib is None:
            _lib = load(build())
    return _lib


class using:
    """Context manager: route the functions below to another oracle library
    (used by the mutation tests, which compile deliberately broken copies)."""

    def __init__(self, L):
        self.L = L

    def __enter__(self):
        global _current
        self.prev, _current = _current, self.L
        return self.L

    def __exit__(self, *exc):
        global _current
        _current = self.prev


def _grid(grid) -> _Grid:
    return _Grid(int(grid.nx), int(grid.ny), float(grid.h), float(grid.x0), float(grid.y0))


def _d(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _i(a):
    return None if a is None else a.ctypes.data_as(_ip)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def num_threads() -> int:
    return int(lib().orc_num_threads())


INTEGRATORS = {"rk4": 0, "heun": 1}


class integrator:
    """Context manager: trace with another integrator ("rk4" default, "heun")."""

    def __init__(self, name: str):
        self.k = INTEGRATORS[name]

    def __enter__(self):
        _check(lib().orc_set_integrator(self.k), "set_integrator")
        return self

    def __exit__(self, *exc):
        lib().orc_set_integrator(0)


LINK_RULES = {"r8": 0, "r13": 1}


class link_rule:
    """Context manager: link fan-started pairs with another rule ("r8" default,
    "r13": the fan model corrected through the traces for the second and third
    angles)."""

    def __init__(self, name: str):
        self.k = LINK_RULES[name]

    def __enter__(self):
        _check(lib().orc_set_link_rule(self.k), "set_link_rule")
        return self

    def __exit__(self, *exc):
        lib().orc_set_link_rule(0)


INTERPOLATORS = {"bilinear": 0, "bspline": 1}


class interpolator:
    """Context manager: sample the field with another interpolator ("bilinear"
    default, "bspline": cubic B-spline with analytic gradient)."""

    def __init__(self, name: str):
        self.k = INTERPOLATORS[name]

    def __enter__(self):
        _check(lib().orc_set_interpolator(self.k), "set_interpolator")
        return self

    def __exit__(self, *exc):
        lib().orc_set_interpolator(0)


def field(grid, c_mps):
    """Nodal (c, dc/dx, dc/dy, s) in mm/us units, each [ny, nx]."""
    c = _f64(c_mps)
    outs = [np.empty_like(c) for _ in range(4)]
    g = _grid(grid)
    _check(lib().orc_field(C.byref(g), _d(c), *[_d(o) for o in outs]), "field")
    return tuple(outs)


def bspline_coef(grid, f, transpose=False):
    """Control coefficients P^-1 f of the interpolating cubic B-spline of the
    nodal field f[ny, nx] (P^-T f with transpose)."""
    f = _f64(f)
    out = np.empty_like(f)
    g = _grid(grid)
    _check(lib().orc_bspline_coef(C.byref(g), _d(f), _d(out), int(bool(transpose))), "bspline_coef")
    return out


def sample(grid, c_mps, xy):
    """(c, dc/dx, dc/dy, s) at points xy[n, 2] -> [n, 4] by the current interpolator."""
    c = _f64(c_mps)
    xy = _f64(xy).reshape(-1, 2)
    out = np.empty((xy.shape[0], 4))
    g = _grid(grid)
    _check(lib().orc_sample(C.byref(g), _d(c), xy.shape[0], _d(xy), _d(out)), "sample")
    return out


def march(grid, c_mps, x, y, theta, ds, n_steps):
    """Positions of n_steps fixed RK4 steps -> [n_steps+1, 2]."""
    c = _f64(c_mps)
    out = np.empty((n_steps + 1, 2))
    g = _grid(grid)
    _check(lib().orc_march(C.byref(g), _d(c), x, y, theta, ds, n_steps, _d(out)), "march")
    return out


def trace(grid, c_mps, R, xe, xr, theta, ds, record=True):
    """One trace; returns dict(T, hit, dir, dsp, flags, pts, alpha)."""
    c = _f64(c_mps)
    cap = int(np.ceil(8.0 * R / ds)) + 2 if record else 0
    pts = np.empty((max(cap, 1), 2))
    alpha = np.empty(max(cap, 1))
    n = C.c_int64(0)
    out6 = np.empty(6)
    flags = C.c_int32(0)
    g = _grid(grid)
    rc = lib().orc_trace(C.byref(g), _d(c), R, xe[0], xe[1], xr[0], xr[1], theta, ds, cap,
                         _d(pts) if record else None, _d(alpha) if record else None,
                         C.byref(n), _d(out6), C.byref(flags))
    _check(rc, "trace")
    res = dict(T=out6[0], hit=out6[1:3].copy(), dir=out6[3:5].copy(), dsp=out6[5],
               flags=int(flags.value), n_pts=int(n.value))
    if record:
        res["pts"] = pts[: n.value].copy()
        res["alpha"] = alpha[: n.value].copy()
    return res


def _pairs_arg(pairs, n_tx):
    if pairs is None:
        return None, n_tx * (n_tx - 1)
    p = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    return p, p.shape[0]


def link(grid, c_mps, tx, R, ds, tol=1e-4, max_iter=30, pairs=None, theta0=None, nthreads=0, fan_rays=0,
         fan_ds=0.0, subfan=0):
    """Link all pairs; returns dict(theta, tof, hit, status, iters). fan_rays = 0:
    straight-line cold start; >= 2: fan-predicted cold start, the fan's rays
    traced at step fan_ds (0 = ds); subfan > 0: a fan-started pair whose second
    trace misses is refined by subfan rays inside its bracket (reading R12)."""
    c = _f64(c_mps)
    tx = _f64(tx).reshape(-1, 2)
    p, n_pairs = _pairs_arg(pairs, tx.shape[0])
    theta = np.full(n_pairs, np.nan) if theta0 is None else _f64(theta0).copy()
    tof = np.empty(n_pairs)
    hit = np.empty((n_pairs, 2))
    status = np.empty(n_pairs, np.int32)
    iters = np.empty(n_pairs, np.int32)
    g = _grid(grid)
    rc = lib().orc_link(C.byref(g), _d(c), tx.shape[0], _d(tx), R, n_pairs, _i(p), ds, tol,
                        max_iter, fan_rays, float(fan_ds), int(subfan), _d(theta), _d(tof), _d(hit), _i(status),
                        _i(iters), nthreads)
    _check(rc, "link")
    return dict(theta=theta, tof=tof, hit=hit, status=status, iters=iters)


def r13_angle(t, m, x1, m1, lo, hi, x2=None, m2=None):
    """R13: the root in (lo, hi) of the fan rays' interpolating polynomial
    moved onto the trace (x1, m1), or onto both traces when (x2, m2) is given
    (NaN when the moved polynomial does not change sign there)."""
    t, m = _f64(t), _f64(m)
    out = np.empty(1)
    two = x2 is not None
    _check(lib().orc_r13_angle(_d(t), _d(m), t.size, float(x1), float(m1), float(x2) if two else 0.0,
                               float(m2) if two else 0.0, int(two), float(lo), float(hi), _d(out)), "r13_angle")
    return float(out[0])


def subfan_angles(ta, tb, M):
    """R12: the M sub-fan ray angles strictly inside the bracket (ta, tb)."""
    out = np.empty(int(M))
    _check(lib().orc_subfan_angles(float(ta), float(tb), int(M), _d(out)), "subfan_angles")
    return out


def subfan_predict(theta, m, pos, c3, R=1.0):
    """R12 prediction from the sequence (bracket end of negative misfit at
    place 0, the sub-fan rays that reached the ring at their index q, the other
    end at M + 1) around c3, the plain rule's third angle, for ring radius R ->
    dict(theta3, ta, tb, start_theta, start_m, changes_sign, refined)."""
    t, mm = _f64(theta).ravel(), _f64(m).ravel()
    it = np.ascontiguousarray(pos, dtype=np.int32).ravel()
    out = np.empty(7)
    _check(lib().orc_subfan_predict(len(t), _d(t), _d(mm), _i(it), float(c3), float(R), _d(out)), "subfan_predict")
    return dict(theta3=out[0], ta=out[1], tb=out[2], start_theta=out[3], start_m=out[4], changes_sign=bool(out[5]),
                refined=bool(out[6]))


def tof(grid, c_mps, tx, R, ds, theta, pairs=None, nthreads=0):
    """Travel time and hit of every pair at fixed angles -> (tof, hit)."""
    c = _f64(c_mps)
    tx = _f64(tx).reshape(-1, 2)
    p, n_pairs = _pairs_arg(pairs, tx.shape[0])
    th = _f64(theta)
    out = np.empty(n_pairs)
    hit = np.empty((n_pairs, 2))
    g = _grid(grid)
    rc = lib().orc_tof(C.byref(g), _d(c), tx.shape[0], _d(tx), R, n_pairs, _i(p), ds, _d(th),
                       _d(out), _d(hit), nthreads)
    _check(rc, "tof")
    return out, hit


def path_matrix(grid, c_mps, tx, R, ds, theta, pairs=None, nthreads=0):
    """Explicit CSR system matrix -> (row_ptr, col, val) with T = L s."""
    c = _f64(c_mps)
    tx = _f64(tx).reshape(-1, 2)
    p, n_pairs = _pairs_arg(pairs, tx.shape[0])
    th = _f64(theta)
    row_ptr = np.empty(n_pairs + 1, np.int64)
    g = _grid(grid)
    L = lib()
    nnz = L.orc_path_matrix(C.byref(g), _d(c), tx.shape[0], _d(tx), R, n_pairs, _i(p), ds,
                            _d(th), row_ptr.ctypes.data_as(_lp), None, None, 0, nthreads)
    if nnz < 0:
        raise ValueError("oracle path_matrix failed")
    col = np.empty(max(nnz, 1), np.int32)
    val = np.empty(max(nnz, 1))
    nnz2 = L.orc_path_matrix(C.byref(g), _d(c), tx.shape[0], _d(tx), R, n_pairs, _i(p), ds,
                             _d(th), row_ptr.ctypes.data_as(_lp), _i(col), _d(val), nnz, nthreads)
    if nnz2 != nnz:
        raise ValueError("oracle path_matrix changed size between passes")
    return row_ptr, col[:nnz], val[:nnz]


def adjoint(grid, c_mps, tx, R, ds, theta, g_tof, pairs=None, nthreads=0):
    """d(sum g_tof*T)/dc per node in us/(m/s), rays frozen at theta -> [ny, nx]."""
    c = _f64(c_mps)
    tx = _f64(tx).reshape(-1, 2)
    p, n_pairs = _pairs_arg(pairs, tx.shape[0])
    th = _f64(theta)
    gt = _f64(g_tof)
    out = np.empty_like(c)
    g = _grid(grid)
    rc = lib().orc_adjoint(C.byref(g), _d(c), tx.shape[0], _d(tx), R, n_pairs, _i(p), ds,
                           _d(th), _d(gt), _d(out), nthreads)
    _check(rc, "adjoint")
    return out


# ---- ray-Born (born.c) ------------------------------------------------------

def fan_angles(xe, R, ds, K):
    """(a_min, step) of the fan of transducer xe: theta_k = a_min + k * step."""
    a, st = C.c_double(0), C.c_double(0)
    _check(lib().orc_fan_angles(float(xe[0]), float(xe[1]), R, ds, K, C.byref(a), C.byref(st)), "fan_angles")
    return a.value, st.value


def fan_ray(grid, c_mps, R, xe, theta, ds):
    """One fan ray with its paraxial ray -> dict of per-sample arrays
    x, y, dx, dy, T, Q, P, c, s (sample points strictly inside the ring)."""
    c = _f64(c_mps)
    cap = int(np.ceil(8.0 * R / ds)) + 2
    rec = np.empty((cap, 9))
    n = C.c_int64(0)
    g = _grid(grid)
    _check(lib().orc_fan_ray(C.byref(g), _d(c), R, float(xe[0]), float(xe[1]), theta, ds, cap, _d(rec),
                             C.byref(n)), "fan_ray")
    rec = rec[: min(n.value, cap)]
    return {k: rec[:, q].copy() for q, k in enumerate(("x", "y", "dx", "dy", "T", "Q", "P", "c", "s"))}


ETA = 1e-2   # us: penalty of the squared distance (in cells) to the ray in the amplitude choice


def fan_maps(grid, c_mps, tx, R, ds, K, eta=ETA, nthreads=0, alpha0=None):
    """First-arrival maps (T us, A) of every transducer -> two [n_tx, ny, nx]
    arrays (T = inf, A = 0 where no fan ray reaches); A from the candidate of
    least T + eta (b/h)^2, b its distance to the ray. With alpha0 [ny, nx]
    (Np (rad/s)^-y m^-1) also the absorption path integrals Lam -> (T, A, Lam)."""
    c = _f64(c_mps)
    tx = _f64(tx).reshape(-1, 2)
    n_tx = tx.shape[0]
    T = np.empty((n_tx, grid.ny, grid.nx))
    A = np.empty((n_tx, grid.ny, grid.nx))
    g = _grid(grid)
    if alpha0 is None:
        _check(lib().orc_fan_maps(C.byref(g), _d(c), n_tx, _d(tx), R, ds, K, eta, _d(T), _d(A), nthreads),
               "fan_maps")
        return T, A
    al = _f64(alpha0)
    Lam = np.empty((n_tx, grid.ny, grid.nx))
    _check(lib().orc_fan_maps_abs(C.byref(g), _d(c), _d(al), n_tx, _d(tx), R, ds, K, eta, _d(T), _d(A), _d(Lam),
                                  nthreads), "fan_maps_abs")
    return T, A, Lam


def born_apply(grid, R, T, A, f_mhz, dc, pairs=None, nthreads=0, Lam=None, y=1.0):
    """Born data, complex: [n_freq, n_tx, n_tx] (pairs None) or [n_freq, n_pairs];
    with Lam the absorption factor exp(-omega_s^y Lam) multiplies each map."""
    T, A = _f64(T), _f64(A)
    Lam = None if Lam is None else _f64(Lam)
    n_tx = T.shape[0]
    f = _f64(f_mhz).ravel()
    dc = _f64(dc)
    p = None if pairs is None else np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    n_out = n_tx * n_tx if p is None else p.shape[0]
    out = np.empty((len(f), n_out, 2))
    g = _grid(grid)
    _check(lib().orc_born_apply_abs(C.byref(g), R, n_tx, _d(T), _d(A), _d(Lam), float(y), len(f), _d(f), _d(dc),
                                    0 if p is None else p.shape[0], _i(p), _d(out), nthreads), "born_apply")
    d = out[..., 0] + 1j * out[..., 1]
    return d.reshape(len(f), n_tx, n_tx) if p is None else d


def born_adjoint(grid, R, T, A, f_mhz, d, nthreads=0, Lam=None, y=1.0):
    """Adjoint of born_apply for complex d [n_freq, n_tx, n_tx] -> [ny, nx]."""
    T, A = _f64(T), _f64(A)
    Lam = None if Lam is None else _f64(Lam)
    n_tx = T.shape[0]
    f = _f64(f_mhz).ravel()
    dd = np.ascontiguousarray(np.stack([np.real(d), np.imag(d)], axis=-1), dtype=np.float64)
    out = np.empty((grid.ny, grid.nx))
    g = _grid(grid)
    _check(lib().orc_born_adjoint_abs(C.byref(g), R, n_tx, _d(T), _d(A), _d(Lam), float(y), len(f), _d(f), _d(dd),
                                      _d(out), nthreads), "born_adjoint")
    return out
