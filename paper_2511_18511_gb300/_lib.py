"""ctypes declarations of the C ABI in include/rt.h (argument marshalling only).

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2511_18511_gb300.build``); loading fails loudly otherwise.
There is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

RT_OK, RT_EINVAL, RT_ECUDA, RT_ENOCONV, RT_ETIMEOUT, RT_ENOMEM = 0, 1, 2, 3, 4, 5
RT_FP64, RT_FP32_COMP = 0, 1
RAY_OK, RAY_MAXITER, RAY_STEPCAP, RAY_BADINPUT = 0, 1, 2, 4

# every function the header declares; the CPU tests check that each is exported
EXPORTED = [
    "rt_version", "rt_ctx_create", "rt_ctx_destroy", "rt_last_error", "rt_ctx_reserve",
    "rt_link", "rt_tof_forward", "rt_tof_adjoint", "rt_path_matrix", "rt_status_counts",
    "rt_tof_forward_noalloc", "rt_batch_run", "rtborn_maps", "rtborn_apply", "rtborn_adjoint",
    "rt_csr_matvec", "rt_csr_rmatvec", "rt_bspline_coef", "rtborn_maps_abs", "rtborn_apply_abs",
    "rtborn_adjoint_abs", "rt_peak_fma", "rt_peak_gather", "rt_peak_read", "rt_wait_selftest", "rt_rows_cap",
    "rt_link_rows", "rt_tof_adjoint_rows",
]
RTBORN_GEMM_FP32, RTBORN_GEMM_TF32X3 = 0, 1
ABI_VERSION = 4   # layout of RtOptions below


class RtGrid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("h_mm", C.c_double),
                ("x0_mm", C.c_double), ("y0_mm", C.c_double)]


class RtOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_iter", C.c_int32), ("ds_mm", C.c_double),
                ("tol_mm", C.c_double), ("fan_rays", C.c_int32), ("block_threads", C.c_int32),
                ("step_unroll", C.c_int32), ("blocks_per_sm", C.c_int32), ("integrator", C.c_int32),
                ("interpolator", C.c_int32), ("fan_ds_mm", C.c_double), ("subfan_rays", C.c_int32)]


class RtProblem(C.Structure):
    _fields_ = [("grid", RtGrid), ("c_mps", C.c_void_p), ("n_tx", C.c_int32),
                ("tx_xy_mm", C.c_void_p), ("ring_radius_mm", C.c_double), ("n_pairs", C.c_int32),
                ("pairs", C.c_void_p)]


class RtRows(C.Structure):
    _fields_ = [("runs", C.c_void_p), ("len", C.c_void_p), ("cap", C.c_int32)]


RUN_BYTES = 20   # rt_run: int32 node + 4 float weights


class RtInstance(C.Structure):
    _fields_ = [("prob", RtProblem), ("theta_io", C.c_void_p), ("tof_us", C.c_void_p),
                ("hit_xy_mm", C.c_void_p), ("status", C.c_void_p), ("iters", C.c_void_p),
                ("tof_ref", C.c_void_p), ("g_c", C.c_void_p)]


_lock = threading.Lock()
_lib = None


class RtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"raytof error {code}: {msg}")
        self.code = code


def path() -> str:
    return _build.LIB


def load():
    """Open libraytof.so (must already be built) and declare its signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library {_build.LIB} is not built; run __graft_entry__.build()")
        L = C.CDLL(_build.LIB)
        vp, P = C.c_void_p, C.POINTER
        L.rt_version.restype = C.c_int
        if L.rt_version() != ABI_VERSION:
            raise RuntimeError(f"{_build.LIB} has ABI version {L.rt_version()}, the binding expects {ABI_VERSION}; "
                               "rebuild with __graft_entry__.build()")
        L.rt_ctx_create.argtypes = [P(vp), C.c_int]
        L.rt_ctx_destroy.argtypes = [vp]
        L.rt_ctx_destroy.restype = None
        L.rt_last_error.argtypes = [vp]
        L.rt_last_error.restype = C.c_char_p
        L.rt_ctx_reserve.argtypes = [vp, C.c_int64]
        L.rt_link.argtypes = [vp, P(RtProblem), P(RtOptions), vp, vp, vp, vp, vp, vp]
        L.rt_tof_forward.argtypes = [vp, P(RtProblem), P(RtOptions), vp, vp, vp, vp]
        L.rt_rows_cap.argtypes = [P(RtProblem)]
        L.rt_rows_cap.restype = C.c_int32
        L.rt_link_rows.argtypes = [vp, P(RtProblem), P(RtOptions), vp, vp, vp, vp, vp, P(RtRows), vp]
        L.rt_tof_adjoint_rows.argtypes = [vp, P(RtProblem), P(RtOptions), P(RtRows), vp, vp, vp, vp, vp]
        L.rt_tof_adjoint.argtypes = [vp, P(RtProblem), P(RtOptions), vp, vp, vp, vp, vp]
        L.rt_path_matrix.argtypes = [vp, P(RtProblem), P(RtOptions), vp, vp, vp, vp, C.c_int64,
                                     P(C.c_int64), vp]
        L.rt_status_counts.argtypes = [vp, P(C.c_int64), vp]
        L.rt_tof_forward_noalloc.argtypes = [P(RtProblem), P(RtOptions), vp, vp, vp, vp]
        L.rt_batch_run.argtypes = [vp, C.c_int32, P(RtInstance), P(RtOptions), vp]
        L.rt_csr_matvec.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp, vp, vp, vp]
        L.rt_csr_rmatvec.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp, vp, vp, vp]
        L.rt_bspline_coef.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, C.c_int32, vp]
        L.rtborn_maps.argtypes = [vp, P(RtProblem), P(RtOptions), C.c_int32, vp, vp, vp]
        L.rtborn_apply.argtypes = [vp, P(RtGrid), C.c_double, C.c_int32, vp, vp, C.c_int32, P(C.c_double), vp,
                                   C.c_int32, vp, vp]
        L.rtborn_adjoint.argtypes = [vp, P(RtGrid), C.c_double, C.c_int32, vp, vp, C.c_int32, P(C.c_double), vp,
                                     C.c_int32, vp, vp]
        L.rtborn_maps_abs.argtypes = [vp, P(RtProblem), P(RtOptions), C.c_int32, vp, vp, vp, vp, vp]
        L.rtborn_apply_abs.argtypes = [vp, P(RtGrid), C.c_double, C.c_int32, vp, vp, vp, C.c_double, C.c_int32,
                                       P(C.c_double), vp, C.c_int32, vp, vp]
        L.rtborn_adjoint_abs.argtypes = [vp, P(RtGrid), C.c_double, C.c_int32, vp, vp, vp, C.c_double, C.c_int32,
                                         P(C.c_double), vp, C.c_int32, vp, vp]
        L.rt_peak_fma.argtypes = [C.c_int32, C.c_int32, C.c_int32, vp, vp]
        L.rt_peak_gather.argtypes = [vp, C.c_int64, C.c_int32, C.c_int32, vp, vp]
        L.rt_peak_read.argtypes = [vp, C.c_int64, C.c_int32, C.c_int32, vp, vp]
        L.rt_wait_selftest.argtypes = [C.c_int64, C.c_int32, vp, vp]
        _lib = L
        return L


def check(ctx, code):
    if code != RT_OK:
        msg = load().rt_last_error(ctx).decode() if ctx else ""
        raise RtError(code, msg)
