"""CPU-side checks of the boundary: the shared library builds for sm_103a,
loads, and exports every function include/rt.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "rt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rt[a-z_]*)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_18511_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_ray_path_calls():
    names = _declared()
    for n in ("rt_link", "rt_tof_forward", "rt_tof_adjoint", "rt_path_matrix", "rt_status_counts",
              "rt_ctx_create", "rt_ctx_destroy", "rt_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2511_18511_gb300 import _lib
    for n in _declared():
        assert hasattr(lib, n), f"{n} declared in rt.h but not exported"
    assert set(_declared()) == set(_lib.EXPORTED)


def test_version_without_gpu(lib):
    from paper_2511_18511_gb300 import _lib
    assert lib.rt_version() == _lib.ABI_VERSION == 4


def test_option_checks_without_gpu(lib):
    """The allocation-free call checks its options before touching the device:
    an unknown integrator or a non-bilinear interpolator is refused."""
    from paper_2511_18511_gb300 import _lib
    g = _lib.RtGrid(8, 8, 1.0, -3.5, -3.5)
    prob = _lib.RtProblem(g, None, 2, None, 1.0, 0, None)
    for integ, interp in ((9, 0), (0, 1), (0, 7)):
        o = _lib.RtOptions(1, 30, 0.1, 1e-4, 0, 0, 0, 0, integ, interp)
        assert lib.rt_tof_forward_noalloc(ctypes.byref(prob), ctypes.byref(o), None, None, None, None) == _lib.RT_EINVAL


def test_rows_capacity_without_gpu(lib):
    """rt_rows_cap: 1.15 x the diagonal cells of a diameter plus 16, rounded up
    to a multiple of 4 (rows on 16-byte boundaries); 0 for an invalid problem."""
    import math
    from paper_2511_18511_gb300 import _lib
    for n, h, R in ((1024, 0.2, 95.0), (128, 0.5, 30.0), (512, 0.2, 45.0), (32, 0.5, 7.0)):
        prob = _lib.RtProblem(_lib.RtGrid(n, n, h, 0.0, 0.0), None, 2, None, R, 0, None)
        cap = lib.rt_rows_cap(ctypes.byref(prob))
        raw = math.ceil(1.15 * math.sqrt(2.0) * 2.0 * R / h + 16.0)
        assert cap % 4 == 0 and raw <= cap < raw + 4, (n, cap, raw)
    assert lib.rt_rows_cap(ctypes.byref(_lib.RtProblem(_lib.RtGrid(8, 8, 1.0, 0.0, 0.0), None, 2, None, 0.0,
                                                        0, None))) == 0
    assert lib.rt_rows_cap(None) == 0


def test_wait_selftest_arguments_without_gpu(lib):
    """The bounded-wait self-test validates before it enqueues: no error word, or
    a limit outside 1 us .. 2 s, is RT_EINVAL."""
    from paper_2511_18511_gb300 import _lib
    word = ctypes.c_int32(0)
    assert lib.rt_wait_selftest(10_000_000, 0, None, None) == _lib.RT_EINVAL
    assert lib.rt_wait_selftest(10, 0, ctypes.byref(word), None) == _lib.RT_EINVAL
    assert lib.rt_wait_selftest(3_000_000_000, 0, ctypes.byref(word), None) == _lib.RT_EINVAL


def test_null_arguments_are_rejected_without_gpu(lib):
    from paper_2511_18511_gb300 import _lib
    assert lib.rt_ctx_create(None, 0) == _lib.RT_EINVAL
    assert lib.rt_link(None, None, None, None, None, None, None, None, None) == _lib.RT_EINVAL
    counts = (ctypes.c_int64 * 8)()
    assert lib.rt_status_counts(None, counts, None) == _lib.RT_EINVAL


def test_library_built_for_sm103a_only():
    from paper_2511_18511_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_noalloc_object_references_no_allocator(lib):
    """The allocation-free entry point's object file calls no CUDA allocator
    (its undefined symbols, read with nm, name no cudaMalloc* or cudaFree*)."""
    import shutil
    import subprocess
    from paper_2511_18511_gb300 import build
    nm = shutil.which("nm")
    if not nm:
        pytest.skip("nm not available")
    obj = os.path.join(build.OUT, "rt_noalloc.o")
    assert os.path.exists(obj)
    out = subprocess.run([nm, "-u", "-C", obj], capture_output=True, text=True, check=True).stdout
    bad = [ln for ln in out.splitlines() if re.search(r"\bcuda(Malloc|Free)\w*|\bcuMem(Alloc|Free)\w*", ln)]
    assert not bad, bad
