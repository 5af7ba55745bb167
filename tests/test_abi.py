"""The C ABI library builds, loads and exports every entry point declared in
include/mixfft.h; host-side argument checks run without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1901_06531_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "mixfft.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[A-Za-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 14
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_covers_the_header(lib):
    from paper_1901_06531_gb300 import mixfft
    assert sorted(mixfft.EXPORTED) == declared_symbols()


def test_create_validates_sizes_without_gpu(lib):
    lib.mf_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                              ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    lib.mf_workspace_bytes.restype = ctypes.c_size_t
    lib.mf_workspace_bytes.argtypes = [ctypes.c_void_p]
    lib.mf_destroy.argtypes = [ctypes.c_void_p]
    h = ctypes.c_void_p()
    bad = [(3, 4, 4), (4, 5, 4), (10, 4, 4), (4, 4, 1), (512, 4, 4), (4, 4, 7), (14, 8, 8),
           (256, 256, 8)]
    for nx, ny, nz in bad:
        assert lib.mf_create(ctypes.byref(h), nx, ny, nz, 0, None) == 1, (nx, ny, nz)
        assert not h.value
    assert lib.mf_create(ctypes.byref(h), 8, 8, 8, 2, None) == 1
    for nx, ny, nz, prec in [(4, 4, 2, 0), (16, 16, 16, 0), (48, 36, 18, 1), (128, 128, 128, 1),
                             (96, 96, 9, 0)]:
        assert lib.mf_create(ctypes.byref(h), nx, ny, nz, prec, None) == 0
        n = nx * ny * nz
        wsb = lib.mf_workspace_bytes(h)
        # F, P, b (FP64) + K (45) + four CG vectors + spectrum, at least
        isz = 4 if prec else 8
        assert wsb >= 27 * 8 * n + 45 * isz * n + 36 * isz * n + 72 * n
        lib.mf_destroy(h)


def test_calls_without_workspace_are_rejected(lib):
    h = ctypes.c_void_p()
    lib.mf_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                              ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    assert lib.mf_create(ctypes.byref(h), 8, 8, 8, 0, None) == 0
    lib.mf_constitutive.argtypes = [ctypes.c_void_p]
    assert lib.mf_constitutive(h) == 7
    lib.mf_set_F.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.mf_set_F(h, None) == 7
    lib.mf_bind_workspace.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
    assert lib.mf_bind_workspace(h, None, 0) == 1
    lib.mf_destroy.argtypes = [ctypes.c_void_p]
    lib.mf_destroy(h)
    lib.mf_status_string.restype = ctypes.c_char_p
    assert lib.mf_status_string(3).startswith(b"CG breakdown")


def test_option_setters_validate_without_gpu(lib):
    """Choices a context's precision or size does not support are rejected on
    the host: the outer-arithmetic projection and the persistent x-y kernel
    need an FP32-inner context, the persistent kernel a 48-128^2 plane."""
    from paper_1901_06531_gb300 import mixfft
    h = ctypes.c_void_p()
    lib.mf_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                              ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    for name in ("mf_set_projection_arith", "mf_set_xy_persistent", "mf_set_xy_split", "mf_set_outer_arith",
                 "mf_set_inexact_newton", "mf_set_predictor", "mf_set_xy_cluster"):
        getattr(lib, name).argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.mf_destroy.argtypes = [ctypes.c_void_p]
    assert lib.mf_create(ctypes.byref(h), 16, 16, 16, mixfft.MF_FP64, None) == 0
    assert lib.mf_set_projection_arith(h, mixfft.MF_PROJ_OUTER) == mixfft.MF_INVALID_ARG
    assert lib.mf_set_projection_arith(h, mixfft.MF_PROJ_FP32) == mixfft.MF_OK
    assert lib.mf_set_projection_arith(h, mixfft.MF_PROJ_AUTO) == mixfft.MF_INVALID_ARG
    assert lib.mf_set_xy_persistent(h, 1) == mixfft.MF_INVALID_ARG
    assert lib.mf_set_xy_cluster(h, 1) == mixfft.MF_INVALID_ARG
    assert lib.mf_set_inexact_newton(h, 1) == mixfft.MF_OK
    assert lib.mf_set_inexact_newton(h, 0) == mixfft.MF_OK
    assert lib.mf_set_inexact_newton(h, 2) == mixfft.MF_INVALID_ARG
    assert lib.mf_set_predictor(h, mixfft.MF_PRED_EXTRAPOLATE) == mixfft.MF_OK
    assert lib.mf_set_predictor(h, mixfft.MF_PRED_UNIFORM) == mixfft.MF_OK
    assert lib.mf_set_predictor(h, mixfft.MF_PRED_QUADRATIC) == mixfft.MF_OK
    assert lib.mf_set_predictor(h, 3) == mixfft.MF_INVALID_ARG
    lib.mf_destroy(h)
    assert lib.mf_create(ctypes.byref(h), 64, 64, 32, mixfft.MF_FP32_INNER, None) == 0
    assert lib.mf_set_projection_arith(h, mixfft.MF_PROJ_OUTER) == mixfft.MF_OK
    assert lib.mf_set_projection_arith(h, 7) == mixfft.MF_INVALID_ARG
    assert lib.mf_set_projection_arith(h, mixfft.MF_PROJ_AUTO) == mixfft.MF_OK
    assert lib.mf_set_xy_persistent(h, 1) == mixfft.MF_OK
    assert lib.mf_set_xy_persistent(h, 0) == mixfft.MF_OK
    assert lib.mf_set_xy_persistent(h, 3) == mixfft.MF_INVALID_ARG
    assert lib.mf_set_xy_cluster(h, 3) == mixfft.MF_INVALID_ARG      # cluster kernels: 128^2 planes only
    assert lib.mf_set_outer_arith(h, 5) == mixfft.MF_INVALID_ARG
    assert lib.mf_set_inexact_newton(h, 1) == mixfft.MF_OK
    assert lib.mf_set_inexact_newton(h, 0) == mixfft.MF_INVALID_ARG
    lib.mf_destroy(h)
    assert lib.mf_create(ctypes.byref(h), 32, 32, 32, mixfft.MF_FP32_INNER, None) == 0
    assert lib.mf_set_xy_persistent(h, 1) == mixfft.MF_INVALID_ARG   # no persistent kernel for 32^2 planes
    lib.mf_destroy(h)
    assert lib.mf_create(ctypes.byref(h), 128, 128, 16, mixfft.MF_FP32_INNER, None) == 0
    lib.mf_xy_schedule.argtypes = [ctypes.c_void_p] * 4
    fwd, inv = ctypes.c_int32(-1), ctypes.c_int32(-1)
    ms = (ctypes.c_float * 5)()
    assert lib.mf_xy_schedule(h, ctypes.byref(fwd), ctypes.byref(inv), ms) == mixfft.MF_OK
    assert (fwd.value, inv.value) == (0, 0) and list(ms) == [-1.0] * 5   # untuned: per plane, nothing timed
    assert lib.mf_set_xy_cluster(h, 4) == mixfft.MF_INVALID_ARG
    assert lib.mf_set_xy_cluster(h, 3) == mixfft.MF_OK
    assert lib.mf_xy_schedule(h, ctypes.byref(fwd), ctypes.byref(inv), None) == mixfft.MF_OK
    assert (fwd.value, inv.value) == (2, 2)
    lib.mf_destroy(h)


def test_binding_enums_match_the_header():
    txt = open(os.path.join(ROOT, "include", "mixfft.h")).read()
    from paper_1901_06531_gb300 import mixfft
    for name, val in re.findall(r"\b(MF_[A-Z0-9_]+)\s*=\s*(\d+)", txt):
        assert getattr(mixfft, name) == int(val), name


def test_wait_selftest_validates_its_bound_without_gpu(lib):
    lib.mf_selftest_wait_timeout.argtypes = [ctypes.c_int]
    assert lib.mf_selftest_wait_timeout(0) == 1
    assert lib.mf_selftest_wait_timeout((1 << 20) + 1) == 1


def test_release_build_has_no_trace_without_gpu(lib):
    lib.mf_trace_read.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    n = ctypes.c_int(5)
    assert lib.mf_trace_read(0, None, None, ctypes.byref(n)) == 1 and n.value == 0
    from paper_1901_06531_gb300 import mixfft
    assert mixfft.TRACE_PHASES[mixfft.MF_TRACE_CG_LOOP] == "cg_loop" and len(mixfft.TRACE_PHASES) == 18


def test_phase_composition_of_synthetic_marks():
    """bench.phase_composition: a phase lasts from the mark before it to its
    own; steps split at the step-start marks; the first steps skipped."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    names = {1: "step_start", 2: "a", 3: "b"}
    # two steps: marks at t (ns) = step 0: 0, 1000 (a), 4000 (b); step 1:
    # 5000, 7000 (a), 13000 (b)
    t = [0, 1000, 4000, 5000, 7000, 13000]
    ids = [1, 2, 3, 1, 2, 3]
    comp, totals = bench.phase_composition(t, ids, names, skip_steps=0)
    assert totals == [5.0, 8.0]
    assert comp == {"b": 4.5, "a": 1.5}
    comp1, _ = bench.phase_composition(t, ids, names, skip_steps=1)
    assert comp1 == {"b": 6.0, "a": 2.0}
