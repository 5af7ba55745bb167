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
