"""Helpers for the GPU parity tests: build the library, set up contexts from
the shared seeded inputs, and relative-error measures."""
import numpy as np

from paper_1901_06531_gb300 import inputs


def lib():
    from paper_1901_06531_gb300 import build
    build.build()
    from paper_1901_06531_gb300 import mixfft
    return mixfft


def rel(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def neohooke_two_phase(shape, seed, contrast=10.0):
    ph = np.random.default_rng(seed).integers(0, 2, shape).astype(np.int32)
    params = np.array([[1.0, 2.0], [contrast, 2.0 * contrast]])
    return ph, params


def polycrystal(shape, ngrains, seed):
    g, _ = inputs.voronoi(shape, ngrains, seed)
    R = inputs.random_rotations(ngrains, seed + 1)
    params = np.tile([168.0, 121.0, 75.0], (ngrains, 1))
    return g, params, R
