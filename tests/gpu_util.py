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


EPS32 = 2.0 ** -24


def fp32_operator_error(got, ref, c=2.0):
    """Element-wise check of an FP32 projected-operator result y = G*(K:x)
    against the FP64 oracle (same FP32-rounded x):
        max |y - y_ref| <= c * log2(N) * eps32 * max |y_ref|,   c = 2,
    N the voxel count.  Each of the log2(N) radix-2 levels of the forward and
    inverse transforms adds rounding of relative size eps32 to every
    coefficient, and the FP32 tangent apply adds a few eps32 per element; a
    plain FP32 pipeline (FP32 FFTs of the same operator) stays at 0.2-0.3 of
    c = 1 on these cells, so c = 2 leaves room for the radix-8/16 stages and
    the FP32 matrix-free tangent while still catching any wrong coefficient
    (a misplaced frequency or Nyquist plane shows up at O(1) of max |y|).
    Returns the measured c."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    n_vox = ref[0].size
    scale = np.log2(n_vox) * EPS32 * float(np.max(np.abs(ref)))
    measured = float(np.max(np.abs(got - ref))) / scale
    assert np.all(np.isfinite(got))
    assert measured <= c, f"FP32 operator error {measured:.3f} x log2(N) eps32 max|ref| (bound {c})"
    return measured
