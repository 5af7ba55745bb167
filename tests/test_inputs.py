"""The seeded input generators: shapes, fractions and the load cases of the
paper's Sec. 3 (control cases (1)-(4))."""
import numpy as np
import pytest

from paper_1901_06531_gb300 import inputs

EYE = np.array([1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0])


@pytest.mark.parametrize("n", [16, 32, 64])
def test_particle_rve_fraction_and_count(n):
    ph = inputs.particle_rve(n, 1001)
    assert ph.shape == (n, n, n) and set(np.unique(ph)) == {0, 1}
    assert abs(ph.mean() - 0.2) < 0.01
    # four separate particles: count the connected components (periodic)
    import scipy.ndimage as ndi
    lab, k = ndi.label(np.tile(ph, (2, 2, 2)))
    assert k >= 4


def test_case1_is_the_rotation_fixed_mixed_control():
    m, t = inputs.history_case1(5, 0.2)
    np.testing.assert_array_equal(m[0], [0, 0, 0, 1, 1, 0, 1, 1, 1])
    np.testing.assert_allclose(t[:, 0], 1.0 + 0.2 * np.arange(1, 6) / 5)
    assert np.all(t[:, [1, 2, 3, 4, 5, 6, 7, 8]] == 0.0)


def test_cases_2_and_3_ramp_to_the_endpoint():
    P_end = np.arange(9.0)
    m, t = inputs.history_case2(P_end, 4)
    assert m.all() and np.allclose(t[-1], P_end) and np.allclose(t[0], P_end / 4)
    F_end = EYE + 0.01 * np.arange(9.0)
    m, t = inputs.history_case3(F_end, 4)
    assert not m.any() and np.allclose(t[-1], F_end) and np.allclose(t[1], EYE + (F_end - EYE) / 2)


def test_case4_pseudo_uniaxial_is_isochoric_at_the_end():
    m, t = inputs.history_case4(20, 0.02)
    assert not m.any()
    F = t[-1].reshape(3, 3)
    assert abs(np.linalg.det(F) - 1.0) < 1e-15
    assert F[0, 0] == 1.02 and F[1, 1] == F[2, 2] and np.all(F - np.diag(np.diag(F)) == 0)


def test_random_control_leaves_no_rotation_plane_free():
    rng = np.random.default_rng(3)
    for _ in range(200):
        m, t = inputs.random_control(3, rng)
        assert (m[0] == 0).any()
        for up, lo in ((1, 3), (2, 6), (5, 7)):
            assert not (m[0, up] and m[0, lo])
        assert np.all(t[:, m[0] == 1] == 0.0)
