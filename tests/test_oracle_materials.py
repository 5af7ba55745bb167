"""Pins of the oracle's constitutive laws: P = dW/dF and K = dP/dF
(Eq. eq:lineariz) by central finite differences, the small-strain limit at
F = I, objectivity, and the symmetries of the rotated cubic stiffness."""
import numpy as np
import pytest

from oracle import materials as mat
from paper_1901_06531_gb300 import inputs

SHAPE = (2, 2, 3)


def laws():
    rng = np.random.default_rng(20)
    ph = rng.integers(0, 2, SHAPE).astype(np.int32)
    nh = mat.Material(ph, mat.NEOHOOKE, [[1.0, 2.0], [10.0, 20.0]])
    R = inputs.random_rotations(2, 21)
    svk = mat.Material(ph, mat.SVK_CUBIC, [[168.0, 121.0, 75.0], [100.0, 60.0, 30.0]], R)
    sc = inputs.lognormal_scale(SHAPE, 0.3, 22)
    nhs = mat.Material(ph, mat.NEOHOOKE, [[1.0, 2.0], [10.0, 20.0]], scale=sc)
    return {"neohooke": nh, "svk": svk, "neohooke_scaled": nhs}


def fields():
    small = inputs.random_F(SHAPE, 23, amp=0.05)
    large = inputs.random_F(SHAPE, 24, amp=0.3)
    stretch = np.zeros((9,) + SHAPE)
    stretch[0], stretch[4], stretch[8] = 1.3, 0.9, 0.95
    stretch[1] = 0.1
    return {"small": small, "large": large, "stretch": stretch}


@pytest.mark.parametrize("law", ["neohooke", "svk", "neohooke_scaled"])
@pytest.mark.parametrize("fname", ["small", "large", "stretch"])
def test_P_is_energy_derivative(law, fname):
    m = laws()[law]
    F = fields()[fname]
    P, _ = m.PK(F)
    h = 1e-6
    for c in range(9):
        Fp = F.copy(); Fp[c] += h
        Fm = F.copy(); Fm[c] -= h
        dW = (m.energy(Fp) - m.energy(Fm)) / (2 * h)
        np.testing.assert_allclose(P[c], dW, rtol=1e-7, atol=1e-8 * np.max(np.abs(P)) + 1e-9)


@pytest.mark.parametrize("law", ["neohooke", "svk", "neohooke_scaled"])
@pytest.mark.parametrize("fname", ["small", "large", "stretch"])
def test_K_is_stress_derivative(law, fname):
    m = laws()[law]
    F = fields()[fname]
    _, K = m.PK(F)
    h = 1e-6
    scale = np.max(np.abs(K))
    for d in range(9):
        Fp = F.copy(); Fp[d] += h
        Fm = F.copy(); Fm[d] -= h
        dP = (m.PK(Fp)[0] - m.PK(Fm)[0]) / (2 * h)
        assert np.max(np.abs(K[:, d] - dP)) <= 1e-7 * scale
    # major symmetry of a hyperelastic tangent
    np.testing.assert_allclose(K, np.swapaxes(K, 0, 1), atol=1e-12 * scale)


def test_small_strain_limit_neohooke():
    lam, mu = 2.0, 1.0
    m = mat.Material(np.zeros(SHAPE, np.int32), mat.NEOHOOKE, [[mu, lam]])
    F = np.zeros((9,) + SHAPE); F[0] = F[4] = F[8] = 1.0
    P, K = m.PK(F)
    assert np.max(np.abs(P)) < 1e-15
    d = np.eye(3)
    C = (lam * np.einsum("ij,kl->ijkl", d, d)
         + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d))).reshape(9, 9)
    np.testing.assert_allclose(K[:, :, 0, 0, 0], C, atol=1e-15)


def test_svk_tangent_at_identity_is_stiffness_in_voigt_form():
    m = mat.Material(np.zeros(SHAPE, np.int32), mat.SVK_CUBIC, [[168.0, 121.0, 75.0]])
    F = np.zeros((9,) + SHAPE); F[0] = F[4] = F[8] = 1.0
    _, K = m.PK(F)
    K0 = K[:, :, 0, 0, 0].reshape(3, 3, 3, 3)
    assert K0[0, 0, 0, 0] == 168.0 and K0[1, 1, 1, 1] == 168.0 and K0[2, 2, 2, 2] == 168.0
    assert K0[0, 0, 1, 1] == 121.0 and K0[1, 1, 2, 2] == 121.0
    assert K0[0, 1, 0, 1] == 75.0 and K0[1, 2, 1, 2] == 75.0 and K0[0, 1, 1, 0] == 75.0
    assert K0[0, 0, 0, 1] == 0.0


def test_cubic_stiffness_rotation_symmetries():
    C = mat.cubic_stiffness(168.0, 121.0, 75.0)
    # 90 degree rotation about z maps the cubic crystal onto itself
    Rz = np.array([[0.0, -1, 0], [1, 0, 0], [0, 0, 1]])
    np.testing.assert_allclose(mat.rotate_stiffness(C, Rz), C, atol=1e-12)
    # an isotropic tensor is invariant under any rotation
    Ciso = mat.isotropic_stiffness(2.0, 1.0)
    R = inputs.random_rotations(1, 25)[0]
    np.testing.assert_allclose(mat.rotate_stiffness(Ciso, R), Ciso, atol=1e-13)
    # a generic rotation changes the cubic tensor but keeps its symmetries
    Cr = mat.rotate_stiffness(C, R)
    assert np.max(np.abs(Cr - C)) > 1.0
    np.testing.assert_allclose(Cr, Cr.transpose(1, 0, 2, 3), atol=1e-12)
    np.testing.assert_allclose(Cr, Cr.transpose(2, 3, 0, 1), atol=1e-12)
    # 45 degrees about z: C'11 = (C11 + C12)/2 + C44
    c, s = np.cos(np.pi / 4), np.sin(np.pi / 4)
    R45 = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
    C45 = mat.rotate_stiffness(C, R45)
    assert abs(C45[0, 0, 0, 0] - ((168.0 + 121.0) / 2 + 75.0)) < 1e-12


@pytest.mark.parametrize("law", ["neohooke", "svk"])
def test_objectivity(law):
    m = laws()[law]
    F = fields()["large"]
    Q = inputs.random_rotations(1, 26)[0]
    QF = np.einsum("ik,kj...->ij...", Q, F.reshape((3, 3) + SHAPE)).reshape((9,) + SHAPE)
    P, _ = m.PK(F)
    PQ, _ = m.PK(QF)
    QP = np.einsum("ik,kj...->ij...", Q, P.reshape((3, 3) + SHAPE)).reshape((9,) + SHAPE)
    np.testing.assert_allclose(PQ, QP, atol=1e-12 * np.max(np.abs(P)))


def test_random_rotations_are_proper_orthogonal():
    R = inputs.random_rotations(50, 27)
    np.testing.assert_allclose(np.einsum("nij,nkj->nik", R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-14)


def test_neohooke_rejects_inverted_voxel():
    m = mat.Material(np.zeros(SHAPE, np.int32), mat.NEOHOOKE, [[1.0, 2.0]])
    F = np.zeros((9,) + SHAPE); F[0] = F[4] = F[8] = 1.0
    F[8, 0, 0, 0] = -0.5
    with pytest.raises(FloatingPointError):
        m.PK(F)
