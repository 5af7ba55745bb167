"""Pins of the oracle's projection operator G-hat-star (Eq. eq:G, eq:Gnew,
eq:Gnewnew): algebra of a projection, major symmetry, compatibility of its
output, the null-frequency control rule, and agreement with the Green
operator of a reference medium (Sec. 2.1, last sentence)."""
import numpy as np
import pytest

from oracle import dft, projector

SHAPES = [(3, 3, 3), (4, 4, 4), (5, 5, 5), (6, 6, 6), (4, 6, 8), (5, 4, 3)]
MASKS = {
    "strain": np.zeros(9, np.uint8),
    "stress": np.ones(9, np.uint8),
    "case1": np.array([0, 0, 0, 1, 1, 0, 1, 1, 1], np.uint8),
    "random": np.array([1, 0, 1, 1, 0, 0, 1, 0, 1], np.uint8),
}


def dot(a, b):
    return float(np.sum(a * b))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mname", list(MASKS))
def test_idempotent_and_self_adjoint(shape, mname):
    m = MASKS[mname]
    rng = np.random.default_rng(10)
    x = rng.standard_normal((9,) + shape)
    y = rng.standard_normal((9,) + shape)
    gx = projector.apply(x, m)
    gy = projector.apply(y, m)
    np.testing.assert_allclose(projector.apply(gx, m), gx, atol=1e-13)
    assert abs(dot(gx, y) - dot(x, gy)) < 1e-12 * np.sqrt(dot(x, x) * dot(y, y))


@pytest.mark.parametrize("shape", SHAPES)
def test_output_is_real(shape):
    rng = np.random.default_rng(11)
    x = rng.standard_normal((9,) + shape)
    full = dft.inverse(projector.apply_hat(dft.forward(x), MASKS["stress"]))
    assert np.max(np.abs(full.imag)) < 1e-14 * np.max(np.abs(full.real))


def test_major_symmetry_per_frequency():
    shape = (5, 6, 7)
    rng = np.random.default_rng(12)
    xi, null, nyq = projector.frequency_grid(shape)
    for _ in range(20):
        z, y, x = (rng.integers(0, s) for s in shape)
        if null[z, y, x]:
            continue
        G = np.zeros((9, 9))
        for d in range(9):
            e = np.zeros((9,) + shape, dtype=complex)
            e[d, z, y, x] = 1.0
            G[:, d] = projector.apply_hat(e, MASKS["stress"])[:, z, y, x].real
        np.testing.assert_allclose(G, G.T, atol=1e-15)
        v = np.array([xi[0][z, y, x], xi[1][z, y, x], xi[2][z, y, x]])
        expect = np.einsum("ik,jl->ijkl", np.eye(3), np.outer(v, v) / v.dot(v)).reshape(9, 9)
        if nyq[z, y, x]:
            expect[:] = 0
        np.testing.assert_allclose(G, expect, atol=1e-15)


@pytest.mark.parametrize("shape", [(4, 6, 8), (6, 6, 6)])
def test_nyquist_and_null_frequencies(shape):
    rng = np.random.default_rng(13)
    ahat = rng.standard_normal((9,) + shape) + 1j * rng.standard_normal((9,) + shape)
    _, null, nyq = projector.frequency_grid(shape)
    for mname, m in MASKS.items():
        out = projector.apply_hat(ahat, m)
        assert np.all(out[:, nyq] == 0)
        np.testing.assert_allclose(out[:, 0, 0, 0], m * ahat[:, 0, 0, 0], atol=0)
    # Nyquist planes: x index n/2, y index n/2, z index n/2 and their
    # intersections are all zero
    nz, ny, nx = shape
    assert nyq[:, :, nx // 2].all() and nyq[:, ny // 2, :].all() and nyq[nz // 2].all()
    assert nyq.sum() == nx * ny * nz - (nx - 1) * (ny - 1) * (nz - 1)


@pytest.mark.parametrize("shape", SHAPES)
def test_mean_is_masked_average(shape):
    rng = np.random.default_rng(14)
    x = rng.standard_normal((9,) + shape)
    for m in MASKS.values():
        gx = projector.apply(x, m)
        np.testing.assert_allclose(gx.reshape(9, -1).mean(1), m * x.reshape(9, -1).mean(1),
                                   atol=1e-14)


@pytest.mark.parametrize("shape", SHAPES)
def test_output_is_curl_free_gradient(shape):
    """Away from the null frequency every output coefficient is q (x) xi
    (Eq. comp): rows of the 3x3 coefficient are parallel to xi."""
    rng = np.random.default_rng(15)
    x = rng.standard_normal((9,) + shape)
    ghat = dft.forward(projector.apply(x, MASKS["random"])).reshape((3, 3) + shape)
    xi, null, _ = projector.frequency_grid(shape)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                res = ghat[i, j] * xi[k] - ghat[i, k] * xi[j]
                assert np.max(np.abs(res)) < 1e-14


@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 6, 3), (6, 8, 4)])
def test_gradient_fields_pass_and_incompatible_fields_vanish(shape):
    """A discrete gradient field (u-hat (x) xi, no Nyquist content, zero mean)
    is reproduced exactly; a field a (x) b with b orthogonal to xi is removed."""
    rng = np.random.default_rng(16)
    xi, null, nyq = projector.frequency_grid(shape)
    u = rng.standard_normal((3,) + shape)
    uhat = dft.forward(u)
    uhat[:, nyq] = 0
    uhat[:, null] = 0
    F = np.zeros((3, 3) + shape, dtype=complex)
    for i in range(3):
        for j in range(3):
            F[i, j] = 1j * uhat[i] * xi[j]
    f = np.real(dft.inverse(F.reshape((9,) + shape)))
    np.testing.assert_allclose(projector.apply(f, MASKS["strain"]), f, atol=1e-13)
    # incompatible: rows orthogonal to xi
    a = rng.standard_normal((3,) + shape)
    bvec = np.stack([xi[1] - xi[2], xi[2] - xi[0], xi[0] - xi[1]])  # b . xi = 0
    Ghat = np.einsum("i...,j...->ij...", dft.forward(a), bvec).reshape((9,) + shape)
    out = projector.apply_hat(Ghat, MASKS["strain"])
    assert np.max(np.abs(out)) < 1e-14 * max(1.0, np.max(np.abs(Ghat)))


def green_operator_reference_medium(shape, lam, mu):
    """Finite-strain Green operator of a homogeneous reference medium with
    stiffness C0 = lam I(x)I + 2 mu II (II_ijkl = d_ik d_jl): with the acoustic
    tensor N_ik = C0_ijkl xi_j xi_l, Gamma_ijkl = (N^-1)_ik xi_j xi_l."""
    xi, null, nyq = projector.frequency_grid(shape)
    d = np.eye(3)
    C0 = lam * np.einsum("ij,kl->ijkl", d, d) + 2 * mu * np.einsum("ik,jl->ijkl", d, d)
    G = np.zeros((3, 3, 3, 3) + shape)
    for idx in np.ndindex(*shape):
        if null[idx] or nyq[idx]:
            continue
        v = np.array([xi[0][idx], xi[1][idx], xi[2][idx]])
        N = np.einsum("ijkl,j,l->ik", C0, v, v)
        Ninv = np.linalg.inv(N)
        G[(slice(None),) * 4 + idx] = np.einsum("ik,j,l->ijkl", Ninv, v, v)
    return G


def test_equals_reference_medium_green_operator():
    """Sec. 2.1: G-hat is the Green operator of an isotropic reference medium
    with lam = 0, mu = 1/2 (read here with the non-symmetrised stiffness
    lam I(x)I + 2 mu II of the finite-strain Lippmann-Schwinger equation)."""
    shape = (4, 5, 6)
    Gam = green_operator_reference_medium(shape, 0.0, 0.5)
    rng = np.random.default_rng(17)
    ahat = rng.standard_normal((9,) + shape) + 1j * rng.standard_normal((9,) + shape)
    ref = np.einsum("ijkl...,kl...->ij...", Gam, ahat.reshape((3, 3) + shape)).reshape((9,) + shape)
    ref[:, 0, 0, 0] = 0
    ours = projector.apply_hat(ahat, MASKS["strain"])
    np.testing.assert_allclose(ours, ref, atol=1e-14)
    # a different reference medium is a different operator
    Gam2 = green_operator_reference_medium(shape, 1.0, 0.5)
    ref2 = np.einsum("ijkl...,kl...->ij...", Gam2, ahat.reshape((3, 3) + shape)).reshape((9,) + shape)
    ref2[:, 0, 0, 0] = 0
    assert np.max(np.abs(ours - ref2)) > 1e-3
