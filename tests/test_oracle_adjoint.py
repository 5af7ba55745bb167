"""Pins of the oracle's adjoint gradient: central finite differences of the
converged response of full oracle solves (Newton + CG, Eq. linequil2ast)
with respect to each phase's (mu, lam) and to voxel scales."""
import numpy as np
import pytest

from oracle import adjoint, materials as omat, solver
from paper_1901_06531_gb300 import inputs

TIGHT = dict(tol_newton=1e-11, tol_cg=1e-12)


def setup(n=6, scale=True):
    ph = inputs.periodic_sphere_phase((n, n, n), [(n / 2, n / 2, n / 2)], 0.3 * n)
    params = np.array([[1.0, 2.0], [10.0, 20.0]])
    sc = inputs.lognormal_scale((n, n, n), 0.3, 9) if scale else None
    return ph, params, sc


def solve_J(ph, params, sc, mask, target, wF, wP):
    m = omat.Material(ph, omat.NEOHOOKE, params, scale=sc)
    out = solver.solve(m, mask, target, **TIGHT)
    return adjoint.response(m, out["F"], wF, wP), out["F"], m


@pytest.mark.parametrize("case", ["uniaxial_stress", "mixed_strain11"])
def test_adjoint_matches_central_differences(case):
    ph, params, sc = setup()
    if case == "uniaxial_stress":
        # P11 = 0.05 with the other stresses zero and the rigid rotation fixed
        # (F12 = F13 = F23 = 0): the free response is <F>_11
        mask, target = inputs.fix_rotation(*inputs.history_uniaxial_stress_ramp(1, 0.05))
        wF = np.zeros(9); wF[0] = 1.0
        wP = np.zeros(9)
    else:
        # the paper's load case (1): F11 prescribed, F12 = F13 = F23 = 0, the
        # rest stress free; the free response is <P>_11
        mask, target = inputs.fix_rotation(*inputs.history_mixed_strain11(1, 1.03))
        wF = np.zeros(9)
        wP = np.zeros(9); wP[0] = 1.0
    J0, F, m = solve_J(ph, params, sc, mask, target, wF, wP)
    grad, dscale = adjoint.gradient(m, F, mask[0], wF, wP)
    h = 1e-5
    for p in range(2):
        for q in range(2):
            pp = params.copy(); pp[p, q] *= 1 + h
            pm = params.copy(); pm[p, q] *= 1 - h
            Jp, _, _ = solve_J(ph, pp, sc, mask, target, wF, wP)
            Jm, _, _ = solve_J(ph, pm, sc, mask, target, wF, wP)
            fd = (Jp - Jm) / (2 * h * params[p, q])
            assert abs(fd - grad[p, q]) <= 1e-6 * max(1e-3, abs(fd)), (p, q, fd, grad[p, q])
    # a few voxel scales
    rng = np.random.default_rng(3)
    for _ in range(3):
        idx = tuple(rng.integers(0, 6, 3))
        sp = sc.copy(); sp[idx] *= 1 + 1e-4
        smn = sc.copy(); smn[idx] *= 1 - 1e-4
        Jp, _, _ = solve_J(ph, params, sp, mask, target, wF, wP)
        Jm, _, _ = solve_J(ph, params, smn, mask, target, wF, wP)
        fd = (Jp - Jm) / (2e-4 * sc[idx])
        assert abs(fd - dscale[idx]) <= 1e-5 * max(1e-6, abs(fd)) + 1e-12, (idx, fd, dscale[idx])


def test_prescribed_components_have_zero_gradient():
    """<P>_IJ is prescribed on stress-controlled components and <F>_ij on
    strain-controlled ones: their derivatives must vanish."""
    ph, params, sc = setup(scale=False)
    mask, target = inputs.fix_rotation(*inputs.history_mixed_strain11(1, 1.03))
    wF = np.zeros(9); wF[0] = 1.0           # <F>_11 prescribed
    wP = np.zeros(9); wP[4] = 1.0           # <P>_22 prescribed (= 0)
    _, F, m = solve_J(ph, params, sc, mask, target, wF, wP)
    grad, dscale = adjoint.gradient(m, F, mask[0], wF, wP)
    assert np.max(np.abs(grad)) < 1e-10
    assert np.max(np.abs(dscale)) < 1e-10
