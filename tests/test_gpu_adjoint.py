"""GPU parity of the adjoint sensitivity (mf_adjoint and the autograd
wrapper) against the oracle's adjoint gradient, central finite differences
of full GPU solves, and the invariants it must satisfy (zero derivative of a
prescribed quantity, additivity over load steps)."""
import numpy as np
import pytest

from oracle import adjoint as oadj, materials as omat, solver as osolver
from paper_1901_06531_gb300 import inputs

from gpu_util import lib, rel

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_newton=1e-11, tol_cg=1e-12, max_cg=20000)
PARAMS = np.array([[1.0, 2.0], [10.0, 20.0]])


def two_phase(shape, scale_seed=9):
    nz, ny, nx = shape
    ph = inputs.periodic_sphere_phase(shape, [(nx / 2, ny / 2, nz / 2)], 0.3 * min(shape))
    sc = None if scale_seed is None else inputs.lognormal_scale(shape, 0.3, scale_seed)
    return ph, sc


def uniaxial():
    """P11 = 0.05, other stresses zero, rotation fixed by F12 = F13 = F23 = 0;
    free response <F>_11."""
    mask, target = inputs.fix_rotation(*inputs.history_uniaxial_stress_ramp(1, 0.05))
    wF = np.zeros(9); wF[0] = 1.0
    return mask, target, wF, np.zeros(9)


def mixed():
    """The paper's load case (1): F11 = 1.03, rotation fixed, the rest stress
    free; free response <P>_11 + 0.5 <F>_22."""
    mask, target = inputs.fix_rotation(*inputs.history_mixed_strain11(1, 1.03))
    wP = np.zeros(9); wP[0] = 1.0
    wF = np.zeros(9); wF[4] = 0.5
    return mask, target, wF, wP


def oracle_gradient(ph, sc, mask, target, wF, wP):
    m = omat.Material(ph, omat.NEOHOOKE, PARAMS, scale=sc)
    out = osolver.solve(m, mask, target, tol_newton=1e-11, tol_cg=1e-12)
    grad, dscale = oadj.gradient(m, out["F"], mask[-1], wF, wP)
    return oadj.response(m, out["F"], wF, wP), grad, dscale


def gpu_gradient(mf, shape, precision, ph, sc, mask, target, wF, wP, solve_kw, adj_kw):
    import torch
    nz, ny, nx = shape
    ctx = mf.Context(nx, ny, nz, precision)
    ctx.set_material(mf.MF_NEOHOOKE, PARAMS, ph, scale=sc)
    ctx.solve(mask, target, **solve_kw)
    ds = torch.zeros(ctx.N, dtype=torch.float64, device=ctx.device)
    J, grad, its = ctx.adjoint(mask[-1], wF, wP, dscale=ds, **adj_kw)
    return J, grad, ds.cpu().numpy().reshape(shape), its


@pytest.mark.parametrize("shape", [(16, 16, 16), (6, 8, 12)])
@pytest.mark.parametrize("case", [uniaxial, mixed])
def test_adjoint_fp64_matches_oracle(shape, case):
    """FP64: J, dJ/d(mu, lam) per phase and dJ/ds_v agree with the oracle to
    1e-8 relative (both sides converged to Newton 1e-11 / CG 1e-12; the
    adjoint CG to 1e-12)."""
    mf = lib()
    ph, sc = two_phase(shape)
    mask, target, wF, wP = case()
    J0, g0, d0 = oracle_gradient(ph, sc, mask, target, wF, wP)
    J, g, d, its = gpu_gradient(mf, shape, mf.MF_FP64, ph, sc, mask, target, wF, wP, TIGHT,
                                dict(tol_cg=1e-12, cg_rel=0.0, max_cg=20000))
    assert its > 0
    assert abs(J - J0) <= 1e-10 * max(1.0, abs(J0))
    assert rel(g, g0) < 1e-8, (g, g0)
    assert rel(d, d0) < 1e-8


@pytest.mark.parametrize("case", [uniaxial, mixed])
def test_adjoint_fp32_inner_matches_oracle(case):
    """FP32 inner solves (the state itself is converged in FP64 by defect
    correction): the adjoint solve runs in FP32 to cg_rel 1e-5, so the
    gradient carries the FP32 solve's relative error, stated as 1e-4."""
    mf = lib()
    shape = (16, 16, 16)
    ph, sc = two_phase(shape)
    mask, target, wF, wP = case()
    J0, g0, d0 = oracle_gradient(ph, sc, mask, target, wF, wP)
    J, g, d, its = gpu_gradient(mf, shape, mf.MF_FP32_INNER, ph, sc, mask, target, wF, wP,
                                dict(tol_newton=1e-10, tol_cg=1e-12, cg_rel=1e-4, max_cg=20000),
                                dict(tol_cg=1e-30, cg_rel=1e-5, max_cg=20000))
    assert abs(J - J0) <= 1e-8 * max(1.0, abs(J0))
    assert rel(g, g0) < 1e-4, (g, g0)
    assert rel(d, d0) < 1e-4


def test_prescribed_quantities_have_zero_gradient():
    """<F>_11 is prescribed and <P>_22 = 0 is prescribed under load case (1):
    their derivatives vanish identically."""
    mf = lib()
    shape = (16, 16, 16)
    ph, sc = two_phase(shape)
    mask, target = inputs.fix_rotation(*inputs.history_mixed_strain11(1, 1.03))
    wF = np.zeros(9); wF[0] = 1.0
    wP = np.zeros(9); wP[4] = 1.0
    J, g, d, _ = gpu_gradient(mf, shape, mf.MF_FP64, ph, sc, mask, target, wF, wP, TIGHT,
                              dict(tol_cg=1e-12, cg_rel=0.0, max_cg=20000))
    assert np.max(np.abs(g)) < 1e-9
    assert np.max(np.abs(d)) < 1e-11


def test_autograd_matches_central_differences():
    """torch.autograd through the load history (two steps, checkpointed F):
    the gradient of a weighted sum of free responses equals central finite
    differences of full GPU solves, for every (mu, lam) and three voxel
    scales."""
    import torch
    mf = lib()
    from paper_1901_06531_gb300.adjoint import homogenized_response
    shape = (16, 16, 16)
    nz, ny, nx = shape
    ph, sc = two_phase(shape)
    mask, target = inputs.fix_rotation(*inputs.history_uniaxial_stress_ramp(2, 0.05))
    wts = torch.tensor(np.random.default_rng(5).normal(size=(2, 9)))
    ctx = mf.Context(nx, ny, nz, mf.MF_FP64)
    kw = dict(tol_newton=1e-11, tol_cg=1e-12, max_cg=20000)

    def J_of(p, s):
        r = homogenized_response(ctx, ph, p, mask, target, scale=s, **kw)
        return float((r * wts).sum())

    p = torch.tensor(PARAMS, requires_grad=True)
    s = torch.tensor(sc, requires_grad=True)
    r = homogenized_response(ctx, ph, p, mask, target, scale=s, **kw)
    (r * wts).sum().backward()
    h = 1e-5
    for a in range(2):
        for b in range(2):
            pp = PARAMS.copy(); pp[a, b] *= 1 + h
            pm = PARAMS.copy(); pm[a, b] *= 1 - h
            fd = (J_of(torch.tensor(pp), torch.tensor(sc)) - J_of(torch.tensor(pm), torch.tensor(sc))) / (
                2 * h * PARAMS[a, b])
            assert abs(fd - float(p.grad[a, b])) <= 1e-6 * max(1e-3, abs(fd)), (a, b, fd, p.grad[a, b])
    rng = np.random.default_rng(3)
    for _ in range(3):
        idx = tuple(int(i) for i in rng.integers(0, 16, 3))
        sp = sc.copy(); sp[idx] *= 1 + 1e-4
        smn = sc.copy(); smn[idx] *= 1 - 1e-4
        fd = (J_of(torch.tensor(PARAMS), torch.tensor(sp)) - J_of(torch.tensor(PARAMS), torch.tensor(smn))) / (
            2e-4 * sc[idx])
        g = float(s.grad[idx])
        assert abs(fd - g) <= 1e-5 * max(1e-6, abs(fd)) + 1e-12, (idx, fd, g)


def test_autograd_history_matches_oracle_per_step():
    """A three-step ramp: the autograd gradient of the summed free responses
    equals the sum over steps of the oracle's adjoint gradient at each step's
    converged state (hyperelastic: steps couple only through the start
    value)."""
    import torch
    mf = lib()
    from paper_1901_06531_gb300.adjoint import homogenized_response
    shape = (8, 8, 8)
    ph, sc = two_phase(shape)
    mask, target = inputs.fix_rotation(*inputs.history_uniaxial_stress_ramp(3, 0.06))
    ctx = mf.Context(8, 8, 8, mf.MF_FP64)
    p = torch.tensor(PARAMS, requires_grad=True)
    r = homogenized_response(ctx, ph, p, mask, target, scale=None, **TIGHT)
    r[:, 0].sum().backward()
    m = omat.Material(ph, omat.NEOHOOKE, PARAMS)
    tot = np.zeros((2, 2))
    wF = np.zeros(9); wF[0] = 1.0
    for k in range(3):
        out = osolver.solve(m, mask[:k + 1], target[:k + 1], tol_newton=1e-11, tol_cg=1e-12)
        g, _ = oadj.gradient(m, out["F"], mask[k], wF, np.zeros(9))
        tot += g
    assert rel(p.grad.numpy(), tot) < 1e-8


def test_adjoint_rejects_unsupported():
    mf = lib()
    ph, _ = two_phase((8, 8, 8), None)
    ctx = mf.Context(8, 8, 8, mf.MF_FP64)
    ctx.set_material(mf.MF_SVK_CUBIC, np.tile([168.0, 121.0, 75.0], (2, 1)), ph)
    with pytest.raises(mf.MixFFTError) as e:
        ctx.adjoint(np.ones(9, np.uint8), np.ones(9), np.zeros(9))
    assert e.value.status == mf.MF_INVALID_ARG
    ctx.set_material(mf.MF_NEOHOOKE, PARAMS, ph)
    bad = np.ones(9, np.uint8); bad[3] = 2
    with pytest.raises(mf.MixFFTError) as e:
        ctx.adjoint(bad, np.ones(9), np.zeros(9))
    assert e.value.status == mf.MF_INVALID_ARG
    with pytest.raises(mf.MixFFTError) as e:
        ctx.adjoint(np.ones(9, np.uint8), np.full(9, np.nan), np.zeros(9))
    assert e.value.status == mf.MF_INVALID_ARG


@pytest.mark.slow
def test_adjoint_full_size_directional_derivative():
    """128^3, two phases, lognormal (sigma 0.3) voxel scale, P11 = 0.05 with
    the rotation fixed (the full-size adjoint workload).  No oracle solve fits
    here; the property checked is the directional derivative: for a random
    scale direction e, (J(s + h e) - J(s - h e)) / 2h equals dJ/ds . e, and
    the same for (mu, lam) of each phase, FP32 inner solves."""
    import torch
    mf = lib()
    n = 128
    shape = (n, n, n)
    ph = inputs.periodic_sphere_phase(shape, [(n / 2, n / 2, n / 2)], 0.3 * n)
    sc = inputs.lognormal_scale(shape, 0.3, 11)
    mask, target, wF, wP = uniaxial()
    ctx = mf.Context(n, n, n, mf.MF_FP32_INNER)
    kw = dict(tol_newton=1e-10, tol_cg=1e-12, cg_rel=1e-4, max_cg=20000)

    def J_of(params, s):
        ctx.set_material(mf.MF_NEOHOOKE, params, ph, scale=s)
        out = ctx.solve(mask, target, **kw)
        return float(np.dot(wF, out["Fbar"][-1]) + np.dot(wP, out["Pbar"][-1]))

    J0 = J_of(PARAMS, sc)
    ds = torch.zeros(ctx.N, dtype=torch.float64, device=ctx.device)
    J, g, its = ctx.adjoint(mask[-1], wF, wP, tol_cg=1e-30, cg_rel=1e-6, max_cg=20000, dscale=ds)
    assert abs(J - J0) < 1e-12 * max(1.0, abs(J0))
    e = np.random.default_rng(2).normal(size=shape) * sc
    h = 1e-3
    fd = (J_of(PARAMS, sc + h * e) - J_of(PARAMS, sc - h * e)) / (2 * h)
    ad = float(np.sum(ds.cpu().numpy().reshape(shape) * e))
    assert abs(fd - ad) <= 2e-3 * abs(fd), (fd, ad)
    for a in range(2):
        for b in range(2):
            pp = PARAMS.copy(); pp[a, b] *= 1 + h
            pm = PARAMS.copy(); pm[a, b] *= 1 - h
            fd = (J_of(pp, sc) - J_of(pm, sc)) / (2 * h * PARAMS[a, b])
            assert abs(fd - g[a, b]) <= 2e-3 * max(abs(fd), 1e-3 * np.max(np.abs(g))), (a, b, fd, g[a, b])


@pytest.mark.slow
def test_adjoint_256_directional_derivative():
    """256^3 (split x-y kernels), two phases, lognormal (sigma 0.3) voxel
    scale, P11 = 0.05 with the rotation fixed, FP32 inner: the adjoint's
    dJ/ds . e against the central difference of two full solves along a
    random scale direction e, and dJ/dmu of the inclusion phase likewise."""
    import torch
    mf = lib()
    n = 256
    shape = (n, n, n)
    ph = inputs.periodic_sphere_phase(shape, [(n / 2, n / 2, n / 2)], 0.3 * n)
    sc = inputs.lognormal_scale(shape, 0.3, 12)
    mask, target, wF, wP = uniaxial()
    ctx = mf.Context(n, n, n, mf.MF_FP32_INNER)
    kw = dict(tol_newton=1e-10, tol_cg=1e-12, cg_rel=1e-4, max_cg=20000)

    def J_of(params, s):
        ctx.set_material(mf.MF_NEOHOOKE, params, ph, scale=s)
        out = ctx.solve(mask, target, **kw)
        return float(np.dot(wF, out["Fbar"][-1]) + np.dot(wP, out["Pbar"][-1]))

    J0 = J_of(PARAMS, sc)
    ds = torch.zeros(ctx.N, dtype=torch.float64, device=ctx.device)
    J, g, its = ctx.adjoint(mask[-1], wF, wP, tol_cg=1e-30, cg_rel=1e-6, max_cg=20000, dscale=ds)
    assert abs(J - J0) < 1e-12 * max(1.0, abs(J0))
    e = np.random.default_rng(4).normal(size=shape) * sc
    h = 1e-3
    fd = (J_of(PARAMS, sc + h * e) - J_of(PARAMS, sc - h * e)) / (2 * h)
    ad = float(np.sum(ds.cpu().numpy().reshape(shape) * e))
    assert abs(fd - ad) <= 2e-3 * abs(fd), (fd, ad)
    pp = PARAMS.copy(); pp[1, 0] *= 1 + h
    pm = PARAMS.copy(); pm[1, 0] *= 1 - h
    fd = (J_of(pp, sc) - J_of(pm, sc)) / (2 * h * PARAMS[1, 0])
    assert abs(fd - g[1, 0]) <= 2e-3 * abs(fd), (fd, g[1, 0])
