"""GPU parity of converged load histories against the oracle (Sec. 2.3 mixed
control, Eq. linequil2ast), the control exactness at every step, the FP32
inner / FP64 outer mode, and the failure statuses."""
import numpy as np
import pytest

from oracle import materials as omat, solver as osolver
from paper_1901_06531_gb300 import inputs

from gpu_util import lib, polycrystal, rel

pytestmark = pytest.mark.gpu

CASE1 = np.array([0, 0, 0, 1, 1, 0, 1, 1, 1], np.uint8)


def sphere_cell(mf, n, precision, r_frac=0.25):
    ph = inputs.centred_sphere(n, r_frac)
    params = np.array([[1.0, 2.0], [10.0, 20.0]])
    ctx = mf.Context(n, n, n, precision)
    ctx.set_material(mf.MF_NEOHOOKE, params, ph)
    return ctx, omat.Material(ph, omat.NEOHOOKE, params)


def invariants(F, P):
    """F^T F and F^T P per voxel: unchanged by a rigid rotation F -> QF, P -> QP.
    Under control patterns that leave a rotation of the cell free (a null mode
    of the linearised problem) only these are unique."""
    Fm = F.reshape((3, 3) + F.shape[1:])
    Pm = P.reshape((3, 3) + P.shape[1:])
    C = np.einsum("ki...,kj...->ij...", Fm, Fm)
    Sg = np.einsum("ki...,kj...->ij...", Fm, Pm)
    return C, Sg


def check_control(out, mask, target, tol_p, tol_f):
    for k in range(mask.shape[0]):
        s = mask[k] == 1
        if s.any():
            assert np.max(np.abs(out["Pbar"][k][s] - target[k][s])) < tol_p
        if (~s).any():
            assert np.max(np.abs(out["Fbar"][k][~s] - target[k][~s])) < tol_f


def test_uniaxial_stress_ramp_16_fp64():
    """16^3 sphere, all nine components stress controlled, P11 -> 0.1 in 5
    steps, Newton tol 1e-8, CG tol 1e-10."""
    mf = lib()
    ctx, om = sphere_cell(mf, 16, mf.MF_FP64)
    mask, target = inputs.history_uniaxial_stress_ramp(5, 0.1)
    out = ctx.solve(mask, target, 1e-8, 1e-10)
    ref = osolver.solve(om, mask, target, 1e-8, 1e-10)
    assert rel(out["Fbar"], ref["Fbar"]) < 1e-10
    assert np.max(np.abs(out["Pbar"] - ref["Pbar"])) < 1e-10
    F, P = ctx.get_fields()
    # all nine components stress controlled with P-bar = diag(p, 0, 0): the
    # rotation about e1 is a null mode (zero curvature, the residual blind to
    # it), so F is unique up to it; F^T F and F^T P are unique and agree with
    # the oracle to the FP64 gate 1e-10 (stress-like field over its largest
    # stiffness, mu = 10)
    C, S = invariants(F, P)
    Cr, Sr = invariants(ref["F"], ref["P"])
    errs = (rel(C, Cr), np.max(np.abs(S - Sr)) / 10.0)
    assert max(errs) < 1e-10, errs
    np.testing.assert_array_equal(out["newton"], ref["newton"])
    assert np.all(np.abs(out["cg"] - ref["cg"]) <= 2 * out["newton"])
    # at these tolerances the control error is at the level of the last CG residual
    check_control(out, mask, target, 1e-10, 1e-14)


@pytest.mark.parametrize("shape", [(8, 8, 8), (12, 8, 6)])
def test_mixed_control_tight_fp64(shape):
    """Converged FP64 solve at Newton tol 1e-10 / CG tol 1e-12: fields agree
    with the oracle to 1e-10 relative."""
    mf = lib()
    nx, ny, nz = shape
    ph = inputs.periodic_sphere_phase((nz, ny, nx), [(nx / 2, ny / 2, nz / 2)], 0.3 * nz)
    params = np.array([[1.0, 2.0], [10.0, 20.0]])
    ctx = mf.Context(nx, ny, nz, mf.MF_FP64)
    ctx.set_material(mf.MF_NEOHOOKE, params, ph)
    om = omat.Material(ph, omat.NEOHOOKE, params)
    mask, target = inputs.history_mixed_strain11(3, 1.05)
    out = ctx.solve(mask, target, 1e-10, 1e-12)
    ref = osolver.solve(om, mask, target, 1e-10, 1e-12)
    F, P = ctx.get_fields()
    assert rel(F, ref["F"]) < 1e-10
    assert rel(P, ref["P"]) < 1e-10
    assert rel(out["Pbar"], ref["Pbar"]) < 1e-10
    check_control(out, mask, target, 1e-12, 1e-14)


def test_polycrystal_cyclic_fp64():
    """SVK cubic polycrystal, cyclic stress with the rigid rotation fixed by
    F12 = F13 = F23 = 0 (the paper's case (1) pattern)."""
    mf = lib()
    n = 16
    g, params, R = polycrystal((n, n, n), 12, 31)
    ctx = mf.Context(n, n, n, mf.MF_FP64)
    ctx.set_material(mf.MF_SVK_CUBIC, params, g, rot=R)
    om = omat.Material(g, omat.SVK_CUBIC, params, R)
    mask, target = inputs.fix_rotation(*inputs.history_cyclic_stress(8, 0.2))
    out = ctx.solve(mask, target, 1e-8, 1e-10)
    ref = osolver.solve(om, mask, target, 1e-8, 1e-10)
    assert rel(out["Fbar"], ref["Fbar"]) < 1e-10
    assert np.max(np.abs(out["Pbar"] - ref["Pbar"])) < 1e-10
    check_control(out, mask, target, 1e-10, 1e-14)


def test_fp32_inner_matches_fp64_oracle():
    """FP32 inner CG with FP64 residual and Newton update: converged averages
    and fields against the FP64 oracle at the same Newton tolerance."""
    mf = lib()
    ctx, om = sphere_cell(mf, 16, mf.MF_FP32_INNER)
    mask, target = inputs.history_uniaxial_stress_ramp(5, 0.1)
    out = ctx.solve(mask, target, 1e-8, 1e-10, cg_rel=1e-4)
    ref = osolver.solve(om, mask, target, 1e-10, 1e-12)
    F, P = ctx.get_fields()
    assert rel(out["Fbar"], ref["Fbar"]) < 1e-9
    assert np.max(np.abs(out["Pbar"] - ref["Pbar"])) < 1e-9
    # full stress control leaves the rotation about the load axis free: F is
    # unique up to that rotation, F^T F and F^T P are unique.  Each FP32
    # correction is projected once more onto range(G*) before the update, so
    # the only components the FP64 residual cannot see are the rounding of
    # that projection; the stated FP32-inner field tolerance is 1e-8
    # (max-norm; stress-like fields times the largest stiffness, mu = 10;
    # measured 4.9e-9 and 7.7e-9).
    C, S = invariants(F, P)
    Cr, Sr = invariants(ref["F"], ref["P"])
    errs = (rel(C, Cr), np.max(np.abs(S - Sr)) / 10.0)
    assert max(errs) < 1e-8, errs
    check_control(out, mask, target, 1e-9, 1e-14)


@pytest.mark.parametrize("outer", ["double_word", "fp64"])
def test_fp32_inner_projection_in_outer_arithmetic(outer):
    """MF_PROJ_OUTER: each FP32 correction widened to FP64 and projected in
    the outer arithmetic (double-word transforms, or FP64 ones): the fields
    agree with the FP64 oracle to 1e-9 (measured about 1e-10), the averages
    to 1e-9 as in the default mode."""
    mf = lib()
    ctx, om = sphere_cell(mf, 16, mf.MF_FP32_INNER)
    if outer == "fp64":
        ctx.set_outer_arith(mf.MF_OUTER_FP64)
    ctx.set_projection_arith(mf.MF_PROJ_OUTER)
    mask, target = inputs.history_uniaxial_stress_ramp(5, 0.1)
    out = ctx.solve(mask, target, 1e-8, 1e-10, cg_rel=1e-4)
    ref = osolver.solve(om, mask, target, 1e-10, 1e-12)
    F, P = ctx.get_fields()
    assert rel(out["Fbar"], ref["Fbar"]) < 1e-9
    assert np.max(np.abs(out["Pbar"] - ref["Pbar"])) < 1e-9
    C, S = invariants(F, P)
    Cr, Sr = invariants(ref["F"], ref["P"])
    errs = (rel(C, Cr), np.max(np.abs(S - Sr)) / 10.0)
    assert max(errs) < 1e-9, errs
    check_control(out, mask, target, 1e-9, 1e-14)


def test_outer_arith_switch_between_solves():
    """A context whose outer arithmetic changes between solves gives what a
    context created with the new setting gives, bit for bit (its captured
    load histories hold the outer level's kernels and are rebuilt)."""
    mf = lib()
    n = 16
    g, params, R = polycrystal((n, n, n), 12, 41)
    mask, target = inputs.fix_rotation(*inputs.history_cyclic_stress(4, 0.2))

    def run(ctx, arith):
        ctx.set_outer_arith(arith)
        ctx.set_F(None)
        return ctx.solve(mask, target, 1e-8, 1e-10, cg_rel=1e-4)

    ctx = mf.Context(n, n, n, mf.MF_FP32_INNER)
    ctx.set_material(mf.MF_SVK_CUBIC, params, g, rot=R)
    for arith in (mf.MF_OUTER_DOUBLE_WORD, mf.MF_OUTER_FP64, mf.MF_OUTER_DOUBLE_WORD):
        o = run(ctx, arith)
        fresh = mf.Context(n, n, n, mf.MF_FP32_INNER)
        fresh.set_material(mf.MF_SVK_CUBIC, params, g, rot=R)
        ref = run(fresh, arith)
        np.testing.assert_array_equal(o["Fbar"], ref["Fbar"])
        np.testing.assert_array_equal(o["cg"], ref["cg"])


def test_projection_arith_is_validated():
    mf = lib()
    with pytest.raises(mf.MixFFTError):
        mf.Context(8, 8, 8, mf.MF_FP64).set_projection_arith(mf.MF_PROJ_OUTER)
    with pytest.raises(mf.MixFFTError):
        mf.Context(8, 8, 8, mf.MF_FP32_INNER).set_projection_arith(7)


def test_fp32_inner_polycrystal():
    mf = lib()
    n = 16
    g, params, R = polycrystal((n, n, n), 12, 41)
    ctx = mf.Context(n, n, n, mf.MF_FP32_INNER)
    ctx.set_material(mf.MF_SVK_CUBIC, params, g, rot=R)
    om = omat.Material(g, omat.SVK_CUBIC, params, R)
    mask, target = inputs.fix_rotation(*inputs.history_cyclic_stress(4, 0.2))
    out = ctx.solve(mask, target, 1e-8, 1e-10, cg_rel=1e-4)
    ref = osolver.solve(om, mask, target, 1e-10, 1e-12)
    F, _ = ctx.get_fields()
    assert rel(out["Fbar"], ref["Fbar"]) < 1e-9
    assert rel(F, ref["F"]) < 1e-8, rel(F, ref["F"])   # measured 4.4e-10


@pytest.mark.parametrize("forcing", [0, 1])
def test_fp64_inexact_newton_forcing(forcing):
    """mf_set_inexact_newton: the FP64 path with the FP32-inner forcing
    sequence reaches the oracle's converged state to the same 1e-10 as the
    absolute CG stop, in fewer CG iterations."""
    mf = lib()
    n = 16
    g, params, R = polycrystal((n, n, n), 12, 31)
    om = omat.Material(g, omat.SVK_CUBIC, params, R)
    mask, target = inputs.fix_rotation(*inputs.history_cyclic_stress(4, 0.2))
    ref = osolver.solve(om, mask, target, 1e-10, 1e-12)
    ctx = mf.Context(n, n, n, mf.MF_FP64)
    ctx.set_material(mf.MF_SVK_CUBIC, params, g, rot=R)
    ctx.set_inexact_newton(forcing)
    out = ctx.solve(mask, target, 1e-8, 1e-10, cg_rel=1e-4)
    F, P = ctx.get_fields()
    assert rel(out["Fbar"], ref["Fbar"]) < 1e-10
    assert np.max(np.abs(out["Pbar"] - ref["Pbar"])) / 168.0 < 1e-10
    assert rel(F, ref["F"]) < 1e-8
    if forcing:
        ctx.set_inexact_newton(0)
        ctx.set_F(None)
        plain = ctx.solve(mask, target, 1e-8, 1e-10, cg_rel=1e-4)
        assert out["cg"].sum() < plain["cg"].sum()


def test_radix3_grid_solve():
    mf = lib()
    nx, ny, nz = 24, 12, 18
    shape = (nz, ny, nx)
    ph = inputs.periodic_sphere_phase(shape, [(12, 6, 9)], 4.0)
    params = np.array([[1.0, 2.0], [5.0, 10.0]])
    ctx = mf.Context(nx, ny, nz, mf.MF_FP64)
    ctx.set_material(mf.MF_NEOHOOKE, params, ph)
    om = omat.Material(ph, omat.NEOHOOKE, params)
    mask = CASE1[None].copy()
    target = np.array([[1.03, 0, 0, 0, 0, 0, 0, 0, 0]])
    out = ctx.solve(mask, target, 1e-10, 1e-12)
    ref = osolver.solve(om, mask, target, 1e-10, 1e-12)
    F, _ = ctx.get_fields()
    assert rel(F, ref["F"]) < 1e-10


def test_status_nonpositive_J():
    mf = lib()
    ctx, _ = sphere_cell(mf, 8, mf.MF_FP64)
    F = inputs.random_F((8, 8, 8), 1, 0.01)
    F[8, 3, 3, 3] = -1.0        # one inverted voxel, planted on the host
    ctx.set_F(F)
    with pytest.raises(mf.MixFFTError) as e:
        ctx.constitutive()
    assert e.value.status == mf.MF_NONPOSITIVE_J


def test_status_not_converged_and_invalid():
    mf = lib()
    ctx, _ = sphere_cell(mf, 8, mf.MF_FP64)
    mask, target = inputs.history_uniaxial_stress_ramp(1, 0.1)
    with pytest.raises(mf.MixFFTError) as e:
        ctx.solve(mask, target, 1e-8, 1e-10, max_cg=1)
    assert e.value.status == mf.MF_NOT_CONVERGED
    ctx.set_F(None)
    with pytest.raises(mf.MixFFTError) as e:
        ctx.solve(mask, target, 1e-8, 1e-10, max_newton=1)
    assert e.value.status == mf.MF_NOT_CONVERGED
    bad = mask.copy(); bad[0, 0] = 2
    with pytest.raises(mf.MixFFTError) as e:
        ctx.solve(bad, target)
    assert e.value.status == mf.MF_INVALID_ARG
    with pytest.raises(mf.MixFFTError) as e:
        ctx.set_material(mf.MF_NEOHOOKE, np.array([[1.0, 2.0]]), np.ones((8, 8, 8), np.int32))
    assert e.value.status == mf.MF_INVALID_ARG


def test_status_cg_breakdown_rotation_mode():
    """Full stress control in compression leaves the rigid rotation with
    negative curvature; the library reports it instead of diverging."""
    mf = lib()
    g, params, R = polycrystal((6, 6, 6), 5, 50)
    ctx = mf.Context(6, 6, 6, mf.MF_FP64)
    ctx.set_material(mf.MF_SVK_CUBIC, params, g, rot=R)
    mask, target = inputs.history_uniaxial_stress_ramp(2, -0.2)
    with pytest.raises(mf.MixFFTError) as e:
        ctx.solve(mask, target, 1e-8, 1e-10, max_cg=2000)
    assert e.value.status in (mf.MF_CG_BREAKDOWN, mf.MF_NOT_CONVERGED)


def test_device_wait_timeout_is_reported():
    """Failure detection without a fault: a device barrier wait that nothing
    completes gives up after its bound and the library reports
    MF_DEVICE_TIMEOUT; the device keeps working (a solve runs afterwards)."""
    mf = lib()
    assert mf.selftest_wait_timeout(1000) == mf.MF_DEVICE_TIMEOUT
    assert mf.selftest_wait_timeout(1) == mf.MF_DEVICE_TIMEOUT
    ctx, om = sphere_cell(mf, 8, mf.MF_FP32_INNER)
    mask, target = inputs.history_uniaxial_stress_ramp(1, 0.02)
    out = ctx.solve(mask, target, 1e-8, 1e-10)
    assert out["newton"][0] >= 1


@pytest.mark.parametrize("prec", [0, 1])
def test_extrapolating_predictor_reaches_the_oracle(prec):
    """mf_set_predictor(MF_PRED_EXTRAPOLATE) on a cyclic stress history (a
    ramp, two reversals): the converged averages and fields are the oracle's
    (uniform predictor) to the precision's tolerance, with no more Newton or
    CG iterations in total than the uniform predictor, and fewer Newton
    iterations on the steps along a ramp."""
    mf = lib()
    n = 16
    g, params, R = polycrystal((n, n, n), 12, 41)
    om = omat.Material(g, omat.SVK_CUBIC, params, R)
    mask, target = inputs.fix_rotation(*inputs.history_cyclic_stress(12, 0.2))
    ref = osolver.solve(om, mask, target, 1e-10, 1e-12)
    outs = {}
    for pred in (mf.MF_PRED_UNIFORM, mf.MF_PRED_EXTRAPOLATE, mf.MF_PRED_QUADRATIC):
        ctx = mf.Context(n, n, n, prec)
        ctx.set_material(mf.MF_SVK_CUBIC, params, g, rot=R)
        ctx.set_predictor(pred)
        out = ctx.solve(mask, target, 1e-8, 1e-10, cg_rel=1e-4)
        F, _ = ctx.get_fields()
        tol_mean = 1e-10 if prec == mf.MF_FP64 else 1e-9
        assert rel(out["Fbar"], ref["Fbar"]) < tol_mean
        assert np.max(np.abs(out["Pbar"] - ref["Pbar"])) / 168.0 < tol_mean
        assert rel(F, ref["F"]) < 1e-8
        outs[pred] = out
    u, x, q = outs[mf.MF_PRED_UNIFORM], outs[mf.MF_PRED_EXTRAPOLATE], outs[mf.MF_PRED_QUADRATIC]
    print("predictor", prec, u["newton"].tolist(), x["newton"].tolist(), q["newton"].tolist(),
          u["cg"].sum(), x["cg"].sum(), q["cg"].sum())
    assert x["newton"].sum() < u["newton"].sum()
    assert x["cg"].sum() <= u["cg"].sum()
    assert q["newton"].sum() <= x["newton"].sum()


@pytest.mark.parametrize("pred", [1, 2])
def test_extrapolating_predictor_across_calls(pred):
    """The predictor's converged steps carry over between mf_solve calls
    (two for the linear, three for the quadratic extrapolation):
    a history solved one step per call takes the same Newton iterations and
    reaches the same states as the same history in one call.  Not bit for
    bit: a launch recomputes <F> from the field (another summation order than
    the constitutive pass), and the forcing of a step's first inner solve
    follows the size of earlier corrections; the converged states agree to
    their accuracy (about the last correction times its forcing, 1e-11)."""
    mf = lib()
    n = 16
    g, params, R = polycrystal((n, n, n), 12, 41)
    mask, target = inputs.fix_rotation(*inputs.history_cyclic_stress(8, 0.2))
    ctx = mf.Context(n, n, n, mf.MF_FP32_INNER)
    ctx.set_material(mf.MF_SVK_CUBIC, params, g, rot=R)
    ctx.set_predictor(pred)
    one = ctx.solve(mask, target, 1e-8, 1e-10, cg_rel=1e-4)
    F1, _ = ctx.get_fields()
    ctx.set_F(None)
    for k in range(mask.shape[0]):
        o = ctx.solve(mask[k:k + 1], target[k:k + 1], 1e-8, 1e-10, cg_rel=1e-4)
        assert rel(o["Fbar"][0], one["Fbar"][k]) < 1e-10
        # within one call a step that ends on an unprojected FP32 correction
        # takes <P> from the linearisation <P> + <K:dF>; one step per call
        # always evaluates P at the final F
        assert np.max(np.abs(o["Pbar"][0] - one["Pbar"][k])) / 168.0 < 1e-10
        np.testing.assert_array_equal(o["newton"][0], one["newton"][k])
    F2, _ = ctx.get_fields()
    # the FP32 inner solves carry the last-bit differences of their inputs
    # into the fields at FP32-solve level (measured 8e-13)
    assert rel(F2, F1) < 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_quadratic_predictor_on_a_bent_path_with_a_mask_change(prec):
    """MF_PRED_QUADRATIC where its conditions fail part of the time: the
    prescribed values turn a corner (the three kept targets are not on one
    line: linear start along the last leg, or none) and the control mask
    changes halfway (kept states of the other mask are not used).  Every
    step reaches the oracle's converged state (uniform start) to the
    precision's tolerance."""
    mf = lib()
    n = 16
    g, params, R = polycrystal((n, n, n), 12, 53)
    om = omat.Material(g, omat.SVK_CUBIC, params, R)
    m1 = np.array([1, 0, 0, 1, 1, 0, 1, 1, 1], np.uint8)   # P11 ramp, F12 = F13 = F23 = 0
    m2 = np.array([1, 0, 0, 0, 1, 0, 0, 1, 1], np.uint8)   # F21, F31 prescribed as well
    mask = np.array([m1] * 5 + [m2] * 5)
    target = np.zeros((10, 9))
    p11 = [0.03, 0.06, 0.09, 0.09, 0.09, 0.12, 0.15, 0.15, 0.12, 0.09]
    p22 = [0.0, 0.0, 0.0, 0.03, 0.06, 0.06, 0.06, 0.09, 0.12, 0.12]
    for k in range(10):
        target[k, 0] = p11[k]
        target[k, 4] = p22[k]
    ref = osolver.solve(om, mask, target, 1e-10, 1e-12)
    ctx = mf.Context(n, n, n, prec)
    ctx.set_material(mf.MF_SVK_CUBIC, params, g, rot=R)
    ctx.set_predictor(mf.MF_PRED_QUADRATIC)
    out = ctx.solve(mask, target, 1e-8, 1e-10, cg_rel=1e-4)
    F, _ = ctx.get_fields()
    tol_mean = 1e-10 if prec == mf.MF_FP64 else 1e-9
    print("bent path", prec, out["newton"].tolist(), out["cg"].tolist())
    assert rel(out["Fbar"], ref["Fbar"]) < tol_mean
    assert np.max(np.abs(out["Pbar"] - ref["Pbar"])) / 168.0 < tol_mean
    assert rel(F, ref["F"]) < 1e-8
    check_control(out, mask, target, tol_mean * 168.0, 1e-14)

