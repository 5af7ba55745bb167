"""Pins of the oracle's Newton-CG solver under stress and mixed control
(Eq. linequil2ast, eq:mixedeqil): the affine solution of a homogeneous cell,
the laminate closed form, exact satisfaction of the prescribed components,
agreement between stress-, mixed- and strain-controlled runs (Sec. 3.1), and
dense brute-force solves."""
import numpy as np
import pytest
from scipy import optimize

from oracle import dense, materials as mat, projector, solver
from paper_1901_06531_gb300 import inputs

CASE1 = np.array([0, 0, 0, 1, 1, 0, 1, 1, 1], np.uint8)   # paper's load case (1)
TIGHT = dict(tol_newton=1e-11, tol_cg=1e-13)


def uniform_P(m, Fv):
    """P of the material's phase 0 at a uniform F (9,)."""
    F = np.broadcast_to(np.asarray(Fv)[:, None, None, None], (9, 1, 1, 1)).copy()
    one = mat.Material(np.zeros((1, 1, 1), np.int32), m.model, m.params[:1],
                       None if m.rot is None else m.rot[:1])
    return one.PK(F)[0][:, 0, 0, 0]


def affine_solution(m, mask, target):
    """Uniform F with F_ij = target on mask 0 and P(F)_IJ = target on mask 1,
    from an independent 9-unknown root solve."""
    free = np.flatnonzero(mask == 1)

    def build(u):
        F = np.where(mask == 0, target, 0.0)
        F[free] = u
        return F

    def fun(u):
        return uniform_P(m, build(u))[free] - target[free]

    if free.size == 0:
        return build(np.zeros(0))
    u0 = np.array([1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0])[free]
    sol = optimize.root(fun, u0, method="hybr", tol=1e-15)
    assert np.max(np.abs(fun(sol.x))) < 1e-13
    return build(sol.x)


@pytest.mark.parametrize("model", ["neohooke", "svk"])
@pytest.mark.parametrize("mname", ["strain", "stress", "case1"])
def test_affine_exact_homogeneous(model, mname):
    shape = (4, 4, 4)
    ph = np.zeros(shape, np.int32)
    if model == "neohooke":
        m = mat.Material(ph, mat.NEOHOOKE, [[1.0, 2.0]])
    else:
        m = mat.Material(ph, mat.SVK_CUBIC, [[168.0, 121.0, 75.0]], inputs.random_rotations(1, 30))
    amp = 0.05 if model == "neohooke" else 0.5
    if mname == "strain":
        mask = np.zeros(9, np.uint8)
        target = np.array([1.03, 0.01, 0, 0.02, 0.99, 0, 0, -0.01, 1.0])
    elif mname == "stress":
        mask = np.ones(9, np.uint8)
        # tensile, so that the rigid rotation has positive curvature
        target = np.zeros(9); target[0] = amp; target[4] = 0.3 * amp; target[1] = target[3] = 0.2 * amp
    else:
        mask = CASE1.copy()
        target = np.zeros(9); target[0] = 1.02
    out = solver.solve(m, mask[None], target[None], **TIGHT)
    Fa = affine_solution(m, mask, target)
    F = out["F"].reshape(9, -1)
    assert np.max(np.abs(F - Fa[:, None])) < 1e-12


def laminate_solution(m_params, model, axis, f, mask, target):
    """Two-layer laminate normal to e_axis, volume fraction f of phase 1.
    F1 = Fbar + (1-f) a (x) e, F0 = Fbar - f a (x) e; traction continuity
    P1 e = P0 e; f P1 + (1-f) P0 = P-bar on the stress-controlled components."""
    e = np.zeros(3); e[axis] = 1.0
    free = np.flatnonzero(mask == 1)
    ph1 = mat.Material(np.zeros((1, 1, 1), np.int32), model, m_params[1:2])
    ph0 = mat.Material(np.zeros((1, 1, 1), np.int32), model, m_params[0:1])

    def P(matl, Fv):
        return matl.PK(Fv[:, None, None, None])[0][:, 0, 0, 0]

    def unpack(u):
        a = u[:3]
        Fb = np.where(mask == 0, target, 0.0)
        Fb[free] = u[3:]
        jump = np.outer(a, e).ravel()
        return Fb, Fb + (1 - f) * jump, Fb - f * jump

    def fun(u):
        Fb, F1, F0 = unpack(u)
        P1, P0 = P(ph1, F1), P(ph0, F0)
        t = (P1 - P0).reshape(3, 3) @ e
        avg = (f * P1 + (1 - f) * P0)[free] - target[free]
        return np.concatenate([t, avg])

    u0 = np.concatenate([np.zeros(3), np.array([1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0])[free]])
    sol = optimize.root(fun, u0, method="hybr", tol=1e-15)
    assert np.max(np.abs(fun(sol.x))) < 1e-13
    return unpack(sol.x)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("mname", ["stress", "case1"])
def test_laminate_closed_form(axis, mname):
    shape = (6, 8, 10)
    n_axis = (shape[2], shape[1], shape[0])[axis]
    n_a = 4 if n_axis > 6 else 2        # even layer thickness: no Nyquist content
    ph = inputs.laminate_phase(shape, axis, n_a, offset=1)
    params = np.array([[1.0, 2.0], [10.0, 20.0]])
    m = mat.Material(ph, mat.NEOHOOKE, params)
    if mname == "stress":
        mask = np.ones(9, np.uint8)
        target = np.zeros(9); target[0] = 0.08; target[4] = 0.03; target[5] = target[7] = 0.01
    else:
        mask = CASE1.copy()
        target = np.zeros(9); target[0] = 1.04
    out = solver.solve(m, mask[None], target[None], **TIGHT)
    f = n_a / n_axis
    Fb, F1, F0 = laminate_solution(params, mat.NEOHOOKE, axis, f, mask, target)
    F = out["F"].reshape(9, -1)
    sel = ph.reshape(-1) == 1
    assert np.max(np.abs(F[:, sel] - F1[:, None])) < 1e-10
    assert np.max(np.abs(F[:, ~sel] - F0[:, None])) < 1e-10
    np.testing.assert_allclose(out["Fbar"][0], Fb, atol=1e-11)


def particle_material(n=8):
    ph = inputs.centred_sphere(n)
    return mat.Material(ph, mat.NEOHOOKE, [[1.0, 2.0], [10.0, 20.0]])


def test_control_exactness_every_step():
    m = particle_material()
    for mask, target in (inputs.history_uniaxial_stress_ramp(3, 0.1),
                         inputs.history_mixed_strain11(3, 1.05),
                         inputs.fix_rotation(*inputs.history_cyclic_stress(4, 0.1))):
        out = solver.solve(m, mask, target, **TIGHT)
        for k in range(mask.shape[0]):
            s = mask[k] == 1
            pb = np.max(np.abs(target[k][s])) if s.any() else 0.0
            assert np.max(np.abs(out["Pbar"][k][s] - target[k][s]), initial=0) < 1e-12 * max(1, pb)
            assert np.max(np.abs(out["Fbar"][k][~s] - target[k][~s]), initial=0) < 1e-14


def test_stress_mixed_strain_cases_share_the_endpoint():
    """Sec. 3.1: case (1) mixed (F11 ramp, the rest stress free), case (2) full
    stress ramp to case (1)'s final P-bar, case (3) full strain ramp to case
    (1)'s final F-bar, reach the same endpoint; for a hyperelastic material
    (1) and (2) are superposed."""
    m = particle_material()
    n = 4
    mask1 = np.tile(CASE1, (n, 1))
    t1 = np.zeros((n, 9)); t1[:, 0] = 1.0 + 0.06 * np.arange(1, n + 1) / n
    o1 = solver.solve(m, mask1, t1, **TIGHT)
    Pend, Fend = o1["Pbar"][-1], o1["Fbar"][-1]
    ramp = np.arange(1, n + 1)[:, None] / n
    o2 = solver.solve(m, np.ones((n, 9), np.uint8), Pend[None] * ramp, **TIGHT)
    eye = np.array([1.0, 0, 0, 0, 1, 0, 0, 0, 1])
    o3 = solver.solve(m, np.zeros((n, 9), np.uint8), eye + (Fend - eye)[None] * ramp, **TIGHT)
    ref = o1["F"]
    for o in (o2, o3):
        assert np.max(np.abs(o["F"] - ref)) < 1e-10
        assert np.max(np.abs(o["P"] - o1["P"])) < 1e-10
    # (1) and (2): the same stress-strain curve at matching P11
    # path independence: one strain-controlled step straight to Fend
    o4 = solver.solve(m, np.zeros((1, 9), np.uint8), Fend[None], **TIGHT)
    assert np.max(np.abs(o4["F"] - ref)) < 1e-10


@pytest.mark.parametrize("n", [3, 4, 5])
def test_dense_linear_solve_matches_cg(n):
    shape = (n, n, n)
    rng = np.random.default_rng(40)
    ph = rng.integers(0, 2, shape).astype(np.int32)
    m = mat.Material(ph, mat.NEOHOOKE, [[1.0, 2.0], [10.0, 20.0]])
    F = inputs.random_F(shape, 41, 0.05)
    P, K = m.PK(F)
    for mask in (np.zeros(9, np.uint8), CASE1):
        G = dense.gstar_matrix(shape, mask)
        A = G @ dense.k_matrix(K) @ G
        np.testing.assert_allclose(A, A.T, atol=1e-12 * np.max(np.abs(A)))
        # G* is an orthogonal projector
        np.testing.assert_allclose(G @ G, G, atol=1e-13)
        np.testing.assert_allclose(G, G.T, atol=1e-14)
        b = solver.residual(P, mask, np.zeros(9))
        x_cg, _ = solver.cg(lambda v: solver.matvec(K, v, mask), b, 1e-15, 5000)
        x_lu, _ = dense.solve_projected(K, b, mask)
        assert np.max(np.abs(x_cg - x_lu)) < 1e-12 * max(1.0, np.max(np.abs(x_lu)))
        # the solution solves the projected system and stays in range(G*)
        np.testing.assert_allclose(A @ x_lu.ravel(), b.ravel(), atol=1e-12)
        np.testing.assert_allclose(G @ x_lu.ravel(), x_lu.ravel(), atol=1e-12)


def test_dense_newton_matches_newton_cg():
    shape = (4, 4, 4)
    m = mat.Material(inputs.centred_sphere(4, 0.3), mat.NEOHOOKE, [[1.0, 2.0], [10.0, 20.0]])
    mask = np.tile(CASE1, (2, 1))
    target = np.zeros((2, 9)); target[:, 0] = [1.03, 1.06]
    o_cg = solver.solve(m, mask, target, **TIGHT)
    o_lu = solver.solve(m, mask, target, linear_solver=dense.solve_projected, **TIGHT)
    assert np.max(np.abs(o_cg["F"] - o_lu["F"])) < 1e-12
    np.testing.assert_allclose(o_cg["Pbar"], o_lu["Pbar"], atol=1e-12)
    np.testing.assert_array_equal(o_cg["newton"], o_lu["newton"])


def test_newton_converges_quadratically():
    m = particle_material()
    ratios = []
    orig = solver.cg

    def spy(apply_A, b, tol, maxit):
        x, it = orig(apply_A, b, tol, maxit)
        ratios.append(np.sqrt(np.sum(x * x)))
        return x, it

    solver.cg = spy
    try:
        solver.solve(m, np.ones((1, 9), np.uint8), np.array([[0.1, 0, 0, 0, 0, 0, 0, 0, 0]]), **TIGHT)
    finally:
        solver.cg = orig
    # |dF_{k+1}| ~ |dF_k|^2 once in the basin
    assert len(ratios) >= 3
    r = np.asarray(ratios)
    assert r[2] < 10 * r[1] ** 2 / r[0] + 1e-12


def test_all_stress_compression_polycrystal_has_rotation_mode():
    """Under full stress control a compressive P11 leaves the rigid rotation of
    the cell unconstrained with negative curvature: CG meets p.Ap <= 0.  The
    paper's case (1) pattern (F12 = F13 = F23 = 0 prescribed) removes it."""
    g, _ = inputs.voronoi((6, 6, 6), 5, 50)
    m = mat.Material(g, mat.SVK_CUBIC, np.tile([168.0, 121.0, 75.0], (5, 1)),
                     inputs.random_rotations(5, 51))
    mask, target = inputs.history_uniaxial_stress_ramp(2, -0.2)
    with pytest.raises((solver.CGBreakdown, solver.NotConverged)):
        solver.solve(m, mask, target, 1e-8, 1e-10, max_cg=2000)
    mask_f, target_f = inputs.fix_rotation(mask, target)
    out = solver.solve(m, mask_f, target_f, 1e-8, 1e-10)
    assert abs(out["Pbar"][-1][0] + 0.2) < 1e-10
