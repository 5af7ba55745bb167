"""GPU parity of the single-application steps against the oracle: the
constitutive update (Eq. eq:lineariz), the projected operator G*(K:x)
(Eq. linequil2ast with G* of Eq. eq:Gnewnew) and the FP64 residual.  One
application involves no iteration, so FP64 must agree to 1e-12 relative."""
import numpy as np
import pytest

from oracle import materials as omat, projector, solver as osolver
from paper_1901_06531_gb300 import inputs

from gpu_util import fp32_operator_error, lib, neohooke_two_phase, polycrystal, rel

pytestmark = pytest.mark.gpu

MASKS = [np.zeros(9, np.uint8), np.ones(9, np.uint8),
         np.array([0, 0, 0, 1, 1, 0, 1, 1, 1], np.uint8)]
# (nx, ny, nz): smallest grid, cubic, anisotropic with radix 3, odd nz, 3-stage
# planes, a grid spanning many z-pass tiles
SHAPES = [(4, 4, 2), (16, 16, 16), (12, 8, 6), (48, 36, 18), (24, 6, 9), (32, 64, 12)]
# square x-y planes with z lengths the fixed-size transform kernels cover
SHAPES_V2 = [(32, 32, 32), (64, 64, 16), (128, 128, 16), (16, 16, 128), (64, 64, 64), (48, 48, 96),
             (96, 96, 48)]


def torch_field(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a).reshape(-1), dtype=dtype, device="cuda")


def make(mf, shape_xyz, precision, model="nh", seed=0, scale=False):
    nx, ny, nz = shape_xyz
    shape = (nz, ny, nx)
    ctx = mf.Context(nx, ny, nz, precision)
    sc = inputs.lognormal_scale(shape, 0.3, seed + 7) if scale else None
    if model == "nh":
        ph, params = neohooke_two_phase(shape, seed)
        ctx.set_material(mf.MF_NEOHOOKE, params, ph, scale=sc)
        om = omat.Material(ph, omat.NEOHOOKE, params, scale=sc)
    else:
        g, params, R = polycrystal(shape, 5, seed)
        ctx.set_material(mf.MF_SVK_CUBIC, params, g, rot=R, scale=sc)
        om = omat.Material(g, omat.SVK_CUBIC, params, R, scale=sc)
    F = inputs.random_F(shape, seed + 1, 0.08)
    ctx.set_F(F)
    return ctx, om, F


def K45_from_oracle(K):
    out = np.empty((45,) + K.shape[2:])
    t = 0
    for a in range(9):
        for b in range(a, 9):
            out[t] = K[a, b]
            t += 1
    return out


@pytest.mark.parametrize("model", ["nh", "svk"])
@pytest.mark.parametrize("scale", [False, True])
def test_constitutive_fp64(model, scale):
    mf = lib()
    ctx, om, F = make(mf, (12, 8, 6), mf.MF_FP64, model, seed=3, scale=scale)
    ctx.constitutive()
    Fg, Pg = ctx.get_fields()
    P, K = om.PK(F)
    assert rel(Pg, P) < 1e-13
    assert rel(ctx.get_tangent(), K45_from_oracle(K)) < 1e-13


@pytest.mark.parametrize("model", ["nh", "svk"])
@pytest.mark.parametrize("scale", [False, True])
@pytest.mark.parametrize("shape", [(12, 8, 6), (32, 32, 32)])
def test_stress_double_word(model, scale, shape):
    """P(F) in the FP32-inner context's double-word outer arithmetic (about
    48 bits, both laws evaluated from H = F - I) agrees with the FP64 oracle
    to 1e-13 relative, and so does <P> (relative to max |P|: the 48-bit
    material constants of a grain give all its voxels the same rounding, so
    the average keeps the per-voxel relative error); the FP64 setting of the
    same context agrees as well."""
    mf = lib()
    ctx, om, F = make(mf, shape, mf.MF_FP32_INNER, model, seed=21, scale=scale)
    P, _ = om.PK(F)
    for arith in (mf.MF_OUTER_DOUBLE_WORD, mf.MF_OUTER_FP64):
        ctx.set_outer_arith(arith)
        meanP = ctx.stress()
        Fg, Pg = ctx.get_fields()
        assert np.array_equal(Fg, F)
        assert rel(Pg, P) < 1e-13, arith
        np.testing.assert_allclose(meanP, P.reshape(9, -1).mean(1), rtol=0, atol=1e-13 * np.abs(P).max())


def test_constitutive_fp32_tangent_is_rounded_fp64():
    mf = lib()
    ctx, om, F = make(mf, (8, 8, 4), mf.MF_FP32_INNER, "svk", seed=4)
    ctx.constitutive()
    _, Pg = ctx.get_fields()
    P, K = om.PK(F)
    assert rel(Pg, P) < 1e-13                      # P stays FP64
    K45 = K45_from_oracle(K)
    # FP64 tangent rounded once to FP32: within half an FP32 ulp (plus FP64 noise)
    Kg = ctx.get_tangent()
    assert np.all(np.abs(Kg - K45) <= 6.0e-8 * np.abs(K45) + 1e-12 * np.max(np.abs(K45)))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mi", range(len(MASKS)))
def test_matvec_fp64(shape, mi):
    import torch
    mf = lib()
    ctx, om, F = make(mf, shape, mf.MF_FP64, "nh" if mi != 1 else "svk", seed=5)
    ctx.constitutive()
    nx, ny, nz = shape
    x = inputs.random_field((nz, ny, nx), 6)
    xt = torch_field(x, torch.float64)
    yt = torch.full_like(xt, float("nan"))
    ctx.matvec(xt, yt, MASKS[mi])
    ctx.sync()
    _, K = om.PK(F)
    ref = osolver.matvec(K, x, MASKS[mi])
    got = yt.cpu().numpy().reshape(ref.shape)
    assert np.all(np.isfinite(got))
    assert rel(got, ref) < 1e-12


@pytest.mark.parametrize("shape", SHAPES[:4])
@pytest.mark.parametrize("model,scale", [("svk", False), ("nh", False), ("nh", True), ("svk", True)])
def test_matvec_fp32(shape, model, scale):
    """FP32 operator with the matrix-free tangent (from F - I in FP32 and the
    phase parameters) against the FP64 oracle: the error is the FP32
    rounding of the tangent apply and of the transforms, relative to the
    field norm."""
    import torch
    mf = lib()
    ctx, om, F = make(mf, shape, mf.MF_FP32_INNER, model, seed=8, scale=scale)
    ctx.constitutive()
    nx, ny, nz = shape
    x = inputs.random_field((nz, ny, nx), 9)
    xt = torch_field(x, torch.float32)
    yt = torch.full_like(xt, float("nan"))
    ctx.matvec(xt, yt, MASKS[2])
    ctx.sync()
    _, K = om.PK(F)
    ref = osolver.matvec(K, x.astype(np.float32).astype(np.float64), MASKS[2])
    got = yt.cpu().numpy().astype(np.float64).reshape(ref.shape)
    print("fp32 operator", shape, model, scale, fp32_operator_error(got, ref))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mi", range(len(MASKS)))
def test_residual_fp64(shape, mi):
    import torch
    mf = lib()
    ctx, om, F = make(mf, shape, mf.MF_FP64, "nh", seed=10)
    ctx.constitutive()
    pbar = np.array([0.05, 0.01, 0.0, -0.01, 0.02, 0.0, 0.0, 0.0, -0.03])
    nx, ny, nz = shape
    b = torch.full((9 * nx * ny * nz,), float("nan"), dtype=torch.float64, device="cuda")
    meanP = ctx.residual(MASKS[mi], pbar, b)
    P, _ = om.PK(F)
    ref = osolver.residual(P, MASKS[mi], pbar)
    got = b.cpu().numpy().reshape(ref.shape)
    assert rel(got, ref) < 1e-12
    np.testing.assert_allclose(meanP, P.reshape(9, -1).mean(1), rtol=0, atol=1e-14)


@pytest.mark.parametrize("shape", SHAPES_V2)
@pytest.mark.parametrize("mi", [0, 2])
def test_fixed_size_kernels_fp64(shape, mi):
    """The fixed-size kernels (half-length real rows, radix-8/16 stages) in
    FP64: operator and residual to 1e-12 relative."""
    import torch
    mf = lib()
    ctx, om, F = make(mf, shape, mf.MF_FP64, "nh", seed=12)
    ctx.constitutive()
    nx, ny, nz = shape
    x = inputs.random_field((nz, ny, nx), 13)
    xt = torch_field(x, torch.float64)
    yt = torch.full_like(xt, float("nan"))
    ctx.matvec(xt, yt, MASKS[mi])
    P, K = om.PK(F)
    ref = osolver.matvec(K, x, MASKS[mi])
    assert rel(yt.cpu().numpy().reshape(ref.shape), ref) < 1e-12
    pbar = np.array([0.05, 0.01, 0.0, -0.01, 0.02, 0.0, 0.0, 0.0, -0.03])
    b = torch.full_like(xt, float("nan"))
    meanP = ctx.residual(MASKS[mi], pbar, b)
    refb = osolver.residual(P, MASKS[mi], pbar)
    assert rel(b.cpu().numpy().reshape(refb.shape), refb) < 1e-12
    np.testing.assert_allclose(meanP, P.reshape(9, -1).mean(1), rtol=0, atol=1e-14)


@pytest.mark.parametrize("shape", SHAPES_V2)
@pytest.mark.parametrize("mi", [0, 2])
@pytest.mark.parametrize("model", ["nh", "svk"])
def test_residual_double_word(shape, mi, model):
    """FP32-inner contexts compute the residual transforms in double-word FP32
    arithmetic (about 48 significant bits): the FP64 residual still agrees
    with the oracle to 1e-12 relative (max norm) and <P> to 1e-13 relative
    to max |P|; the FP64 setting of the same context gives the same
    agreement."""
    import torch
    mf = lib()
    ctx, om, F = make(mf, shape, mf.MF_FP32_INNER, model, seed=18)
    ctx.constitutive()
    nx, ny, nz = shape
    P, _ = om.PK(F)
    pbar = np.array([0.05, 0.01, 0.0, -0.01, 0.02, 0.0, 0.0, 0.0, -0.03])
    refb = osolver.residual(P, MASKS[mi], pbar)
    for arith in (mf.MF_OUTER_DOUBLE_WORD, mf.MF_OUTER_FP64):
        ctx.set_outer_arith(arith)
        b = torch.full((9 * nx * ny * nz,), float("nan"), dtype=torch.float64, device="cuda")
        meanP = ctx.residual(MASKS[mi], pbar, b)
        assert rel(b.cpu().numpy().reshape(refb.shape), refb) < 1e-12, arith
        np.testing.assert_allclose(meanP, P.reshape(9, -1).mean(1), rtol=0, atol=1e-13 * np.abs(P).max())


def test_outer_arith_rejects_unknown():
    mf = lib()
    ctx = mf.Context(16, 16, 16, mf.MF_FP32_INNER)
    with pytest.raises(mf.MixFFTError) as e:
        ctx.set_outer_arith(2)
    assert e.value.status == mf.MF_INVALID_ARG


@pytest.mark.parametrize("shape", SHAPES_V2)
def test_fixed_size_kernels_fp32(shape):
    import torch
    mf = lib()
    ctx, om, F = make(mf, shape, mf.MF_FP32_INNER, "svk", seed=14)
    ctx.constitutive()
    nx, ny, nz = shape
    x = inputs.random_field((nz, ny, nx), 15)
    xt = torch_field(x, torch.float32)
    yt = torch.full_like(xt, float("nan"))
    ctx.matvec(xt, yt, MASKS[2])
    _, K = om.PK(F)
    ref = osolver.matvec(K, x.astype(np.float32).astype(np.float64), MASKS[2])
    got = yt.cpu().numpy().astype(np.float64).reshape(ref.shape)
    print("fp32 fixed-size operator", shape, fp32_operator_error(got, ref))


def test_full_size_polycrystal_operator_and_residual():
    """The bench's workload and launch configuration (128^3, 200-grain SVK
    polycrystal, rotation-fixed mask): FP32 operator against the FP64
    oracle element by element (within 2 log2(N) eps32 max|y|), and the FP64 residual (double-word transforms
    in the FP32-inner context) to 1e-12."""
    import torch
    mf = lib()
    n = 128
    g, _ = inputs.voronoi((n, n, n), 200, 1003)
    R = inputs.random_rotations(200, 1004)
    params = np.tile([168.0, 121.0, 75.0], (200, 1))
    mask, target = inputs.fix_rotation(*inputs.history_cyclic_stress(20, 0.2))
    m0 = mask[0]
    F = inputs.random_F((n, n, n), 16, 0.002)
    om = omat.Material(g, omat.SVK_CUBIC, params, R)
    P, K = om.PK(F)
    for prec in (mf.MF_FP32_INNER, mf.MF_FP64):
        ctx = mf.Context(n, n, n, prec)
        ctx.set_material(mf.MF_SVK_CUBIC, params, g, rot=R)
        ctx.set_F(F)
        ctx.constitutive()
        if prec == mf.MF_FP32_INNER:
            x = inputs.random_field((n, n, n), 17)
            xt = torch_field(x, torch.float32)
            yt = torch.empty_like(xt)
            ctx.matvec(xt, yt, m0)
            ref = osolver.matvec(K, x.astype(np.float32).astype(np.float64), m0)
            got = yt.cpu().numpy().astype(np.float64).reshape(ref.shape)
            print("fp32 operator 128^3 polycrystal", fp32_operator_error(got, ref))
        # the FP64 residual: double-word transforms in the FP32-inner
        # context, FP64 transforms in the FP64 one
        b = torch.empty(9 * n ** 3, dtype=torch.float64, device="cuda")
        ctx.residual(m0, target[0] * m0, b)
        refb = osolver.residual(P, m0, target[0] * m0)
        assert rel(b.cpu().numpy().reshape(refb.shape), refb) < 1e-12
        del ctx
        torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", [0, 1])
def test_split_xy_kernels_match_oracle(prec):
    """The separate row (x) and column (y) kernels of large planes, forced on
    a 32^3 cell: operator and residual against the oracle, FP64 to 1e-12,
    FP32 operator element-wise within 2 log2(N) eps32 max|y|."""
    import torch
    mf = lib()
    shape = (32, 32, 32)
    ctx, om, F = make(mf, shape, prec, "svk", seed=31, scale=True)
    ctx.set_xy_split(1)
    ctx.constitutive()
    P, K = om.PK(F)
    x = inputs.random_field((32, 32, 32), 32)
    dt = torch.float32 if prec else torch.float64
    xt = torch_field(x, dt)
    yt = torch.full_like(xt, float("nan"))
    ctx.matvec(xt, yt, MASKS[2])
    xin = x.astype(np.float32).astype(np.float64) if prec else x
    ref = osolver.matvec(K, xin, MASKS[2])
    got = yt.cpu().numpy().astype(np.float64).reshape(ref.shape)
    if prec:
        print("fp32 split operator", fp32_operator_error(got, ref))
    else:
        assert rel(got, ref) < 1e-12
    pbar = np.array([0.05, 0.01, 0.0, -0.01, 0.02, 0.0, 0.0, 0.0, -0.03])
    b = torch.full((9 * 32 ** 3,), float("nan"), dtype=torch.float64, device="cuda")
    ctx.residual(MASKS[2], pbar, b)
    refb = osolver.residual(P, MASKS[2], pbar)
    assert rel(b.cpu().numpy().reshape(refb.shape), refb) < 1e-12


def test_split_xy_choice_is_validated():
    mf = lib()
    ctx = mf.Context(48, 48, 48, mf.MF_FP32_INNER)
    with pytest.raises(mf.MixFFTError):
        ctx.set_xy_split(1)          # no split kernels for 48^2 planes
    big = mf.Context(256, 256, 16, mf.MF_FP32_INNER)
    with pytest.raises(mf.MixFFTError):
        big.set_xy_split(0)          # a 256^2 plane does not fit one block


@pytest.mark.parametrize("prec", [0, 1])
def test_256_plane_operator_matches_oracle(prec):
    """256 x 256 x 16 cell (split x-y kernels): the operator against the
    oracle, FP64 to 1e-12, FP32 element-wise within 2 log2(N) eps32 max|y|; the FP64 residual (double-word
    transforms in the FP32-inner context) to 1e-12."""
    import torch
    mf = lib()
    shape = (256, 256, 16)
    ctx, om, F = make(mf, shape, prec, "nh", seed=33)
    ctx.constitutive()
    P, K = om.PK(F)
    nx, ny, nz = shape
    x = inputs.random_field((nz, ny, nx), 34)
    dt = torch.float32 if prec else torch.float64
    xt = torch_field(x, dt)
    yt = torch.full_like(xt, float("nan"))
    ctx.matvec(xt, yt, MASKS[0])
    xin = x.astype(np.float32).astype(np.float64) if prec else x
    ref = osolver.matvec(K, xin, MASKS[0])
    got = yt.cpu().numpy().astype(np.float64).reshape(ref.shape)
    if prec:
        print("fp32 256-plane operator", fp32_operator_error(got, ref))
    else:
        assert rel(got, ref) < 1e-12
    pbar = np.zeros(9)
    b = torch.empty(9 * nx * ny * nz, dtype=torch.float64, device="cuda")
    ctx.residual(MASKS[0], pbar, b)
    refb = osolver.residual(P, MASKS[0], pbar)
    assert rel(b.cpu().numpy().reshape(refb.shape), refb) < 1e-12


@pytest.mark.parametrize("graph", [False, True])
def test_time_kernels_modes(graph):
    """Both timing modes of mf_time_kernels return four positive finite
    per-launch times; an unknown mode is rejected."""
    mf = lib()
    ctx, _, _ = make(mf, (32, 32, 32), mf.MF_FP32_INNER, model="svk")
    ctx.constitutive()
    mask = np.array([1, 0, 0, 0, 1, 0, 0, 0, 1], dtype=np.uint8)
    ms = ctx.time_kernels(mask, reps=3, graph=graph)
    assert ms.shape == (4,) and np.all(np.isfinite(ms)) and np.all(ms > 0)
    m = np.ascontiguousarray(mask)
    out = np.zeros(4, dtype=np.float32)
    st = mf._lib.mf_time_kernels(ctx.h, m.ctypes.data, 3, 2, out.ctypes.data)
    assert st == mf.MF_INVALID_ARG


@pytest.mark.parametrize("shape", [(128, 128, 16), (96, 96, 48), (48, 48, 96), (64, 64, 64)])
def test_persistent_xy_forward_is_identical(shape):
    """The persistent bulk-copy x-y forward kernel runs the same stages in the
    same order as the per-plane kernel: the FP32 operator is bit-identical."""
    import torch
    mf = lib()
    ctx, _, _ = make(mf, shape, mf.MF_FP32_INNER, "svk", seed=21)
    ctx.constitutive()
    nx, ny, nz = shape
    xt = torch_field(inputs.random_field((nz, ny, nx), 22), torch.float32)
    ys = []
    for on in (0, 1):
        ctx.set_xy_persistent(on)
        y = torch.full_like(xt, float("nan"))
        ctx.matvec(xt, y, MASKS[2])
        ys.append(y.cpu().numpy())
    np.testing.assert_array_equal(ys[0], ys[1])


@pytest.mark.parametrize("which,nz", [(1, 16), (2, 16), (3, 16), (3, 128)])
def test_cluster_xy_kernels_match_oracle(which, nz):
    """The two-CTA cluster x-y kernels (bit 0 the forward pass, bit 1 the
    inverse) in the FP32 operator on 128 x 128 planes: element-wise against
    the FP64 oracle within the FP32 operator bound, and against the
    per-plane kernels to FP32 rounding (the radix-2 y stage moved before the
    x transform changes only the order of the roundings)."""
    import torch
    mf = lib()
    shape = (128, 128, nz)
    ctx, om, F = make(mf, shape, mf.MF_FP32_INNER, "svk", seed=23)
    ctx.constitutive()
    x = inputs.random_field((nz, 128, 128), 24)
    xt = torch_field(x, torch.float32)
    ys = {}
    for w in (0, which):
        ctx.set_xy_cluster(w)
        assert ctx.xy_schedule()[:2] == (2 if w & 1 else 0, 2 if w & 2 else 0)
        y = torch.full_like(xt, float("nan"))
        ctx.matvec(xt, y, MASKS[2])
        ys[w] = y.cpu().numpy().astype(np.float64)
    _, K = om.PK(F)
    ref = osolver.matvec(K, x.astype(np.float32).astype(np.float64), MASKS[2])
    c_cl = fp32_operator_error(ys[which].reshape(ref.shape), ref)
    c_pp = fp32_operator_error(ys[0].reshape(ref.shape), ref)
    d = rel(ys[which], ys[0])
    print("cluster x-y", which, shape, "c", c_cl, "per-plane c", c_pp, "cluster vs per-plane", d)
    assert d < 1e-5


def test_cluster_xy_choice_is_validated():
    mf = lib()
    with pytest.raises(mf.MixFFTError):
        mf.Context(128, 128, 16, mf.MF_FP64).set_xy_cluster(1)          # FP32 inner only
    with pytest.raises(mf.MixFFTError):
        mf.Context(64, 64, 64, mf.MF_FP32_INNER).set_xy_cluster(1)      # 128 x 128 planes only
    with pytest.raises(mf.MixFFTError):
        mf.Context(128, 128, 16, mf.MF_FP32_INNER).set_xy_cluster(4)
    ctx = mf.Context(128, 128, 16, mf.MF_FP32_INNER)
    ctx.set_xy_cluster(2)
    assert ctx.xy_schedule()[:2] == (0, 2)
    ctx.set_xy_persistent(1)
    ctx.set_xy_cluster(3)
    assert ctx.xy_schedule()[:2] == (2, 2)   # the cluster forward pass takes precedence


def test_persistent_xy_forward_solve_and_validation():
    """A load step with the persistent kernel in the CG loop gives the same
    fields as with the per-plane kernel; the choice is validated."""
    mf = lib()
    cell = inputs.batch_of_cells(1, 9, sizes=(48,), nsteps=2)[0]
    fields = []
    for on in (0, 1):
        ctx = mf.Context(48, 48, 48, mf.MF_FP32_INNER)
        ctx.set_material(mf.MF_NEOHOOKE, cell["params"], cell["phase"])
        ctx.set_xy_persistent(on)
        ctx.solve(cell["mask"], cell["target"], 1e-9, 1e-11)
        fields.append(ctx.get_fields()[0])
    np.testing.assert_array_equal(fields[0], fields[1])
    with pytest.raises(mf.MixFFTError):
        mf.Context(48, 48, 48, mf.MF_FP64).set_xy_persistent(1)      # FP32 inner only
    with pytest.raises(mf.MixFFTError):
        mf.Context(32, 32, 32, mf.MF_FP32_INNER).set_xy_persistent(1)   # no kernel for 32^2 planes
    with pytest.raises(mf.MixFFTError):
        mf.Context(48, 48, 48, mf.MF_FP32_INNER).set_xy_persistent(2)
