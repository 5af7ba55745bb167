"""Batched solve (many cells of different sizes and control masks at once,
each on its own stream): every cell's result equals that of its own
single-cell solve, and the oracle's."""
import numpy as np
import pytest

from oracle import materials as omat, solver as osolver
from paper_1901_06531_gb300 import inputs

from gpu_util import lib, rel

pytestmark = pytest.mark.gpu


def make_cells():
    rng = np.random.default_rng(77)
    cells = []
    for shape in [(16, 16, 16), (12, 8, 6), (32, 32, 32), (24, 24, 12), (16, 16, 32)]:
        nx, ny, nz = shape
        ph, _ = inputs.rsa_spheres((nz, ny, nx), min(shape) / 6.0, 0.2, int(rng.integers(1 << 30)))
        contrast = rng.uniform(5, 50)
        params = np.array([[1.0, 2.0], [contrast, 2 * contrast]])
        mask, target = inputs.random_control(3, rng)
        cells.append((shape, ph, params, mask, target))
    return cells


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_equals_single_cell_solves(prec):
    import torch
    mf = lib()
    cells = make_cells()
    ctxs = []
    for shape, ph, params, mask, target in cells:
        c = mf.Context(*shape, prec, stream=torch.cuda.Stream())
        c.set_material(mf.MF_NEOHOOKE, params, ph)
        ctxs.append(c)
    masks = np.stack([c[3] for c in cells])
    targets = np.stack([c[4] for c in cells])
    out = mf.solve_batch(ctxs, masks, targets, 1e-9, 1e-11)
    assert np.all(out["status"] == 0)
    for i, (shape, ph, params, mask, target) in enumerate(cells):
        F_b, P_b = ctxs[i].get_fields()
        single = mf.Context(*shape, prec)
        single.set_material(mf.MF_NEOHOOKE, params, ph)
        o = single.solve(mask, target, 1e-9, 1e-11)
        F_s, _ = single.get_fields()
        # the same kernels on the same data: identical results
        np.testing.assert_array_equal(F_b, F_s)
        np.testing.assert_array_equal(out["newton"][i], o["newton"])
        np.testing.assert_array_equal(out["cg"][i], o["cg"])
        if prec == 0 and i < 3:
            ref = osolver.solve(omat.Material(ph, omat.NEOHOOKE, params), mask, target, 1e-9, 1e-11)
            assert rel(out["Fbar"][i], ref["Fbar"]) < 1e-9
            assert np.max(np.abs(out["Pbar"][i] - ref["Pbar"])) < 1e-9


def test_batch_reports_per_cell_status():
    import torch
    mf = lib()
    cells = make_cells()[:2]
    ctxs = []
    for shape, ph, params, mask, target in cells:
        c = mf.Context(*shape, mf.MF_FP64, stream=torch.cuda.Stream())
        c.set_material(mf.MF_NEOHOOKE, params, ph)
        ctxs.append(c)
    # the second cell starts from an inverted voxel (planted on the host)
    F = inputs.random_F((cells[1][0][2], cells[1][0][1], cells[1][0][0]), 3, 0.01)
    F[8, 0, 0, 0] = -1.0
    ctxs[1].set_F(F)
    masks = np.stack([c[3] for c in cells])
    targets = np.stack([c[4] for c in cells])
    with pytest.raises(mf.MixFFTError) as e:
        mf.solve_batch(ctxs, masks, targets, 1e-9, 1e-11)
    assert e.value.status == mf.MF_NONPOSITIVE_J


@pytest.mark.parametrize("prec", [0, 1])
def test_autotuned_tile_gives_identical_results(prec):
    """The autotuner only changes how many columns a z-pass block takes; the
    arithmetic per column is the same, so results are bitwise identical."""
    import torch
    mf = lib()
    n = 32
    ph, _ = inputs.rsa_spheres((n, n, n), 4.0, 0.2, 5)
    ctx = mf.Context(n, n, n, prec)
    ctx.set_material(mf.MF_NEOHOOKE, np.array([[1.0, 2.0], [10.0, 20.0]]), ph)
    ctx.set_F(inputs.random_F((n, n, n), 6, 0.02))
    ctx.constitutive()
    dt = torch.float32 if prec else torch.float64
    x = torch.as_tensor(inputs.random_field((n, n, n), 7).reshape(-1), dtype=dt, device="cuda")
    mask = np.array([0, 0, 0, 1, 1, 0, 1, 1, 1], np.uint8)
    y0 = torch.empty_like(x)
    ctx.matvec(x, y0, mask)
    zs, ms, xy, xyms = ctx.autotune()
    assert zs in (4, 8, 16) and np.all(ms[ms >= 0] > 0)
    assert xy == 0 and np.all(xyms == -1.0)     # no persistent x-y kernel for 32^2 planes
    y1 = torch.empty_like(x)
    ctx.matvec(x, y1, mask)
    assert torch.equal(y0, y1)



def test_autotuner_picks_the_xy_schedule():
    """For an FP32-inner cell with 64^2 planes the autotuner times both x-y
    forward schedules and keeps the per-plane one unless the persistent one
    is faster by more than 3%; an explicit choice wins over it;
    the operator is bitwise the same under either."""
    import torch
    mf = lib()
    n = 64
    ph, _ = inputs.rsa_spheres((n, n, n), 5.0, 0.2, 8)
    ctx = mf.Context(n, n, n, mf.MF_FP32_INNER)
    ctx.set_material(mf.MF_NEOHOOKE, np.array([[1.0, 2.0], [10.0, 20.0]]), ph)
    ctx.set_F(inputs.random_F((n, n, n), 9, 0.02))
    ctx.constitutive()
    zs, ms, xy, xyms = ctx.autotune()
    assert xy in (0, 1) and np.all(xyms > 0)
    assert xy == (1 if xyms[1] < 0.97 * xyms[0] else 0)   # the persistent kernel only when clearly faster
    x = torch.as_tensor(inputs.random_field((n, n, n), 10).reshape(-1), dtype=torch.float32, device="cuda")
    mask = np.array([0, 0, 0, 1, 1, 0, 1, 1, 1], np.uint8)
    ys = []
    for on in (1 - xy, xy):
        ctx.set_xy_persistent(on)
        _, _, xy2, _ = ctx.autotune()
        assert xy2 == on                          # the explicit choice stays
        y = torch.empty_like(x)
        ctx.matvec(x, y, mask)
        ys.append(y)
    assert torch.equal(ys[0], ys[1])
