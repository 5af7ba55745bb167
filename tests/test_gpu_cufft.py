"""The cuFFT comparison path (timing baseline only) computes the same
projected operator as the library's own transforms."""
import numpy as np
import pytest

from paper_1901_06531_gb300 import inputs

from gpu_util import lib, neohooke_two_phase, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(16, 16, 16), (32, 32, 32), (48, 36, 18), (64, 64, 16)])
@pytest.mark.parametrize("prec", [0, 1])
def test_cufft_path_matches_library_transforms(shape, prec):
    import torch
    mf = lib()
    nx, ny, nz = shape
    ph, params = neohooke_two_phase((nz, ny, nx), 21)
    ctx = mf.Context(nx, ny, nz, prec)
    ctx.set_material(mf.MF_NEOHOOKE, params, ph)
    ctx.set_F(inputs.random_F((nz, ny, nx), 22, 0.05))
    ctx.constitutive()
    ctx.cufft_bind()
    dt = torch.float32 if prec else torch.float64
    x = torch.as_tensor(inputs.random_field((nz, ny, nx), 23).reshape(-1), dtype=dt, device="cuda")
    mask = np.array([0, 0, 0, 1, 1, 0, 1, 1, 1], np.uint8)
    y1 = torch.empty_like(x)
    y2 = torch.empty_like(x)
    ctx.matvec(x, y1, mask)
    ctx.matvec_cufft(x, y2, mask)
    a, b = y1.double().cpu().numpy(), y2.double().cpu().numpy()
    if prec:
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 2e-6
    else:
        assert rel(a, b) < 1e-12
    ms = ctx.time_cufft(mask, reps=2)
    assert np.all(ms > 0)
