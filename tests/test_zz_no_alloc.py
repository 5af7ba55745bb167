"""mf_residual_noalloc: the residual for callers that cannot allocate device
memory when they need it (host callbacks, allocator hooks, runtimes with a
fixed device budget).  It keeps its spectrum, tables and partials in the
library's static device scratch; its output must equal that of the context-
based mf_residual, call after call.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1901_06531_gb300 import inputs

from gpu_util import lib, neohooke_two_phase, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(32, 24, 16), (64, 64, 64)])
def test_noalloc_residual_matches_context_residual_twice(shape):
    import torch
    mf = lib()
    nx, ny, nz = shape
    N = nx * ny * nz
    ph, params = neohooke_two_phase((nz, ny, nx), 3)
    ctx = mf.Context(nx, ny, nz, mf.MF_FP64)
    ctx.set_material(mf.MF_NEOHOOKE, params, ph)
    ctx.set_F(inputs.random_F((nz, ny, nx), 4, 0.05))
    ctx.constitutive()
    _, P = ctx.get_fields()
    Pd = torch.as_tensor(P.reshape(-1), device="cuda")
    cases = [(np.array([0, 0, 0, 1, 1, 0, 1, 1, 1], np.uint8), np.array([0, 0, 0, 0.02, 0.01, 0, 0, 0, -0.03])),
             (np.ones(9, np.uint8), np.array([0.05, 0.01, 0, 0.01, 0, 0, 0, 0, 0]))]
    for call, (mask, pbar) in enumerate(cases):   # two calls in a row, different controls
        b_ref = torch.empty(9 * N, dtype=torch.float64, device="cuda")
        mean_ref = ctx.residual(mask, pbar, b_ref)
        b = torch.full((9 * N,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        mean = mf.residual_noalloc(nx, ny, nz, Pd, mask, pbar, b)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        if call > 0:
            # the first call has loaded the kernels and looked up the scratch
            # address; from then on a call takes no device memory at all
            assert free_after == free_before, (free_before, free_after)
        assert rel(b.cpu().numpy(), b_ref.cpu().numpy()) < 1e-12
        np.testing.assert_allclose(mean, mean_ref, rtol=0, atol=1e-14)


def test_noalloc_rejects_cells_beyond_its_scratch():
    import torch
    mf = lib()
    P = torch.zeros(9 * 96 * 96 * 32, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(P)
    with pytest.raises(mf.MixFFTError) as e:
        mf.residual_noalloc(96, 96, 32, P, np.ones(9, np.uint8), np.zeros(9), b)
    assert e.value.status == mf.MF_TOO_LARGE
