"""The debug build (MF_DEBUG: every shared- and global-memory index of the
transform, tangent and pointwise kernels checked against its buffer, a
failure recorded and the access redirected in bounds) on small odd and even
grids: the operator, the residual and short solves in both precisions match
the oracle as in the release tests, and no check fails.  The debug library
is loaded in a child process (the release library is already loaded here)."""
import json
import os
import subprocess
import sys

import pytest

from paper_1901_06531_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, ROOT)
import numpy as np, torch
from paper_1901_06531_gb300 import mixfft as mf, inputs
from oracle import materials as omat, solver as osolver
out = {"selftest": None, "cases": []}
# the mechanism itself: one recorded failure with its index and extent
st = mf.debug_selftest()
out["selftest"] = [st, list(mf.debug_report())]
rel = lambda a, b: float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b))))
mask = np.array([0, 0, 0, 1, 1, 0, 1, 1, 1], np.uint8)
for (nx, ny, nz) in [(4, 4, 2), (4, 4, 3), (6, 4, 3), (6, 6, 6), (8, 6, 4), (8, 8, 8), (16, 16, 16), (16, 16, 3)]:
    shape = (nz, ny, nx)
    ph = np.random.default_rng(nx * 100 + ny * 10 + nz).integers(0, 2, shape).astype(np.int32)
    params = np.array([[1.0, 2.0], [10.0, 20.0]])
    om = omat.Material(ph, omat.NEOHOOKE, params)
    F = inputs.random_F(shape, 3, 0.05)
    P, K = om.PK(F)
    case = {"shape": [nx, ny, nz]}
    for prec in (mf.MF_FP64, mf.MF_FP32_INNER):
        ctx = mf.Context(nx, ny, nz, prec)
        ctx.set_material(mf.MF_NEOHOOKE, params, ph)
        ctx.set_F(F)
        ctx.constitutive()
        x = inputs.random_field(shape, 4)
        dt = torch.float64 if prec == mf.MF_FP64 else torch.float32
        xt = torch.as_tensor(x.reshape(-1), dtype=dt, device="cuda")
        yt = torch.empty_like(xt)
        ctx.matvec(xt, yt, mask)
        xin = x if prec == mf.MF_FP64 else x.astype(np.float32).astype(np.float64)
        ref = osolver.matvec(K, xin, mask)
        case["matvec_%d" % prec] = rel(yt.cpu().numpy().astype(np.float64).reshape(ref.shape), ref)
        b = torch.empty(9 * nx * ny * nz, dtype=torch.float64, device="cuda")
        pbar = np.array([0, 0, 0, 0.01, 0.02, 0, 0.0, 0.0, -0.01])
        ctx.residual(mask, pbar, b)
        refb = osolver.residual(P, mask, pbar)
        case["residual_%d" % prec] = rel(b.cpu().numpy().reshape(refb.shape), refb)
        m, t = inputs.fix_rotation(*inputs.history_uniaxial_stress_ramp(3, 0.05))
        ctx.set_predictor(mf.MF_PRED_EXTRAPOLATE)
        ctx.set_F(None)
        o = ctx.solve(m, t, 1e-10, 1e-12, cg_rel=1e-4, max_cg=5000)
        r = osolver.solve(om, m, t, 1e-10, 1e-12)
        case["solve_Fbar_%d" % prec] = rel(o["Fbar"], r["Fbar"])
    case["report"] = list(mf.debug_report())
    out["cases"].append(case)
print(json.dumps(out))
"""


def test_debug_build_on_small_grids():
    lib = build.build(debug=True)
    assert os.path.exists(lib)
    env = dict(os.environ, MF_LIBRARY="debug")
    res = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], capture_output=True,
                         text=True, env=env, timeout=1500)
    assert res.returncode == 0, res.stderr[-3000:]
    out = json.loads(res.stdout.strip().splitlines()[-1])
    print(json.dumps(out))
    st, rep = out["selftest"]
    assert st == 0 and rep[0] == 1 and rep[2] == 7 and rep[3] == 4, out["selftest"]
    for c in out["cases"]:
        assert c["report"][0] == 0, c          # no bounds check failed
        assert c["matvec_0"] < 1e-12 and c["residual_0"] < 1e-12, c
        assert c["matvec_1"] < 1e-5 and c["residual_1"] < 1e-12, c
        assert c["solve_Fbar_0"] < 1e-10 and c["solve_Fbar_1"] < 1e-9, c


def test_release_build_reports_no_checks():
    from paper_1901_06531_gb300 import mixfft as mf
    if os.environ.get("MF_LIBRARY") == "debug":
        pytest.skip("the debug library is loaded")
    assert mf.debug_report()[0] == -1
    assert mf.debug_selftest() == mf.MF_INVALID_ARG
