"""The trace build (MF_TRACE: a one-thread kernel between the phases of a
load history's graph records the device's global timer and the phase id).
A short FP32-inner history with the quadratic predictor on the trace build
gives results bit-identical to the release build's (the marks change no
arithmetic), and its marks are consistent with the iteration counts: one
step start and one step end per load step, one iteration start per Newton
iteration, non-decreasing times.  The trace library is loaded in a child
process (the release library is already loaded here)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1901_06531_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, ROOT)
import numpy as np
from paper_1901_06531_gb300 import mixfft as mf, inputs
n = 16
ph = (inputs.voronoi((n, n, n), 6, 11)[0] % 2).astype(np.int32)
params = np.array([[1.0, 2.0], [10.0, 20.0]])
m, t = inputs.fix_rotation(*inputs.history_uniaxial_stress_ramp(5, 0.02))
out = {}
ctx = mf.Context(n, n, n, mf.MF_FP32_INNER)
ctx.set_material(mf.MF_NEOHOOKE, params, ph)
ctx.set_predictor(mf.MF_PRED_QUADRATIC)
ctx.set_F(None)
try:
    mf.trace_read()
    out["release"] = False
except Exception:
    out["release"] = True
o = ctx.solve(m, t, 1e-9, 1e-12, cg_rel=1e-4, max_cg=5000)
out["Fbar"] = np.asarray(o["Fbar"]).tolist()
out["Pbar"] = np.asarray(o["Pbar"]).tolist()
out["newton"] = [int(x) for x in o["newton"]]
if not out["release"]:
    tt, ids = mf.trace_read()
    out["t"] = [int(x) for x in tt]
    out["ids"] = [int(x) for x in ids]
print(json.dumps(out))
"""


def run_child(env_lib):
    env = dict(os.environ)
    env.pop("MF_LIBRARY", None)
    if env_lib:
        env["MF_LIBRARY"] = env_lib
    res = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], capture_output=True,
                         text=True, env=env, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    return json.loads(res.stdout.strip().splitlines()[-1])


def test_trace_build_marks_and_results():
    assert os.path.exists(build.build(trace=True))
    tr = run_child("trace")
    rel = run_child(None)
    assert rel["release"] and not tr["release"]
    # the marks change no arithmetic
    assert tr["Fbar"] == rel["Fbar"] and tr["Pbar"] == rel["Pbar"] and tr["newton"] == rel["newton"]
    t, ids = np.array(tr["t"], dtype=np.int64), np.array(tr["ids"])
    nsteps = len(tr["newton"])
    assert np.all(np.diff(t) >= 0)
    assert int(np.sum(ids == 1)) == nsteps and int(np.sum(ids == 31)) == nsteps
    assert int(np.sum(ids == 10)) == sum(tr["newton"])
    assert int(np.sum(ids == 13)) == sum(tr["newton"])   # one CG loop per Newton iteration
    sys.path.insert(0, ROOT)
    import bench
    from paper_1901_06531_gb300 import mixfft as mf
    comp, totals = bench.phase_composition(t, ids, mf.TRACE_PHASES, skip_steps=0)
    assert len(totals) == nsteps and all(x > 0 for x in totals)
    assert comp["cg_loop"] > 0 and comp["first_residual"] > 0
