#!/usr/bin/env python
"""Writes the oracle's expected values for the parity tests that run the
workloads at their own sizes (the JSON files beside this script).

Every number written here comes from the CPU oracle (``oracle/``) run on the
seeded inputs of ``paper_1901_06531_gb300/inputs.py``; nothing is read from
the CUDA path.  The oracle solves each load history in FP64 at Newton
tolerance 1e-10 and CG tolerance 1e-12 (tight enough that its own stopping
error is far below every tolerance the tests assert), step by step, and the
file is rewritten after every step so that an interrupted run still leaves
the steps it finished.  The 64^3 mixed-control workload is the exception:
with only F11 prescribed, a rigid rotation about e1 is an exact null mode of
the linearised problem (zero curvature), and plain CG driven to 1e-12 picks
up rounding along it until p.Ap turns negative (the oracle broke down at
iteration 108 of the first solve); its CG tolerance is the 1e-10 of the
workload's own runs, which stops before that happens.

Recorded per step: <F> and <P> (Sec. 2.2: the null-frequency coefficients),
the Newton and CG iteration counts; at selected steps the full F and P at a
seeded sample of voxels plus the voxels where F departs most from <F> (the
oracle computes every voxel, so any sample is an exact expected value).

Workloads (Sec. 3 stand-ins; the recipes are those of the bench and tests):
  c2_spheres64  64^3 random non-overlapping spheres r = 4 at 25 % (seed
                1002), neo-Hookean (1, 2) / (10, 20); F11 -> 1.05 in 10
                steps, the other eight components stress free (Sec. 2.3 mixed
                control)
  c3_poly128    128^3 200-grain Voronoi (seed 1003), SVK cubic 168/121/75
                GPa rotated per grain (seed 1004); cyclic P11 +-0.2 GPa in 20
                steps with F12 = F13 = F23 = 0 prescribed
  c4_cell48, c4_cell96
                single cells of the batched recipe (batch_of_cells(1, 5,
                sizes=(n,), nsteps=2)): sphere particles, neo-Hookean
                contrast U(5, 50), random mixed control
  c5_adjoint128 128^3 two-phase neo-Hookean (RSA spheres r = 10, vf 0.2,
                seed 1005, contrast 10) with a lognormal voxel scale (sigma
                0.3, seed 1006); one step P11 = 0.05 with the rotation fixed;
                the adjoint gradient of J = <F>_11 (oracle.adjoint)

Usage: python tests/golden/make_goldens.py NAME [--steps K]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import adjoint as oadj, materials as omat, solver as osolver  # noqa: E402
from paper_1901_06531_gb300 import inputs  # noqa: E402

TOL_NEWTON, TOL_CG = 1e-10, 1e-12
SAMPLE_SEED = 20190118
N_RANDOM, N_EXTREME = 48, 16


def c2():
    n = 64
    ph, _ = inputs.rsa_spheres((n, n, n), 4.0, 0.25, 1002)
    params = np.array([[1.0, 2.0], [10.0, 20.0]])
    mask, target = inputs.history_mixed_strain11(10, 1.05)
    return omat.Material(ph, omat.NEOHOOKE, params), mask, target, [1, 5, 10]


# CG tolerance per workload where it differs from TOL_CG (see the module note)
TOL_CG_OF = {"c2_spheres64": 1e-10}


def c3():
    n = 128
    g, _ = inputs.voronoi((n, n, n), 200, 1003)
    R = inputs.random_rotations(200, 1004)
    params = np.tile([168.0, 121.0, 75.0], (200, 1))
    mask, target = inputs.fix_rotation(*inputs.history_cyclic_stress(20, 0.2))
    return omat.Material(g, omat.SVK_CUBIC, params, R), mask, target, [1, 2, 5, 10, 15, 20]


def c4(n):
    cell = inputs.batch_of_cells(1, 5, sizes=(n,), nsteps=2)[0]
    return omat.Material(cell["phase"], omat.NEOHOOKE, cell["params"]), cell["mask"], cell["target"], [1, 2]


def c5():
    n = 128
    shape = (n, n, n)
    ph, _ = inputs.rsa_spheres(shape, 10.0, 0.2, 1005)
    sc = inputs.lognormal_scale(shape, 0.3, 1006)
    params = np.array([[1.0, 2.0], [10.0, 20.0]])
    mask, target = inputs.fix_rotation(*inputs.history_uniaxial_stress_ramp(1, 0.05))
    return omat.Material(ph, omat.NEOHOOKE, params, scale=sc), mask, target, [1]


WORKLOADS = {"c2_spheres64": c2, "c3_poly128": c3, "c4_cell48": lambda: c4(48),
             "c4_cell96": lambda: c4(96), "c5_adjoint128": c5}


def sample_voxels(F, rng_idx):
    """The seeded random voxels plus the N_EXTREME voxels where |F - <F>| is
    largest (flat indices into [z, y, x])."""
    dev = np.sqrt(np.sum((F - osolver.mean9(F)[:, None, None, None]) ** 2, axis=0)).ravel()
    ext = np.argsort(dev)[::-1][:N_EXTREME]
    idx = np.concatenate([rng_idx, ext[~np.isin(ext, rng_idx)]])
    return idx.astype(np.int64)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("name", choices=sorted(WORKLOADS))
    ap.add_argument("--steps", type=int, default=0, help="load steps to solve (0: all)")
    args = ap.parse_args()
    material, mask, target, record = WORKLOADS[args.name]()
    nsteps = mask.shape[0] if args.steps <= 0 else min(args.steps, mask.shape[0])
    shape = material.phase.shape
    N = int(np.prod(shape))
    rng_idx = np.random.default_rng(SAMPLE_SEED).choice(N, N_RANDOM, replace=False)
    tol_cg = TOL_CG_OF.get(args.name, TOL_CG)
    out = {"workload": args.name, "shape_zyx": list(shape), "tol_newton": TOL_NEWTON, "tol_cg": tol_cg,
           "source": "oracle/ (FP64, DFT by definition), written by tests/golden/make_goldens.py",
           "mask": mask[:nsteps].tolist(), "target": target[:nsteps].tolist(),
           "Fbar": [], "Pbar": [], "newton": [], "cg": [], "samples": {}, "seconds": []}
    path = os.path.join(HERE, args.name + ".json")
    F = None
    for k in range(nsteps):
        t0 = time.perf_counter()
        o = osolver.solve(material, mask[k:k + 1], target[k:k + 1], TOL_NEWTON, tol_cg,
                          max_newton=50, max_cg=20000, F0=F)
        F = o["F"]
        out["Fbar"].append(o["Fbar"][0].tolist())
        out["Pbar"].append(o["Pbar"][0].tolist())
        out["newton"].append(int(o["newton"][0]))
        out["cg"].append(int(o["cg"][0]))
        out["seconds"].append(time.perf_counter() - t0)
        if (k + 1) in record or k + 1 == nsteps:
            idx = sample_voxels(F, rng_idx)
            Ff = F.reshape(9, -1)
            Pf = o["P"].reshape(9, -1)
            out["samples"][str(k + 1)] = {"index": idx.tolist(), "F": Ff[:, idx].T.tolist(),
                                          "P": Pf[:, idx].T.tolist()}
        if args.name == "c5_adjoint128":
            wF = np.zeros(9)
            wF[0] = 1.0
            wP = np.zeros(9)
            grad, dscale = oadj.gradient(material, F, mask[k], wF, wP, tol_cg=1e-12)
            idx = np.asarray(out["samples"][str(k + 1)]["index"])
            out["adjoint"] = {"wF": wF.tolist(), "wP": wP.tolist(),
                              "J": oadj.response(material, F, wF, wP),
                              "dJ_dmu_lam": grad.tolist(), "dJ_dscale_sample": dscale.ravel()[idx].tolist(),
                              "dJ_dscale_sum": float(dscale.sum()),
                              "dJ_dscale_absmax": float(np.max(np.abs(dscale)))}
        out["steps_done"] = k + 1
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(out, f, separators=(",", ":"))
        os.replace(tmp, path)
        print(f"{args.name}: step {k + 1}/{nsteps} newton {out['newton'][-1]} cg {out['cg'][-1]} "
              f"{out['seconds'][-1]:.0f} s", flush=True)


if __name__ == "__main__":
    main()
