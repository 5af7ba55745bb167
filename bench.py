#!/usr/bin/env python
"""Benchmark: Newton load steps of Galerkin FFT homogenization under stress
control on a 128^3 polycrystal (arXiv:1901.06531, Sec. 2.2-2.3 and 4).

Workload (synthetic, seeded): 128^3 voxels, 200-grain periodic Voronoi
tessellation, St Venant-Kirchhoff cubic stiffness C11=168, C12=121, C44=75 GPa
rotated by uniform random orientations per grain; cyclic stress control
P11 = 0 -> +0.2 -> -0.2 -> 0 GPa in 20 steps, other P-bar components 0, with
F12 = F13 = F23 = 0 prescribed to fix the rigid rotation (the paper's load
case (1) pattern).  Solver: FP32 inner CG / FP64 outer Newton, Newton tol
1e-8, CG tol 1e-10 (FP64 floor) with a 1e-4 relative forcing term.

A step is one load increment: predictor, Newton iterations (constitutive
update, FP64 residual, CG on the projected operator, update) to convergence.
Prints one JSON line.  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N1 = 128
NGRAINS = 200
SEED = 1003
TOL_NEWTON, TOL_CG, CG_REL = 1e-8, 1e-10, 1e-4
WORKLOAD = ("polycrystal 128^3, 200-grain Voronoi, SVK cubic (168/121/75 GPa) rotated per grain, "
            "cyclic stress P11 +-0.2 GPa in 20 steps (F12=F13=F23=0), FP32 inner CG / double-word outer "
            "(averages, control and Newton update in FP64), Newton start interpolated quadratically from the "
            "last three converged states")
METRIC = ("Newton load steps/s at 128^3 (FP32-inner CG / double-word outer), polycrystal cyclic stress "
          "control")
# algorithmic bytes per voxel of each kernel of one CG iteration.  FP32 (matrix-
# free tangent): the tangent pass reads r, p', x, H = F - I (9 x 4 B each) and
# the phase id (4 B) and writes p, x, t; the x-y forward reads t and writes the
# half spectrum (9 x 0.5 x 8 B); the z-pass reads and writes the spectrum; the
# x-y inverse reads the spectrum and r and writes r.  FP64 (packed tangent):
# the tangent pass reads r, p', x (9 x 8 B each) and K (45 x 8 B), writes p, x, t.
KERNELS = ["tangent_cg", "xy_forward", "zpass_projection", "xy_inverse_residual"]
ALGO_BYTES_F32 = [4 * 36 + 4 + 3 * 36, 36 + 36, 36 + 36, 3 * 36]
ALGO_BYTES_F64 = [3 * 72 + 360 + 3 * 72, 72 + 72, 72 + 72, 3 * 72]
# one projected-operator application y = G*(K:x), FP32 with the matrix-free
# tangent: K:x (x, H, phase in; t out), x-y forward, z-pass, x-y inverse
MATVEC_BYTES_F32 = (36 + 36 + 4 + 36) + 72 + 72 + 72
# flops per voxel of one FP64 operator application: forward and inverse 3D
# transforms of the nine components (2.5 log2(N) flops per real point each
# at 128^3: 945), the packed tangent apply (162), G-hat-star (about 30)
MATVEC_FLOP_F64 = 1140


def workload(n=N1, ngrains=NGRAINS, seed=SEED):
    from paper_1901_06531_gb300 import inputs
    g, _ = inputs.voronoi((n, n, n), ngrains, seed)
    R = inputs.random_rotations(ngrains, seed + 1)
    params = np.tile([168.0, 121.0, 75.0], (ngrains, 1))
    mask, target = inputs.fix_rotation(*inputs.history_cyclic_stress(20, 0.2))
    return g, params, R, mask, target


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# source files each timed kernel is compiled from
KERNEL_SOURCES = {
    "tangent_cg": ("cg.cu", "common.cuh", "launch.h"),
    "xy_forward": ("transform2.cuh", "transform2c.cuh", "transform2_impl.cuh", "fft2.cuh", "common.cuh", "dw.cuh",
                   "launch.h"),
    "zpass_projection": ("transform2.cuh", "transform2_impl.cuh", "fft2.cuh", "common.cuh", "dw.cuh", "launch.h"),
    "xy_inverse_residual": ("transform2.cuh", "transform2c.cuh", "transform2_impl.cuh", "fft2.cuh", "common.cuh",
                            "dw.cuh", "launch.h"),
}
XY_SCHEDULES = {0: "one block per plane", 1: "persistent bulk-copy", 2: "two-CTA cluster"}


def src_hash(kernel):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1901_06531_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary (its ```json
    block), if it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "cg_kernels_polycrystal128_fp32inner.md")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        text = f.read()
    try:
        block = text.split("```json", 1)[1].split("```", 1)[0]
        d = json.loads(block)
    except (IndexError, ValueError):
        return None
    e = d.get(kernel)
    if not e or e.get("source_sha") != src_hash(kernel):
        return None
    return e.get("bytes_per_launch")


def replica_throughput(total_ms, steps, dist=None, device="cpu"):
    """Replicas (one independent cell per rank, no data-path collective): the
    job's time is the slowest rank's, its throughput all ranks' load steps
    over that time.  Returns (max_ms, load steps/s)."""
    world = 1
    if dist is not None:
        import torch
        world = dist.get_world_size()
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * steps / (total_ms / 1e3)


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        finally:
            os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
ORACLE_SAMPLE = r"""
import json, os, sys, time
import numpy as np
sys.path.insert(0, {root!r})
import bench
from oracle import materials as omat, solver as osolver
g, params, R, mask, target = bench.workload()
n = g.shape[0]
m0, t0 = mask[0], target[0]
pbar = np.where(m0 == 1, t0, 0.0)
n_newton, n_cg, counts = {n_newton}, {n_cg}, {counts!r}
if n_newton <= 0:
    # iteration counts of the first load step, from the oracle on the same recipe at 16^3
    gs, ps, Rs, _, _ = bench.workload(16, 12, {seed})
    os_ = osolver.solve(omat.Material(gs, omat.SVK_CUBIC, ps, Rs), mask[:1], target[:1], {tn}, {tc})
    n_newton, n_cg = int(os_["newton"][0]), int(os_["cg"][0])
# constitutive update on a 16-plane slab at the predictor state, scaled to the cell
slab = 16
F = np.zeros((9, slab) + g.shape[1:]); F[0] = F[4] = F[8] = 1.0
F[0] += 2e-4
t = time.perf_counter()
P_s, K_s = omat.Material(g[:slab], omat.SVK_CUBIC, params, R).PK(F)
t_pk = (time.perf_counter() - t) * (n / slab)
P = np.tile(P_s, (1, n // slab, 1, 1))
K = np.tile(K_s, (1, 1, n // slab, 1, 1))
t = time.perf_counter(); b = osolver.residual(P, m0, pbar); t_res = time.perf_counter() - t
t_mv = []
for _ in range({nmv}):
    t = time.perf_counter(); y = osolver.matvec(K, b, m0); t_mv.append(time.perf_counter() - t)
est = [(n_newton + 1) * t_pk + n_newton * t_res + n_cg * tm for tm in t_mv]
print(json.dumps(dict(t_pk=t_pk, t_res=t_res, t_mv=t_mv, n_newton=n_newton, n_cg=n_cg, counts=counts, est=est)))
"""

# A full oracle run of a whole load history, timed as it stands (no sampling).
ORACLE_FULL = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, {root!r})
from oracle import materials as omat, solver as osolver
from paper_1901_06531_gb300 import inputs
name = {name!r}
if name == "c1_sphere16":
    ph = inputs.centred_sphere(16, 0.25)
    m = omat.Material(ph, omat.NEOHOOKE, np.array([[1.0, 2.0], [10.0, 20.0]]))
    mask, target = inputs.history_uniaxial_stress_ramp(5, 0.1)
else:
    ph, _ = inputs.rsa_spheres((64, 64, 64), 4.0, 0.25, 1002)
    m = omat.Material(ph, omat.NEOHOOKE, np.array([[1.0, 2.0], [10.0, 20.0]]))
    mask, target = inputs.history_mixed_strain11(10, 1.05)
nsteps = {nsteps} if {nsteps} > 0 else mask.shape[0]
t = time.perf_counter()
o = osolver.solve(m, mask[:nsteps], target[:nsteps], {tn}, {tc})
wall = time.perf_counter() - t
print(json.dumps(dict(name=name, steps=nsteps, seconds=wall, newton=o["newton"].tolist(), cg=o["cg"].tolist())))
"""


def _oracle_env(cores):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    return env


def oracle_sample(cores, nmv=1, n_newton=0, n_cg=0, counts="oracle 16^3"):
    """128^3 oracle components (constitutive pass, residual, nmv operator
    applications) timed on `cores` threads, and a load step modelled from them
    with the given iteration counts (0: the oracle's own first step at 16^3)."""
    code = ORACLE_SAMPLE.format(root=ROOT, seed=SEED, tn=TOL_NEWTON, tc=TOL_CG, nmv=nmv, n_newton=int(n_newton),
                                n_cg=int(n_cg), counts=counts)
    t = time.perf_counter()
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=_oracle_env(cores),
                         timeout=1800)
    wall = time.perf_counter() - t
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    d = json.loads(out.stdout.strip().splitlines()[-1])
    d["wall"] = wall
    return d


def oracle_full(name, cores, nsteps=0):
    """A whole oracle load history, timed as it runs (seconds, iterations)."""
    code = ORACLE_FULL.format(root=ROOT, name=name, nsteps=int(nsteps), tn=TOL_NEWTON, tc=TOL_CG)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=_oracle_env(cores),
                         timeout=7200)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    d = json.loads(out.stdout.strip().splitlines()[-1])
    d["threads"] = cores
    d["load_steps_per_s"] = d["steps"] / d["seconds"]
    return d


def cpu_baseline_entry(d, cores):
    return {"value": 1.0 / float(np.mean(d["est"])), "unit": "load steps/s", "cores": cores,
            "kind": "oracle-model",
            "sample": (f"128^3 oracle (FP64, DFT by definition), measured on {cores} threads: constitutive "
                       f"pass on a 16-plane slab x8 ({d['t_pk']:.1f} s), one residual ({d['t_res']:.1f} s), "
                       f"projected operator ({np.mean(d['t_mv']):.1f} s each, {len(d['t_mv'])} runs); "
                       f"load step MODELLED as (n_newton+1) constitutive + n_newton residuals + n_cg "
                       f"operators with n_newton={d['n_newton']}, n_cg={d['n_cg']} ({d['counts']}); "
                       f"{d['wall']:.0f} s of CPU work")}


def run_oracle_full(args):
    """`--oracle-full`: whole oracle runs at the bench's tolerances of the
    16^3 workload (five load steps) on one thread and on every core, and of
    the 64^3 workload (ten steps) on every core and its first two steps on
    one thread; one JSON line."""
    cores = os.cpu_count() or 1
    res = {"nproc": cores, "runs": []}
    for name, threads, nsteps in (("c1_sphere16", 1, 0), ("c1_sphere16", cores, 0),
                                  ("c2_spheres64", cores, 0), ("c2_spheres64", 1, 2)):
        res["runs"].append(oracle_full(name, threads, nsteps))
        print(json.dumps(res["runs"][-1]), file=sys.stderr, flush=True)
    print(json.dumps(res))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    d = oracle_sample(cores, nmv=args.warmup + args.steps)
    d["est"] = d["est"][args.warmup:]
    d["t_mv"] = d["t_mv"][args.warmup:]
    est = float(np.mean(d["est"]))
    value = 1.0 / est
    line = {"metric": METRIC, "value": value, "unit": "load steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": est * 1e3,
            "ms_per_step_kind": ("modelled load step (see cpu_baseline.sample); each timed step of this run is "
                                 "one measured 128^3 oracle operator application"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD + " [CPU oracle, modelled from measured components]"},
            "cpu_baseline": cpu_baseline_entry(d, cores),
            "e2e": {"value": value, "unit": "load steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    line["cpu_baseline"]["value"] = value
    print(json.dumps(line))


# ---------------------------------------------------------------- GPU path
def time_residual(ctx, mask, pbar, b, reps):
    """Median ms of one FP64 residual (three transform kernels), L2 flushed
    before each; a 151 MB memset of b does the flush."""
    import torch
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        b.zero_()
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.residual(mask, pbar, b)
        e.record(stream)
        ts.append((a, e))
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(e) for a, e in ts]))


def run_matvec_only(args):
    """Profiling driver: the 128^3 polycrystal tangent at the first load step,
    then `--matvec-only` applications of the FP32 (or FP64) projected operator,
    or (`--kernels-only R`) R L2-flushed launches of each CG-iteration kernel."""
    import torch
    from paper_1901_06531_gb300 import build
    build.build()
    from paper_1901_06531_gb300 import mixfft as mf
    g, params, R, mask, target = workload()
    n = N1
    prec = mf.MF_FP64 if args.fp64 else mf.MF_FP32_INNER
    ctx = mf.Context(n, n, n, prec)
    ctx.set_material(mf.MF_SVK_CUBIC, params, g, rot=R)
    if args.fp64 or args.xy_cluster < 0:
        ctx.autotune()
    else:
        ctx.set_xy_cluster(args.xy_cluster)
    ctx.constitutive()
    if args.kernels_only:
        ms = ctx.time_kernels(mask[0], reps=args.kernels_only)
        ms_graph = ctx.time_kernels(mask[0], reps=args.kernels_only, graph=True)
        b = torch.empty(9 * n ** 3, dtype=torch.float64, device="cuda")
        res_ms = time_residual(ctx, mask[0], target[0] * mask[0], b, args.kernels_only)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        ctx.stress()
        ev[1].record()
        torch.cuda.synchronize()
        fwd, inv, _ = ctx.xy_schedule()
        print(json.dumps({"kernels_only": args.kernels_only, "fp64": bool(args.fp64),
                          "xy_schedule": {"forward": XY_SCHEDULES[fwd], "inverse": XY_SCHEDULES[inv]},
                          "ms": dict(zip(KERNELS, [float(m) for m in ms])),
                          "ms_graph": dict(zip(KERNELS, [float(m) for m in ms_graph])),
                          "frac_graph": {k: b * n ** 3 / (m * 1e-3) / 1e9 / measured_peaks()[0]
                                         for k, m, b in zip(KERNELS, ms_graph, ALGO_BYTES_F64 if args.fp64
                                                            else ALGO_BYTES_F32)},
                          "residual_ms": res_ms,
                          "stress_ms": ev[0].elapsed_time(ev[1])}))
        return
    x = torch.randn(9 * n ** 3, dtype=ctx.inner_dtype, device="cuda")
    y = torch.empty_like(x)
    for _ in range(args.matvec_only):
        ctx.matvec(x, y, mask[0])
    torch.cuda.synchronize()
    print(json.dumps({"matvec_only": args.matvec_only, "fp64": bool(args.fp64),
                      "y_norm": float(y.double().norm())}))


BATCH_CELLS, BATCH_SEED, BATCH_STEPS = 48, 1004, 4


def run_batched(args):
    """The batched workload: 48 sphere-particle cells with sizes drawn from
    {32, 48, 64, 96}^3, random mixed control, FP32 inner / FP64 outer, all
    solved at once (mf_solve_batch, one stream per cell), against the same
    cells solved one after another."""
    import torch
    from paper_1901_06531_gb300 import inputs
    from paper_1901_06531_gb300 import mixfft as mf
    cells = inputs.batch_of_cells(BATCH_CELLS, BATCH_SEED, nsteps=BATCH_STEPS)
    ctxs = []
    for cell in cells:
        n = cell["n"]
        c = mf.Context(n, n, n, mf.MF_FP32_INNER, stream=torch.cuda.Stream())
        c.set_material(mf.MF_NEOHOOKE, cell["params"], cell["phase"])
        c.set_predictor(mf.MF_PRED_QUADRATIC)
        ctxs.append(c)
    masks = np.stack([cell["mask"] for cell in cells])
    targets = np.stack([cell["target"] for cell in cells])
    voxels = sum(cell["n"] ** 3 for cell in cells)
    # warm-up (graph instantiation, first touches), then from F = I again
    mf.solve_batch(ctxs, masks[:, :1], targets[:, :1], TOL_NEWTON, TOL_CG, CG_REL)
    for c in ctxs:
        c.set_F(None)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = mf.solve_batch(ctxs, masks, targets, TOL_NEWTON, TOL_CG, CG_REL)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    for c in ctxs:
        c.set_F(None)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, c in enumerate(ctxs):
        c.solve(masks[i], targets[i], TOL_NEWTON, TOL_CG, CG_REL)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    sizes = {}
    for cell in cells:
        sizes[str(cell["n"])] = sizes.get(str(cell["n"]), 0) + 1
    res = {"workload": (f"{BATCH_CELLS} sphere-particle neo-Hookean cells, sizes from {{32,48,64,96}}^3 "
                        f"(seed {BATCH_SEED}), vf U(0.1,0.3), contrast U(5,50), random mixed control, "
                        f"{BATCH_STEPS} load steps, FP32 inner / double-word outer, extrapolated (quadratic) Newton starts; "
                        "all cells one graph launch (mf_solve_batch)"),
           "cells_by_size": sizes, "voxels_total": voxels,
           "batch_s": t_batch, "sequential_s": t_seq,
           "cell_load_steps_per_s": BATCH_CELLS * BATCH_STEPS / t_batch,
           "gvoxel_load_steps_per_s": voxels * BATCH_STEPS / t_batch / 1e9,
           "speedup_vs_sequential": t_seq / t_batch,
           "newton_total": int(out["newton"].sum()), "cg_total": int(out["cg"].sum())}
    del ctxs
    torch.cuda.empty_cache()
    return res


CASES_N, CASES_SEED = 64, 1001


def run_paper_cases(args):
    """The paper's performance comparison (Sec. 4) on synthetic stand-ins at
    its own 64^3 size, FP32 inner: CG iterations per load increment (summed
    over the Newton iterations) for the control cases (1) mixed, (2) full
    stress, (3) full strain on the particle-reinforced cell (SVK, matrix
    mu = 28, k = 140/3, particles x10; lambda_end = 0.2 in 100 increments),
    and cases (1)-(4) on a 200-grain cubic SVK polycrystal (lambda_end = 0.02
    in 20 increments; (4) is the pseudo-uniaxial full strain control); wall
    time per case normalized by case (3)'s.  Plus the C2 workload (64^3
    random spheres r = 4 at 25 %, neo-Hookean contrast 10, F11 -> 1.05 in 10
    steps, the other eight components stress free): load-step time of the
    whole history in one call, FP64 (with and without the inexact-Newton
    forcing) and FP32 inner."""
    import torch
    from paper_1901_06531_gb300 import inputs
    from paper_1901_06531_gb300 import mixfft as mf
    n = CASES_N
    stream = torch.cuda.current_stream()

    def timed(ctx, m, t, **kw):
        ctx.set_F(None)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        o = ctx.solve(m, t, TOL_NEWTON, TOL_CG, CG_REL, **kw)
        b.record(stream)
        torch.cuda.synchronize()
        return o, a.elapsed_time(b)

    def run_case(ctx, m, t):
        try:
            o, ms = timed(ctx, m, t)
            return {"o": o, "ms": ms}
        except mf.MixFFTError as e:
            return {"error": str(e)}

    def summary(r, ref):
        if "error" in r:
            return {"status": r["error"]}
        o, ms = r["o"], r["ms"]
        d = {"ms": ms, "newton_total": int(o["newton"].sum()), "cg_total": int(o["cg"].sum()),
             "cg_per_step": o["cg"].tolist(), "newton_per_step": o["newton"].tolist()}
        if "o" in ref:
            d["time_vs_case3"] = ms / ref["ms"]
            d["cg_vs_case3"] = o["cg"].sum() / ref["o"]["cg"].sum()
        return d

    res = {}
    # particle-reinforced cell, cases (1)-(3)
    ph = inputs.particle_rve(n, CASES_SEED)
    mat = np.array([[84.0, 28.0, 28.0], [840.0, 280.0, 280.0]])
    ctx = mf.Context(n, n, n, mf.MF_FP32_INNER)
    ctx.set_material(mf.MF_SVK_CUBIC, mat, ph, rot=np.tile(np.eye(3), (2, 1, 1)))
    m1, t1 = inputs.history_case1(100, 0.2)
    timed(ctx, m1[:2], t1[:2])   # warm-up (tuner, graph capture)
    r1 = run_case(ctx, m1, t1)
    part = {"workload": f"{n}^3 four-particle cell (seed {CASES_SEED}, vf 0.2), SVK matrix 84/28/28, "
                        "particles x10, lambda_end 0.2 in 100 increments"}
    if "o" in r1:
        r2 = run_case(ctx, *inputs.history_case2(r1["o"]["Pbar"][-1], 100))
        r3 = run_case(ctx, *inputs.history_case3(r1["o"]["Fbar"][-1], 100))
        part.update({"case1": summary(r1, r3), "case2": summary(r2, r3), "case3": summary(r3, r3)})
    else:
        part["case1"] = summary(r1, {})
    res["particle"] = part
    del ctx
    # polycrystal, cases (1)-(4)
    g, _ = inputs.voronoi((n, n, n), 200, CASES_SEED + 1)
    R = inputs.random_rotations(200, CASES_SEED + 2)
    ctx = mf.Context(n, n, n, mf.MF_FP32_INNER)
    ctx.set_material(mf.MF_SVK_CUBIC, np.tile([168.0, 121.0, 75.0], (200, 1)), g, rot=R)
    m1, t1 = inputs.history_case1(20, 0.02)
    timed(ctx, m1[:2], t1[:2])
    r1 = run_case(ctx, m1, t1)
    poly = {"workload": f"{n}^3 200-grain Voronoi (seed {CASES_SEED + 1}), SVK cubic 168/121/75 GPa, "
                        "lambda_end 0.02 in 20 increments"}
    r4 = run_case(ctx, *inputs.history_case4(20, 0.02))
    if "o" in r1:
        r2 = run_case(ctx, *inputs.history_case2(r1["o"]["Pbar"][-1], 20))
        r3 = run_case(ctx, *inputs.history_case3(r1["o"]["Fbar"][-1], 20))
        poly.update({"case1": summary(r1, r3), "case2": summary(r2, r3), "case3": summary(r3, r3),
                     "case4": summary(r4, r3),
                     "case1_final_Pbar_diag": [float(r1["o"]["Pbar"][-1][i]) for i in (0, 4, 8)]})
    else:
        poly.update({"case1": summary(r1, {}), "case4": summary(r4, {})})
    if "o" in r4:
        poly["case4_final_Pbar_diag"] = [float(r4["o"]["Pbar"][-1][i]) for i in (0, 4, 8)]
    res["polycrystal"] = poly
    del ctx
    # C2: 64^3 random spheres, F11 ramp with eight stress-free components
    phs, _ = inputs.rsa_spheres((n, n, n), 4.0, 0.25, 1002)
    params = np.array([[1.0, 2.0], [10.0, 20.0]])
    mask, target = inputs.history_mixed_strain11(10, 1.05)
    c2 = {"workload": f"{n}^3 RSA spheres r=4 vf 0.25 (seed 1002), neo-Hookean contrast 10, "
                      "F11 -> 1.05 in 10 steps, other components stress free"}
    for name, prec, forcing, pred in (("fp32_inner", mf.MF_FP32_INNER, None, mf.MF_PRED_QUADRATIC),
                                      ("fp32_inner_uniform_predictor", mf.MF_FP32_INNER, None, mf.MF_PRED_UNIFORM),
                                      ("fp64", mf.MF_FP64, 0, mf.MF_PRED_UNIFORM),
                                      ("fp64_forcing", mf.MF_FP64, 1, mf.MF_PRED_QUADRATIC)):
        ctx = mf.Context(n, n, n, prec)
        ctx.set_material(mf.MF_NEOHOOKE, params, phs)
        ctx.set_predictor(pred)
        if forcing is not None:
            ctx.set_inexact_newton(forcing)
        try:
            timed(ctx, mask[:1], target[:1])
            o, ms = timed(ctx, mask, target)     # the whole history, one call
            its = [[int(a), int(b)] for a, b in zip(o["newton"], o["cg"])]
            c2[name] = {"load_step_ms": ms / mask.shape[0], "newton_cg_per_step": its,
                        "final_Pbar11": float(o["Pbar"][-1][0])}
        except mf.MixFFTError as e:
            c2[name] = {"status": str(e)}
        del ctx
    for name in ("fp64", "fp64_forcing"):
        if "load_step_ms" in c2[name] and "load_step_ms" in c2["fp32_inner"]:
            c2[name + "_over_fp32_inner"] = c2[name]["load_step_ms"] / c2["fp32_inner"]["load_step_ms"]
    res["c2"] = c2
    torch.cuda.empty_cache()
    return res


ADJ_N, ADJ_SEED = 128, 1005


def run_adjoint(args):
    """The adjoint workload: 128^3, two neo-Hookean phases (periodic RSA
    spheres of radius 10 voxels to volume fraction 0.2, contrast 10), voxel
    stiffness scale lognormal with sigma 0.3, one load step P11 = 0.05 with
    the other stresses zero and the rotation fixed (F12 = F13 = F23 = 0).
    Times the forward solve and the adjoint solve of d<F>_11 / d(mu, lam, s)
    in both precisions; then the same recipe at 256^3 (r = 20), FP32 inner,
    on the split row/column x-y kernels."""
    import torch
    from paper_1901_06531_gb300 import inputs
    from paper_1901_06531_gb300 import mixfft as mf
    n = ADJ_N
    shape = (n, n, n)
    ph, _ = inputs.rsa_spheres(shape, 10.0, 0.2, ADJ_SEED)
    sc = inputs.lognormal_scale(shape, 0.3, ADJ_SEED + 1)
    params = np.array([[1.0, 2.0], [10.0, 20.0]])
    mask, target = inputs.fix_rotation(*inputs.history_uniaxial_stress_ramp(1, 0.05))
    wF = np.zeros(9)
    wF[0] = 1.0
    wP = np.zeros(9)
    stream = torch.cuda.current_stream()
    res = {"workload": (f"{n}^3 two-phase neo-Hookean (RSA spheres r=10, vf 0.2, seed {ADJ_SEED}, contrast 10), "
                        f"lognormal voxel scale sigma 0.3, P11 = 0.05 rotation fixed; J = <F>_11; "
                        f"256^3: the same recipe with r=20")}
    for name, prec, kw, akw, reps in (
            ("fp32_inner", mf.MF_FP32_INNER, dict(tol_newton=TOL_NEWTON, tol_cg=TOL_CG, cg_rel=CG_REL),
             dict(tol_cg=1e-30, cg_rel=1e-6), 3),
            ("fp64", mf.MF_FP64, dict(tol_newton=TOL_NEWTON, tol_cg=TOL_CG, cg_rel=CG_REL),
             dict(tol_cg=1e-10, cg_rel=1e-8), 1)):
        ctx = mf.Context(n, n, n, prec)
        ctx.set_material(mf.MF_NEOHOOKE, params, ph, scale=sc)
        ds = torch.empty(ctx.N, dtype=torch.float64, device=ctx.device)
        ctx.solve(mask, target, **kw)
        ctx.adjoint(mask[0], wF, wP, dscale=ds, max_cg=20000, **akw)
        fwd, adj = [], []
        for _ in range(reps):
            ctx.set_F(None)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            o = ctx.solve(mask, target, **kw)
            e[1].record(stream)
            J, g, its = ctx.adjoint(mask[0], wF, wP, dscale=ds, max_cg=20000, **akw)
            e[2].record(stream)
            torch.cuda.synchronize()
            fwd.append(e[0].elapsed_time(e[1]))
            adj.append(e[1].elapsed_time(e[2]))
        res[name] = {"forward_ms": float(np.median(fwd)), "adjoint_ms": float(np.median(adj)),
                     "adjoint_over_forward": float(np.median(adj) / np.median(fwd)),
                     "forward_newton_cg": [int(o["newton"][0]), int(o["cg"][0])], "adjoint_cg": its,
                     "J": J, "dJ_dmu_lam": g.tolist(), "dJ_dscale_sum": float(ds.sum())}
        del ctx, ds
        torch.cuda.empty_cache()
    # 256^3 (split x-y kernels), FP32 inner: one forward step and its adjoint
    n2 = 2 * n
    ph2, _ = inputs.rsa_spheres((n2, n2, n2), 20.0, 0.2, ADJ_SEED)
    sc2 = inputs.lognormal_scale((n2, n2, n2), 0.3, ADJ_SEED + 1)
    ctx = mf.Context(n2, n2, n2, mf.MF_FP32_INNER)
    ctx.set_material(mf.MF_NEOHOOKE, params, ph2, scale=sc2)
    kw = dict(tol_newton=TOL_NEWTON, tol_cg=TOL_CG, cg_rel=CG_REL)
    akw = dict(tol_cg=1e-30, cg_rel=1e-6, max_cg=20000)
    ds = torch.empty(ctx.N, dtype=torch.float64, device=ctx.device)
    ctx.solve(mask, target, **kw)
    ctx.adjoint(mask[0], wF, wP, dscale=ds, **akw)
    ctx.set_F(None)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    o = ctx.solve(mask, target, **kw)
    e[1].record(stream)
    J, g, its = ctx.adjoint(mask[0], wF, wP, dscale=ds, **akw)
    e[2].record(stream)
    torch.cuda.synchronize()
    res["fp32_inner_256"] = {"forward_ms": e[0].elapsed_time(e[1]), "adjoint_ms": e[1].elapsed_time(e[2]),
                             "forward_newton_cg": [int(o["newton"][0]), int(o["cg"][0])], "adjoint_cg": its,
                             "J": J, "dJ_dmu_lam": g.tolist()}
    del ctx, ds
    torch.cuda.empty_cache()
    return res


def run_ours(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1901_06531_gb300 import build
    build.build()
    from paper_1901_06531_gb300 import mixfft as mf

    g, params, R, mask, target = workload()
    n = N1
    N = n ** 3
    nsteps_hist = mask.shape[0]
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ctx = mf.Context(n, n, n, mf.MF_FP32_INNER)
    ctx.set_material(mf.MF_SVK_CUBIC, params, g, rot=R)
    # each step starts from the quadratic through the last three converged
    # states (mf_set_predictor); the linear extrapolation and the paper's
    # uniform start are timed beside it below
    ctx.set_predictor(mf.MF_PRED_QUADRATIC)
    ztile, ztile_ms, _, _ = ctx.autotune()
    xy_fwd, xy_inv, xy_ms = ctx.xy_schedule()

    def steps(c, k0, k1):
        idx = [k % nsteps_hist for k in range(k0, k1)]
        return c.solve(mask[idx], target[idx], TOL_NEWTON, TOL_CG, CG_REL)

    # warm-up steps, then restart the history from F = I
    steps(ctx, 0, args.warmup)
    ctx.set_F(None)
    # the timed region: the whole load history in one call, which is one
    # graph launch (steps, Newton and CG iterations as device-side loops)
    l0 = mf.kernel_launches()
    barrier()
    torch.cuda.nvtx.range_push("timed_steps")
    with ClockSampler(local) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        o = steps(ctx, 0, args.steps)
        ev1.record(stream)
        barrier()
    torch.cuda.nvtx.range_pop()
    launches = mf.kernel_launches() - l0
    its = [(int(a), int(b)) for a, b in zip(o["newton"], o["cg"])]
    total_ms = ev0.elapsed_time(ev1)
    total_ms, value = replica_throughput(total_ms, args.steps, dist, "cuda")
    clocks = clk.summary()
    # the same steps one call (one launch) per step, for the per-step spread
    ctx.set_F(None)
    per_step = []
    for k in range(args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        steps(ctx, k, k + 1)
        b.record(stream)
        per_step.append((a, b))
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in per_step]
    # the paper's uniform start (the last converged state, strain-controlled
    # components shifted to the new F-bar), whole history in one call
    ctx.set_predictor(mf.MF_PRED_UNIFORM)
    steps(ctx, 0, 1)
    ctx.set_F(None)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    o_uni = steps(ctx, 0, args.steps)
    b.record(stream)
    torch.cuda.synchronize()
    uniform_ms = a.elapsed_time(b) / args.steps
    its_uniform = [(int(x), int(y)) for x, y in zip(o_uni["newton"], o_uni["cg"])]
    # linear extrapolation along the last load increment, whole history
    ctx.set_predictor(mf.MF_PRED_EXTRAPOLATE)
    steps(ctx, 0, 1)
    ctx.set_F(None)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    o_lin = steps(ctx, 0, args.steps)
    b.record(stream)
    torch.cuda.synchronize()
    linear_ms = a.elapsed_time(b) / args.steps
    its_linear = [(int(x), int(y)) for x, y in zip(o_lin["newton"], o_lin["cg"])]
    ctx.set_predictor(mf.MF_PRED_QUADRATIC)
    steps(ctx, 0, 1)

    # end to end through the C ABI with host buffers: step inputs go in as
    # arguments, <F>, <P> and the full F field come back to pinned host memory
    ctx.set_F(None)
    Fhost = torch.empty(9 * N, dtype=torch.float64, pin_memory=True).numpy()
    import ctypes
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        steps(ctx, k, k + 1)
        mf._check("mf_get_fields", mf._lib.mf_get_fields(ctx.h, Fhost.ctypes.data_as(ctypes.c_void_p),
                                                         None))
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * args.steps / e2e_s, "unit": "load steps/s",
           "h2d_bytes_per_step": 9 + 9 * 8, "d2h_bytes_per_step": 2 * 9 * 8 + 9 * N * 8}

    # inner-operator kernels: per-kernel time after an L2 flush, and the whole
    # projected operator in FP32 and FP64 (Gvoxel/s)
    ctx.set_F(None)
    steps(ctx, 0, 1)
    ctx.constitutive()
    m0 = mask[0]
    # per-kernel times: as back-to-back graph nodes (what the CG graph runs)
    # and with events around every single launch
    kms = ctx.time_kernels(m0, reps=20, graph=True)
    kms_single = ctx.time_kernels(m0, reps=20)
    bres = torch.empty(9 * N, dtype=torch.float64, device="cuda")
    res_ms = {}
    for name, arith in (("double_word", mf.MF_OUTER_DOUBLE_WORD), ("fp64", mf.MF_OUTER_FP64)):
        ctx.set_outer_arith(arith)
        time_residual(ctx, m0, target[0] * m0, bres, 2)
        res_ms[name] = time_residual(ctx, m0, target[0] * m0, bres, 10)
    del bres
    # the same load steps with the outer level (P and every residual
    # transform) in strict FP64 instead of double word: all timed steps
    ctx.set_outer_arith(mf.MF_OUTER_FP64)
    steps(ctx, 0, 1)     # untimed: re-tunes the residual tile for FP64
    ctx.set_F(None)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    steps(ctx, 0, args.steps)
    b.record(stream)
    torch.cuda.synchronize()
    fp64_outer_ms = a.elapsed_time(b) / args.steps
    ctx.set_outer_arith(mf.MF_OUTER_DOUBLE_WORD)
    ctx.constitutive()   # the tangent again, for the operator timings below
    x = torch.randn(9 * N, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)

    def time_matvec(c, xx, yy, reps):
        ts = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            c.matvec(xx, yy, m0)
            b.record(stream)
            ts.append((a, b))
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in ts]))

    time_matvec(ctx, x, y, 3)
    mv32_ms = time_matvec(ctx, x, y, 100)

    def time_cufft_matvec(c, xx, yy, reps):
        ts = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            c.matvec_cufft(xx, yy, m0)
            b.record(stream)
            ts.append((a, b))
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in ts]))

    # comparison: the same operator with cuFFT transforms
    ctx.cufft_bind()
    time_cufft_matvec(ctx, x, y, 3)
    cf32_ms = time_cufft_matvec(ctx, x, y, 30)
    cf32_parts = ctx.time_cufft(m0, reps=10)
    del x, y
    torch.cuda.empty_cache()

    # plain FP64 GPU path on the same steps, with the absolute CG stop
    # (Sec. 4's rule) and with the FP32-inner mode's inexact-Newton forcing,
    # run in lockstep with the FP32-inner path: per step <F>, <P> and the F
    # field of the FP32-inner run against the plain FP64 run, over the whole
    # history (tension, unloading, compression)
    nacc = args.steps if args.fp64_steps <= 0 else max(1, min(args.fp64_steps, args.steps))
    ctx64 = mf.Context(n, n, n, mf.MF_FP64)
    ctx64.set_material(mf.MF_SVK_CUBIC, params, g, rot=R)
    steps(ctx64, 0, 1)
    fp64 = {}
    for name, forcing, pred in (("plain", 0, mf.MF_PRED_UNIFORM), ("plain_extrapolated", 0, mf.MF_PRED_QUADRATIC),
                                ("forcing", 1, mf.MF_PRED_QUADRATIC)):
        ctx64.set_inexact_newton(forcing)
        ctx64.set_predictor(pred)
        steps(ctx64, 0, 1)
        ctx64.set_F(None)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        o = steps(ctx64, 0, nacc)
        b.record(stream)
        torch.cuda.synchronize()
        fp64[name] = {
            "ms_per_step": a.elapsed_time(b) / nacc,
            "newton_cg_per_step": [(int(x), int(y)) for x, y in zip(o["newton"], o["cg"])], "steps": nacc}
    # accuracy, lockstep: FP32 inner (double-word outer, quadratic
    # starts) against plain FP64 with the paper's uniform start
    ctx64.set_inexact_newton(0)
    ctx64.set_predictor(mf.MF_PRED_UNIFORM)
    ctx64.set_F(None)
    ctx.set_F(None)
    acc = {"Fbar": [], "Pbar": [], "F_field": []}
    for k in range(nacc):
        o32 = steps(ctx, k, k + 1)
        o64 = steps(ctx64, k, k + 1)
        F32 = ctx.get_fields()[0]
        F64 = ctx64.get_fields()[0]
        acc["Fbar"].append(float(np.max(np.abs(o32["Fbar"] - o64["Fbar"])) / np.max(np.abs(o64["Fbar"]))))
        acc["Pbar"].append(float(np.max(np.abs(o32["Pbar"] - o64["Pbar"]))) / 168.0)
        acc["F_field"].append(float(np.max(np.abs(F32 - F64)) / np.max(np.abs(F64))))
        del F32, F64
    accuracy = {"steps": nacc,
                "Fbar_max_rel": max(acc["Fbar"]), "Pbar_max_abs_over_C11": max(acc["Pbar"]),
                "F_field_max_rel": max(acc["F_field"]),
                "per_step": {k: [float("%.3g" % v) for v in acc[k]] for k in ("Fbar", "Pbar", "F_field")},
                "note": ("FP32 inner with double-word outer arithmetic and quadratic starts (the timed "
                         "configuration) against the plain FP64 path with uniform starts, every step of the "
                         "history, same tolerances; <P> error over C11 = 168")}
    # the FP64 path with forcing (and quadratic starts) against plain FP64
    # at the end of the history
    F64p = ctx64.get_fields()[0]
    ctx64.set_inexact_newton(1)
    ctx64.set_predictor(mf.MF_PRED_QUADRATIC)
    ctx64.set_F(None)
    of = steps(ctx64, 0, nacc)
    F64f = ctx64.get_fields()[0]
    accuracy["fp64_forcing_vs_plain_F_field_max_rel"] = float(np.max(np.abs(F64f - F64p)) / np.max(np.abs(F64p)))
    del F64p, F64f, of
    ctx64.set_inexact_newton(0)
    del ctx
    torch.cuda.empty_cache()
    ctx64.constitutive()
    x64 = torch.randn(9 * N, dtype=torch.float64, device="cuda")
    y64 = torch.empty_like(x64)
    time_matvec(ctx64, x64, y64, 2)
    mv64_ms = time_matvec(ctx64, x64, y64, 10)
    ctx64.cufft_bind()
    time_cufft_matvec(ctx64, x64, y64, 2)
    cf64_ms = time_cufft_matvec(ctx64, x64, y64, 10)
    kms64 = ctx64.time_kernels(m0, reps=5)
    del ctx64, x64, y64

    # the arithmetic roof of the FP64 path: measured FP64 (and FP32) FMA rate
    fp64_peak = mf.probe_fma(mf.MF_FP64)
    fp32_peak = mf.probe_fma(mf.MF_FP32_INNER)

    batched = run_batched(args) if not args.no_batched else None
    adjoint = run_adjoint(args) if not args.no_adjoint else None
    paper_cases = run_paper_cases(args) if not args.no_paper_cases else None

    peak, peak_kind = measured_peaks()
    dom = int(np.argmax(kms))
    achieved = ALGO_BYTES_F32[dom] * N / (kms[dom] * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "load steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "voxels": N, "grains": NGRAINS, "load_steps": nsteps_hist,
                   "l2": "inputs larger than L2 (K alone is 377 MB); kernel timings flush L2",
                   "parallelism": "replicas"},
        "gpu_launches": int(launches),
        "e2e": e2e,
        "clocks": clocks,
        "roofline": {"bound": "hbm", "kernel": KERNELS[dom], "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind + " (MEASURED_PEAKS hbm_gbs)" if peak_kind == "measured"
                     else peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": ncu_traffic(KERNELS[dom]),
                     "algorithmic_bytes_per_voxel": ALGO_BYTES_F32[dom]},
        "kernels_fp32": {k: {"ms": float(t), "GB_s": b * N / (t * 1e-3) / 1e9,
                             "frac": b * N / (t * 1e-3) / 1e9 / peak, "ms_single_launch": float(t1)}
                         for k, t, t1, b in zip(KERNELS, kms, kms_single, ALGO_BYTES_F32)},
        "kernel_timing": ("ms: 20 (L2 flush, launch) pairs as one CUDA graph, events around it, minus the "
                          "graph of the flushes alone, per launch; ms_single_launch: events around each "
                          "launch after its flush"),
        "kernels_fp64": {k: {"ms": float(t), "GB_s": b * N / (t * 1e-3) / 1e9}
                         for k, t, b in zip(KERNELS, kms64, ALGO_BYTES_F64)},
        "autotune": {"zpass_tile_columns": ztile,
                     "zpass_ms_by_tile": {str(w): float(m) for w, m in zip((4, 8, 16), ztile_ms)},
                     "xy_forward_schedule": XY_SCHEDULES[xy_fwd],
                     "xy_inverse_schedule": XY_SCHEDULES[xy_inv],
                     "xy_forward_ms_by_schedule": {"per_plane": float(xy_ms[0]), "persistent": float(xy_ms[1]),
                                                   "cluster": float(xy_ms[2])},
                     "xy_inverse_ms_by_schedule": {"per_plane": float(xy_ms[3]), "cluster": float(xy_ms[4])}},
        "matvec_gvoxel_s": {"fp32": N / (mv32_ms * 1e-3) / 1e9, "fp64": N / (mv64_ms * 1e-3) / 1e9,
                            "reps": "median of 100 (FP32) and 10 (FP64) warm applications, events per application"},
        "fp64_roofline": {"bound": "fp64 FMA", "flop_per_voxel": MATVEC_FLOP_F64,
                          "achieved_TFLOP_s": MATVEC_FLOP_F64 * N / (mv64_ms * 1e-3) / 1e12,
                          "peak_TFLOP_s": fp64_peak, "peak_kind": "measured here (mf_probe_fma, FP64)",
                          "frac": MATVEC_FLOP_F64 * N / (mv64_ms * 1e-3) / 1e12 / fp64_peak,
                          "fp32_fma_TFLOP_s": fp32_peak,
                          "note": ("plain FP64 projected operator: the FP64 pipe, not HBM, bounds it "
                                   "(about 1.1 kflop per voxel per application against 504 B)")},
        "matvec_roofline_fp32": {"bytes_per_voxel": MATVEC_BYTES_F32,
                                 "achieved_GB_s": MATVEC_BYTES_F32 * N / (mv32_ms * 1e-3) / 1e9,
                                 "frac": MATVEC_BYTES_F32 * N / (mv32_ms * 1e-3) / 1e9 / peak,
                                 "unit": "GB/s", "peak": peak},
        "matvec_cufft_comparison_gvoxel_s": {
            "fp32": N / (cf32_ms * 1e-3) / 1e9, "fp64": N / (cf64_ms * 1e-3) / 1e9,
            "fp32_parts_ms": {"r2c": float(cf32_parts[0]), "gstar": float(cf32_parts[1]),
                              "c2r": float(cf32_parts[2])}},
        "residual_ms": res_ms,
        "load_step_ms": {
            "timing": ("each path runs the whole history in one call (one graph launch) and reports its time "
                       "over the steps; fp32_inner_dw_outer_per_call_median: one call per step"),
            "fp32_inner_dw_outer": total_ms / args.steps,
            "fp32_inner_dw_outer_per_call_median": float(np.median(step_ms)),
            "fp32_inner_fp64_outer": fp64_outer_ms,
            "fp32_inner_dw_outer_uniform_predictor": uniform_ms,
            "fp32_inner_dw_outer_linear_predictor": linear_ms,
            "fp64_plain": fp64["plain"]["ms_per_step"],
            "fp64_plain_extrapolated": fp64["plain_extrapolated"]["ms_per_step"],
            "fp64_forcing": fp64["forcing"]["ms_per_step"],
            "fp64_steps_timed": nacc,
            "labels": {
                "fp32_inner_dw_outer": ("the timed configuration: FP32 inner CG; outer level (P, residual "
                                        "transforms) in double-word FP32 (about 48 bits), FP32 first residual "
                                        "of a step that did not start extrapolated; averages, control and "
                                        "Newton update in FP64; each step starts from the quadratic through the "
                                        "last three converged states (distinct loads) at the new load"),
                "fp32_inner_dw_outer_linear_predictor": ("the same with the start extrapolated linearly along the "
                                                         "last load increment"),
                "fp32_inner_dw_outer_uniform_predictor": ("the same with the paper's uniform start (last "
                                                          "converged state, strain-controlled components "
                                                          "shifted to the new F-bar)"),
                "fp64_plain_extrapolated": "plain FP64, CG to the absolute tolerance, quadratic starts",
                "fp32_inner_fp64_outer": "FP32 inner CG, outer level (P and every residual) in strict FP64",
                "fp64_plain": "every step in FP64, CG to the absolute tolerance (Sec. 4's rule), uniform starts",
                "fp64_forcing": ("every step in FP64 with the same inexact-Newton forcing and quadratic starts "
                                 "as the FP32-inner path (mf_set_inexact_newton): same stopping rule")},
            "ratio_fp64_plain_over_fp32_inner": fp64["plain"]["ms_per_step"] / (total_ms / args.steps),
            "ratio_fp64_forcing_over_fp32_inner": fp64["forcing"]["ms_per_step"] / (total_ms / args.steps)},
        "accuracy_fp32_inner_vs_fp64": accuracy,
        "iterations": {"fp32_inner_newton_cg_per_step": its,
                       "fp32_inner_uniform_predictor_newton_cg_per_step": its_uniform,
                       "fp32_inner_linear_predictor_newton_cg_per_step": its_linear,
                       "fp64_plain_extrapolated_newton_cg_per_step": fp64["plain_extrapolated"]["newton_cg_per_step"],
                       "fp64_plain_newton_cg_per_step": fp64["plain"]["newton_cg_per_step"],
                       "fp64_forcing_newton_cg_per_step": fp64["forcing"]["newton_cg_per_step"]},
    }
    if batched is not None:
        line["batched"] = batched
    if adjoint is not None:
        line["adjoint"] = adjoint
    if paper_cases is not None:
        line["paper_cases"] = paper_cases
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        # the model takes this run's plain FP64 iteration counts (median per
        # step), the oracle being a plain FP64 solver with the same stop rule
        nn = int(np.median([a for a, _ in fp64["plain"]["newton_cg_per_step"]]))
        nc = int(np.median([b for _, b in fp64["plain"]["newton_cg_per_step"]]))
        cb = cpu_baseline_entry(oracle_sample(cores, n_newton=nn, n_cg=nc,
                                              counts="median per step of this run's plain FP64 GPU path"), cores)
        # measured, not modelled: whole oracle runs of the 16^3 workload
        cb["full_runs_16cubed"] = [oracle_full("c1_sphere16", t) for t in sorted({1, cores})]
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def phase_composition(t, ids, names, skip_steps=2):
    """Per-phase durations of a traced history (mf_trace_read marks): each
    phase lasts from the mark before it to its own; the steps are split at
    the step-start marks.  Returns the per-step averages (us) over the steps
    after the first `skip_steps`, and every step's total."""
    starts = [i for i, x in enumerate(ids) if x == 1]
    totals, acc = [], {}
    for si, a in enumerate(starts):
        b = starts[si + 1] if si + 1 < len(starts) else len(ids)
        end = t[b] if b < len(ids) else t[b - 1]
        totals.append(round((int(end) - int(t[a])) / 1e3, 1))
        if si < skip_steps:
            continue
        for i in range(a + 1, b):
            k = names.get(int(ids[i]), str(int(ids[i])))
            acc[k] = acc.get(k, 0.0) + (int(t[i]) - int(t[i - 1])) / 1e3
    n = max(1, len(starts) - skip_steps)
    return {k: round(v / n, 1) for k, v in sorted(acc.items(), key=lambda kv: -kv[1])}, totals


def run_phase_trace(args):
    """The composition of a load step of the timed workload: the history run
    on the trace build of the library (phase timestamps from the device),
    in a child process that loads that build."""
    import subprocess
    from paper_1901_06531_gb300 import build
    build.build(trace=True)
    env = dict(os.environ, MF_LIBRARY="trace")
    res = subprocess.run([sys.executable, os.path.abspath(__file__), "--phase-trace-child", "--steps",
                          str(args.steps), "--warmup", str(args.warmup)], env=env, capture_output=True, text=True)
    sys.stdout.write(res.stdout)
    sys.stderr.write(res.stderr)
    if res.returncode:
        raise SystemExit(res.returncode)


def phase_trace_child(args):
    import torch
    from paper_1901_06531_gb300 import mixfft as mf
    g, params, R, mask, target = workload()
    n = N1
    ctx = mf.Context(n, n, n, mf.MF_FP32_INNER)
    ctx.set_material(mf.MF_SVK_CUBIC, params, g, rot=R)
    ctx.set_predictor(mf.MF_PRED_QUADRATIC)
    ctx.autotune()
    nst = mask.shape[0]

    def steps(k0, k1):
        idx = [k % nst for k in range(k0, k1)]
        return ctx.solve(mask[idx], target[idx], TOL_NEWTON, TOL_CG, CG_REL)

    steps(0, args.warmup)
    ctx.set_F(None)
    mf.trace_read()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    o = steps(0, args.steps)
    b.record()
    torch.cuda.synchronize()
    t, ids = mf.trace_read()
    comp, totals = phase_composition(t, ids, mf.TRACE_PHASES)
    print(json.dumps({"phase_trace": {
        "workload": "128^3 polycrystal, the timed history on the trace build (a mark kernel between phases)",
        "traced_ms_per_step": a.elapsed_time(b) / args.steps, "marks": int(len(t)),
        "newton_cg_per_step": [[int(x), int(y)] for x, y in zip(o["newton"], o["cg"])],
        "step_us": totals, "us_per_step_after_step_2": comp}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=0,
                    help="load steps of the FP64 comparison and accuracy runs (0: all timed steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched 48-cell workload")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the 128^3 adjoint workload")
    ap.add_argument("--no-paper-cases", action="store_true",
                    help="skip the 64^3 control-case comparison and the C2 workload")
    ap.add_argument("--matvec-only", type=int, default=0,
                    help="profiling driver: run this many projected-operator applications only")
    ap.add_argument("--kernels-only", type=int, default=0,
                    help="profiling driver: time the four CG-iteration kernels this many times each")
    ap.add_argument("--fp64", action="store_true", help="with --matvec-only / --kernels-only: FP64")
    ap.add_argument("--xy-cluster", type=int, default=-1, choices=[-1, 0, 1, 2, 3],
                    help=("with --matvec-only / --kernels-only (FP32): x-y passes as two-CTA cluster kernels "
                          "(bit 0 forward, bit 1 inverse); -1: the autotuner's choice"))
    ap.add_argument("--oracle-full", action="store_true",
                    help="time whole oracle runs of the 16^3 and 64^3 workloads (1 and all threads)")
    ap.add_argument("--phase-trace", action="store_true",
                    help="the composition of a load step from the trace build's phase timestamps")
    ap.add_argument("--phase-trace-child", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.phase_trace_child:
        phase_trace_child(args)
    elif args.phase_trace:
        run_phase_trace(args)
    elif args.oracle_full:
        run_oracle_full(args)
    elif args.matvec_only or args.kernels_only:
        run_matvec_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
