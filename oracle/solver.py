"""Newton + conjugate-gradient solution of the Galerkin FFT equilibrium under
per-component stress/strain control (Sec. 2, Eq. linequil2ast, eq:mixedeqil).

Per load step k (Sec. 2.1 increments, Sec. 2.3 mixed control):
  1. predictor: on every strain-controlled component (mask 0) add the uniform
     amount that brings the voxel average of F to the prescribed F-bar;
     stress-controlled components keep the last converged field;
  2. Newton (Eq. eq:lineariz): compute P(F), K(F); solve
         G*(K : dF) = -G*(P(F) - P-bar)                       (Eq. linequil2ast)
     by conjugate gradients started at dF = 0; F += dF;
  3. stop when max_v |dF_v| / |<F>| < tol_newton (Sec. 4).

The CG runs on A(x) = G*(K : x).  b lies in the range of the projection G*
and so do all search directions; on that range A = G* K G* is symmetric.

Readings (Sec. 4 gives only "voxel averaged L2 norm of the residual" and
"maximum deformation gradient correction relative to the averaged deformation
gradient"):
  * CG stops when sqrt(sum_v |r_v|^2 / N) <= tol_cg, or at max_cg;
    a direction with p.Ap <= 0 is a breakdown;
  * Newton stops when max_v |dF_v|_F / |<F>|_F < tol_newton, measured on the
    correction just applied; P and the averages reported for the step are
    those of the final F.
"""
from __future__ import annotations

import numpy as np

from . import materials, projector


class CGBreakdown(RuntimeError):
    pass


class NotConverged(RuntimeError):
    pass


def matvec(K, x, mask):
    """y = G*(K : x) (left-hand side of Eq. linequil2ast)."""
    return projector.apply(materials.apply_K(K, x), mask)


def residual(P, mask, pbar):
    """b = -G*(P - P-bar) (right-hand side of Eq. linequil2ast)."""
    return -projector.apply_with_mean(P, mask, pbar)


def rms(x):
    """Voxel-averaged L2 norm sqrt(sum_v |x_v|_F^2 / N) of a [9, *s] field."""
    n = x[0].size
    return float(np.sqrt(np.sum(x * x) / n))


def cg(apply_A, b, tol, maxit):
    """Plain conjugate gradients from x0 = 0.  Returns (x, iterations)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    n = b[0].size
    it = 0
    while np.sqrt(rr / n) > tol:
        if it >= maxit:
            raise NotConverged(f"CG: {it} iterations, residual {np.sqrt(rr / n):.3e}")
        Ap = apply_A(p)
        pAp = float(np.sum(p * Ap))
        if not pAp > 0.0:
            raise CGBreakdown(f"CG: p.Ap = {pAp:.3e} at iteration {it}")
        alpha = rr / pAp
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(np.sum(r * r))
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        it += 1
    return x, it


def mean9(a):
    return a.reshape(9, -1).mean(axis=1)


def solve(material, mask, target, tol_newton=1e-8, tol_cg=1e-10,
          max_newton=50, max_cg=5000, F0=None, record_fields=False,
          linear_solver=None):
    """Run a load history.

    mask, target: (nsteps, 9); mask 1 -> target is P-bar, 0 -> F-bar.
    Returns dict with Fbar, Pbar (nsteps, 9), newton / cg iteration counts
    per step, and the final F, P fields.
    linear_solver(K, b, mask) may replace CG (dense brute-force checks); it
    returns (dF, iterations).
    """
    mask = np.asarray(mask, dtype=np.uint8)
    target = np.asarray(target, dtype=np.float64)
    shape = material.phase.shape
    if F0 is None:
        F = np.zeros((9,) + shape)
        F[0] = F[4] = F[8] = 1.0
    else:
        F = np.array(F0, dtype=np.float64)
    nsteps = mask.shape[0]
    out = {"Fbar": np.zeros((nsteps, 9)), "Pbar": np.zeros((nsteps, 9)),
           "newton": np.zeros(nsteps, dtype=np.int64),
           "cg": np.zeros(nsteps, dtype=np.int64), "fields": []}
    for k in range(nsteps):
        m = mask[k]
        tgt = target[k]
        Fm = mean9(F)
        for c in range(9):
            if m[c] == 0:
                F[c] += tgt[c] - Fm[c]
        pbar = np.where(m == 1, tgt, 0.0)
        ratio = np.inf
        n_newton = 0
        n_cg = 0
        while True:
            P, K = material.PK(F)
            if n_newton > 0 and ratio < tol_newton:
                break
            if n_newton >= max_newton:
                raise NotConverged(f"Newton: step {k}, ratio {ratio:.3e}")
            b = residual(P, m, pbar)
            if linear_solver is None:
                dF, its = cg(lambda x: matvec(K, x, m), b, tol_cg, max_cg)
            else:
                dF, its = linear_solver(K, b, m)
            F += dF
            n_newton += 1
            n_cg += its
            dnorm = np.sqrt(np.sum(dF * dF, axis=0))
            ratio = float(np.max(dnorm) / np.linalg.norm(mean9(F)))
        out["Fbar"][k] = mean9(F)
        out["Pbar"][k] = mean9(P)
        out["newton"][k] = n_newton
        out["cg"][k] = n_cg
        if record_fields:
            out["fields"].append((F.copy(), P.copy()))
    out["F"] = F
    out["P"] = P
    return out
