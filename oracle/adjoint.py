"""Adjoint sensitivity of the homogenized response at a converged load step.

At convergence the discrete equilibrium of Eq. (linequil2ast) holds,
R(F, theta) = G*(P(F, theta) - P-bar) = 0, with F - F-bar in the range of G*.
For a linear response J = w_F . <F> + w_P . <P> (the free macroscopic
quantities: <F> on stress-controlled and <P> on strain-controlled
components), differentiating R gives A dF = -G*(dP/dtheta) with the
symmetric projected tangent A = G* K G* (K of Eq. eq:lineariz).  With W_F, W_P
the uniform fields of the weights and lambda the solution of
    A lambda = G*(W_F + K : W_P),       lambda in range(G*),
    dJ/dtheta = (1/N) sum_v (W_P - lambda_v) : dP_v/dtheta.
Neo-Hookean (per phase p, voxel scale s_v): dP/dmu = s (F - F^-T),
dP/dlam = s ln J F^-T on the voxels of phase p; dP_v/ds_v = P_v / s_v.
"""
from __future__ import annotations

import numpy as np

from . import materials, projector, solver


def response(material, F, wF, wP):
    P, _ = material.PK(F)
    return float(np.dot(wF, solver.mean9(F)) + np.dot(wP, solver.mean9(P)))


def gradient(material, F, mask, wF, wP, tol_cg=1e-11, max_cg=20000):
    """dJ/d(mu_p, lam_p) (nphase, 2) and dJ/ds_v [z, y, x] at the state F."""
    if material.model != materials.NEOHOOKE:
        raise ValueError("adjoint parameters are defined for the neo-Hookean law")
    shape = F.shape[1:]
    N = F[0].size
    P, K = material.PK(F)
    WF = np.broadcast_to(np.asarray(wF, dtype=np.float64)[:, None, None, None], F.shape)
    WP = np.broadcast_to(np.asarray(wP, dtype=np.float64)[:, None, None, None], F.shape)
    g = projector.apply(WF + materials.apply_K(K, WP), mask)
    lam_adj, _ = solver.cg(lambda x: solver.matvec(K, x, mask), g, tol_cg, max_cg)
    D = WP - lam_adj                          # (W_P - lambda), [9, z, y, x]
    Fm = np.moveaxis(F.reshape((3, 3) + shape), (0, 1), (-2, -1))
    J = np.linalg.det(Fm)
    FinvT = np.swapaxes(np.linalg.inv(Fm), -1, -2)
    FinvT = np.moveaxis(FinvT, (-2, -1), (0, 1)).reshape((9,) + shape)
    s = material.scale if material.scale is not None else np.ones(shape)
    dP_dmu = s * (F - FinvT)
    dP_dlam = s * np.log(J) * FinvT
    c_mu = np.sum(D * dP_dmu, axis=0) / N
    c_lam = np.sum(D * dP_dlam, axis=0) / N
    nphase = material.params.shape[0]
    grad = np.zeros((nphase, 2))
    for p in range(nphase):
        sel = material.phase == p
        grad[p, 0] = c_mu[sel].sum()
        grad[p, 1] = c_lam[sel].sum()
    Phat = P / s
    dscale = np.sum(D * Phat, axis=0) / N
    return grad, dscale
