"""Differentiable homogenized response: a ``torch.autograd.Function`` whose
forward pass is the library's load-step solver and whose backward pass is the
library's adjoint (``mf_adjoint``), one linear solve per load step.

The response of a load history is, per step, the nine FREE macroscopic
quantities: <F>_ij on the stress-controlled components and <P>_ij on the
strain-controlled ones (the prescribed ones have zero derivative).  For a
hyperelastic law the converged state of a step depends on the material only
through that step's equilibrium G*(P(F) - P-bar) = 0 (Eq. linequil2ast with
dF = 0), so the vector-Jacobian product of step k is one adjoint solve at the
converged F of step k, with weights w_F = g_k on the stress-controlled and
w_P = g_k on the strain-controlled components.  The forward pass saves the
converged F of every step on the device (9N doubles each; the Newton-history
checkpoints), the backward pass reloads them.

Differentiable inputs: the neo-Hookean parameters (mu, lam) per phase and the
per-voxel stiffness scale s_v (P_v = s_v P(F_v; mu, lam)).
"""
from __future__ import annotations

import numpy as np
import torch

from . import mixfft


def free_response(Fbar, Pbar, mask):
    """<F> on stress-controlled components (mask 1), <P> on the others."""
    return np.where(np.asarray(mask, dtype=bool), Fbar, Pbar)


class _HomogenizedResponse(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params, scale, cell, phase, mask, target, opts):
        mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1, 9)
        target = np.ascontiguousarray(target, dtype=np.float64).reshape(-1, 9)
        p = params.detach().to("cpu", torch.float64).numpy()
        sc = None if scale is None else scale.detach().to("cpu", torch.float64).numpy().reshape(cell.shape)
        cell.set_material(mixfft.MF_NEOHOOKE, p, phase, scale=sc)
        cell.set_F(None)
        nsteps = mask.shape[0]
        out = np.zeros((nsteps, 9))
        checkpoints = []
        iters = []
        for k in range(nsteps):
            r = cell.solve(mask[k:k + 1], target[k:k + 1], tol_newton=opts["tol_newton"], tol_cg=opts["tol_cg"],
                           cg_rel=opts["cg_rel"], max_newton=opts["max_newton"], max_cg=opts["max_cg"])
            checkpoints.append(cell.save_F())
            out[k] = free_response(r["Fbar"][0], r["Pbar"][0], mask[k])
            iters.append((int(r["newton"][0]), int(r["cg"][0])))
        fctx.cell = cell
        fctx.mask = mask
        fctx.opts = opts
        fctx.checkpoints = checkpoints
        fctx.params_shape = tuple(params.shape)
        fctx.params_meta = (params.dtype, params.device)
        fctx.scale_meta = None if scale is None else (tuple(scale.shape), scale.dtype, scale.device)
        fctx.iters = iters
        return torch.from_numpy(out).to(params.dtype)

    @staticmethod
    def backward(fctx, grad_out):
        cell = fctx.cell
        g = grad_out.detach().to("cpu", torch.float64).numpy().reshape(-1, 9)
        want_scale = fctx.scale_meta is not None and fctx.needs_input_grad[1]
        gp = np.zeros(fctx.params_shape)
        gs = buf = None
        if want_scale:
            gs = torch.zeros(cell.N, dtype=torch.float64, device=cell.device)
            buf = torch.empty(cell.N, dtype=torch.float64, device=cell.device)
        o = fctx.opts
        for k in range(g.shape[0] - 1, -1, -1):
            if not np.any(g[k]):
                continue
            m = fctx.mask[k]
            wF = np.where(m == 1, g[k], 0.0)
            wP = np.where(m == 1, 0.0, g[k])
            cell.load_F(fctx.checkpoints[k])
            _, gk, _ = cell.adjoint(m, wF, wP, tol_cg=o["adj_tol_cg"], cg_rel=o["adj_cg_rel"],
                                    max_cg=o["adj_max_cg"], dscale=buf)
            gp += gk
            if want_scale:
                gs += buf
        # leave the cell at the last converged state, as after the forward pass
        cell.load_F(fctx.checkpoints[-1])
        dtype, device = fctx.params_meta
        grad_params = torch.from_numpy(gp).to(device=device, dtype=dtype) if fctx.needs_input_grad[0] else None
        grad_scale = None
        if want_scale:
            shape, sdtype, sdevice = fctx.scale_meta
            grad_scale = gs.reshape(shape).to(device=sdevice, dtype=sdtype)
        return grad_params, grad_scale, None, None, None, None, None


def homogenized_response(cell, phase, params, mask, target, scale=None, tol_newton=1e-8, tol_cg=1e-10,
                         cg_rel=1e-4, max_newton=50, max_cg=5000, adj_tol_cg=1e-12, adj_cg_rel=1e-9,
                         adj_max_cg=20000):
    """Free macroscopic response (nsteps, 9) of a load history on ``cell`` (a
    ``mixfft.Context``), differentiable in ``params`` ((nphase, 2) neo-Hookean
    (mu, lam)) and ``scale`` ((nz, ny, nx) or None).

    mask, target: (nsteps, 9) control masks and prescribed values as for
    ``Context.solve``; the cell starts from F = I.  The adjoint CG stops at
    rms(r) <= max(adj_tol_cg, adj_cg_rel * rms(r0)).
    """
    opts = dict(tol_newton=tol_newton, tol_cg=tol_cg, cg_rel=cg_rel, max_newton=max_newton, max_cg=max_cg,
                adj_tol_cg=adj_tol_cg, adj_cg_rel=adj_cg_rel, adj_max_cg=adj_max_cg)
    phase = np.ascontiguousarray(phase, dtype=np.int32)
    return _HomogenizedResponse.apply(params, scale, cell, phase, mask, target, opts)
