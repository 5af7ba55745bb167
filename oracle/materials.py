"""Constitutive laws: first Piola stress P(F) and tangent K = dP/dF
(Eq. eq:lineariz), voxel-wise, in FP64.

Two hyperelastic laws:

* Compressible neo-Hookean (the paper does not fix a form; this one is the
  textbook reading used throughout the project):
      W = mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2
      P = mu F + (lam ln J - mu) F^-T
      K_ijkl = mu d_ik d_jl + lam Finv_ji Finv_lk + (mu - lam ln J) Finv_jk Finv_li
  At F = I this is isotropic linear elasticity with Lame constants (lam, mu).
* St Venant-Kirchhoff (Sec. 3.1 uses it; the cubic, rotated form stands in
  for the polycrystal of Sec. 3.2):
      E = (F^T F - I)/2,  S = C : E,  P = F S
      K_ijkl = d_ik S_lj + F_ia F_kc C_ajcl
  with C cubic in the crystal frame (C11, C12, C44) rotated per grain,
  C'_ijkl = R_ia R_jb R_kc R_ld C_abcd.

An optional per-voxel scale s multiplies both P and K.
Fields: F, P are [9, z, y, x] (c = 3i + j); K is [9, 9, z, y, x] with
K[3i+j, 3k+l] = K_ijkl.
"""
from __future__ import annotations

import numpy as np

NEOHOOKE = "neohooke"
SVK_CUBIC = "svk_cubic"


def cubic_stiffness(c11, c12, c44):
    """Cubic elasticity tensor C_abcd in the crystal frame."""
    d = np.eye(3)
    C = (c12 * np.einsum("ab,cd->abcd", d, d)
         + c44 * (np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)))
    aniso = c11 - c12 - 2.0 * c44
    for e in range(3):
        C[e, e, e, e] += aniso
    return C


def rotate_stiffness(C, R):
    """C'_ijkl = R_ia R_jb R_kc R_ld C_abcd."""
    return np.einsum("ia,jb,kc,ld,abcd->ijkl", R, R, R, R, C)


def isotropic_stiffness(lam, mu):
    return cubic_stiffness(lam + 2.0 * mu, lam, mu)


def _as_mats(F):
    """[9, *s] -> [*s, 3, 3]."""
    s = F.shape[1:]
    return np.moveaxis(F.reshape((3, 3) + s), (0, 1), (-2, -1))


def _from_mats(A):
    s = A.shape[:-2]
    return np.moveaxis(A, (-2, -1), (0, 1)).reshape((9,) + s)


def neohooke_PK(F, mu, lam):
    """P and K for the neo-Hookean law; mu, lam broadcast over voxels."""
    Fm = _as_mats(F)
    J = np.linalg.det(Fm)
    if np.any(J <= 0):
        raise FloatingPointError("neo-Hookean: det F <= 0")
    Finv = np.linalg.inv(Fm)
    lnJ = np.log(J)
    FinvT = np.swapaxes(Finv, -1, -2)
    mu = np.asarray(mu, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    P = mu[..., None, None] * Fm + (lam * lnJ - mu)[..., None, None] * FinvT
    d = np.eye(3)
    K = (mu[..., None, None, None, None] * np.einsum("ik,jl->ijkl", d, d)
         + lam[..., None, None, None, None] * np.einsum("...ji,...lk->...ijkl", Finv, Finv)
         + (mu - lam * lnJ)[..., None, None, None, None]
         * np.einsum("...jk,...li->...ijkl", Finv, Finv))
    return _from_mats(P), _K_to_field(K)


def neohooke_energy(F, mu, lam):
    Fm = _as_mats(F)
    J = np.linalg.det(Fm)
    lnJ = np.log(J)
    I1 = np.einsum("...ij,...ij->...", Fm, Fm)
    return 0.5 * mu * (I1 - 3.0) - mu * lnJ + 0.5 * lam * lnJ ** 2


def svk_PK(F, Cv):
    """P and K for St Venant-Kirchhoff with a per-voxel stiffness Cv
    [*s, 3, 3, 3, 3]."""
    Fm = _as_mats(F)
    E = 0.5 * (np.einsum("...ki,...kj->...ij", Fm, Fm) - np.eye(3))
    S = np.einsum("...abcd,...cd->...ab", Cv, E)
    P = np.einsum("...ik,...kj->...ij", Fm, S)
    d = np.eye(3)
    K = (np.einsum("ik,...lj->...ijkl", d, S)
         + np.einsum("...ia,...kc,...ajcl->...ijkl", Fm, Fm, Cv))
    return _from_mats(P), _K_to_field(K)


def svk_energy(F, Cv):
    Fm = _as_mats(F)
    E = 0.5 * (np.einsum("...ki,...kj->...ij", Fm, Fm) - np.eye(3))
    return 0.5 * np.einsum("...ab,...abcd,...cd->...", E, Cv, E)


def _K_to_field(K):
    """[*s, 3,3,3,3] -> [9, 9, *s]."""
    s = K.shape[:-4]
    K = K.reshape(s + (9, 9))
    return np.moveaxis(K, (-2, -1), (0, 1))


class Material:
    """Phase map plus per-phase parameters.

    model NEOHOOKE: params (nphase, 2) = (mu, lam).
    model SVK_CUBIC: params (nphase, 3) = (C11, C12, C44); rot (nphase, 3, 3)
    rotates phase p's crystal frame into the sample frame (None = identity).
    scale: optional per-voxel multiplier of P and K.
    """

    def __init__(self, phase, model, params, rot=None, scale=None):
        self.phase = np.asarray(phase, dtype=np.int64)
        self.model = model
        self.params = np.asarray(params, dtype=np.float64)
        self.rot = None if rot is None else np.asarray(rot, dtype=np.float64)
        self.scale = None if scale is None else np.asarray(scale, dtype=np.float64)
        if model == SVK_CUBIC:
            tabs = []
            for p in range(self.params.shape[0]):
                C = cubic_stiffness(*self.params[p])
                if self.rot is not None:
                    C = rotate_stiffness(C, self.rot[p])
                tabs.append(C)
            self.C_table = np.asarray(tabs)
        elif model != NEOHOOKE:
            raise ValueError(model)

    def PK(self, F):
        if self.model == NEOHOOKE:
            mu = self.params[self.phase, 0]
            lam = self.params[self.phase, 1]
            P, K = neohooke_PK(F, mu, lam)
        else:
            P, K = svk_PK(F, self.C_table[self.phase])
        if self.scale is not None:
            P = P * self.scale
            K = K * self.scale
        return P, K

    def energy(self, F):
        if self.model == NEOHOOKE:
            W = neohooke_energy(F, self.params[self.phase, 0], self.params[self.phase, 1])
        else:
            W = svk_energy(F, self.C_table[self.phase])
        if self.scale is not None:
            W = W * self.scale
        return W


def apply_K(K, x):
    """(K : x)_ij = K_ijkl x_kl voxel-wise; K [9,9,*s], x [9,*s]."""
    return np.einsum("cd...,d...->c...", K, x)
