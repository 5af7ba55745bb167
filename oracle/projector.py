"""The modified projection operator G-hat-star (Sec. 2.1-2.3).

Eq. (eq:G): away from the null and Nyquist frequencies,
    (G-hat : A)_ij = delta_ik xi_j xi_l / (xi.xi) A_kl = xi_j xi_l A_il / (xi.xi),
the compatible part of A (Eq. comp).  Eq. (eq:Gnew) replaces the value at the
null frequency by the fourth-order identity (stress control) and Eq.
(eq:Gnewnew) makes it component-wise: identity on the stress-controlled
components IJ, zero on the strain-controlled components ij.  Nyquist
frequencies give zero.

Readings taken where the paper is not explicit:
  * "Nyquist frequencies" = every frequency with at least one axis index at
    n_a/2 on an even axis (then G(-xi) = G(xi) on what is kept, and the
    operator is real, symmetric and idempotent);
  * voxels are unit cubes, so xi_a = k_a / n_a (only the direction of xi
    enters).
Fields are [c, z, y, x] arrays with c = 3*i + j.
"""
from __future__ import annotations

import numpy as np

from . import dft


def frequency_grid(shape):
    """xi components (xi_x, xi_y, xi_z) broadcast to [z, y, x], plus masks of
    the null frequency and of the Nyquist frequencies."""
    nz, ny, nx = shape
    kx = dft.signed_index(nx) / nx
    ky = dft.signed_index(ny) / ny
    kz = dft.signed_index(nz) / nz
    xi = [np.broadcast_to(kx[None, None, :], shape),
          np.broadcast_to(ky[None, :, None], shape),
          np.broadcast_to(kz[:, None, None], shape)]
    nyq = (dft.nyquist_flag(nz)[:, None, None] | dft.nyquist_flag(ny)[None, :, None]
           | dft.nyquist_flag(nx)[None, None, :])
    null = np.zeros(shape, dtype=bool)
    null[0, 0, 0] = True
    return xi, null, nyq


def apply_hat(ahat: np.ndarray, mask) -> np.ndarray:
    """G-hat-star : A-hat at every frequency, Eq. (eq:Gnewnew).

    ahat: complex [9, z, y, x]; mask: 9 flags, 1 = stress-controlled component.
    """
    shape = ahat.shape[1:]
    xi, null, nyq = frequency_grid(shape)
    xi2 = xi[0] ** 2 + xi[1] ** 2 + xi[2] ** 2
    safe = np.where(null, 1.0, xi2)
    A = ahat.reshape((3, 3) + shape)
    out = np.zeros_like(A)
    # rest of frequencies: out_ij = xi_j * (sum_l A_il xi_l) / (xi.xi)
    for i in range(3):
        q = (A[i, 0] * xi[0] + A[i, 1] * xi[1] + A[i, 2] * xi[2]) / safe
        for j in range(3):
            out[i, j] = q * xi[j]
    # Nyquist frequencies: zero
    out[:, :, nyq] = 0.0
    # null frequency: identity on stress-controlled, zero on strain-controlled
    m = np.asarray(mask, dtype=np.float64).reshape(3, 3)
    out[:, :, 0, 0, 0] = m * A[:, :, 0, 0, 0]
    return out.reshape(ahat.shape)


def apply(a: np.ndarray, mask) -> np.ndarray:
    """G-star(a) = F^-1{ G-hat-star : F{a} } for a real field a [9, z, y, x]."""
    return np.real(dft.inverse(apply_hat(dft.forward(a), mask)))


def apply_with_mean(a: np.ndarray, mask, mean_target) -> np.ndarray:
    """G-star(a - mean_target) for a uniform mean_target (9,) -- the right-hand
    side of Eq. (linequil2ast) uses this with a = P, mean_target = P-bar.  A
    uniform field only has a null-frequency coefficient, so it is subtracted
    there."""
    ahat = dft.forward(a)
    ahat[:, 0, 0, 0] -= np.asarray(mean_target, dtype=np.float64)
    return np.real(dft.inverse(apply_hat(ahat, mask)))
