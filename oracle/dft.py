"""Discrete Fourier transform by its definition (Eq. eql_discrete2, Sec. 2.1).

The forward transform carries the 1/N factor so that the null frequency of a
field is its voxel average, which Sec. 2.2 uses (the transform of P at xi = 0
equals <P>).  The inverse is the plain sum.  Each axis is transformed by a
dense n x n matrix of twiddles exp(-+2 pi i j k / n); the phase j*k is reduced
modulo n before the exponential so that every twiddle is accurate to a few ulp.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(n: int, sign: int) -> np.ndarray:
    """W[k, j] = exp(sign * 2 pi i * (j*k mod n) / n)."""
    j = np.arange(n)
    phase = np.outer(j, j) % n
    return np.exp(sign * 2j * np.pi * phase / n)


def _transform(a: np.ndarray, sign: int) -> np.ndarray:
    out = np.asarray(a, dtype=np.complex128)
    for ax in (-3, -2, -1):
        n = out.shape[ax]
        W = dft_matrix(n, sign)
        out = np.moveaxis(np.tensordot(out, W, axes=([ax], [1])), -1, ax)
    return out


def forward(a: np.ndarray) -> np.ndarray:
    """F{a}(k) = (1/N) sum_x a(x) exp(-2 pi i k.x/n) over the last three axes."""
    n = a.shape[-1] * a.shape[-2] * a.shape[-3]
    return _transform(a, -1) / n


def inverse(ahat: np.ndarray) -> np.ndarray:
    """F^-1{ahat}(x) = sum_k ahat(k) exp(+2 pi i k.x/n) over the last three axes."""
    return _transform(ahat, +1)


def signed_index(n: int) -> np.ndarray:
    """Integer frequency of each DFT index: 0..n/2-1, -n/2 (Nyquist, even n),
    -n/2+1..-1."""
    k = np.arange(n)
    return np.where(k <= (n - 1) // 2, k, k - n)


def nyquist_flag(n: int) -> np.ndarray:
    """True at the Nyquist index n/2 of an even-length axis."""
    k = np.arange(n)
    return (n % 2 == 0) & (k == n // 2)
