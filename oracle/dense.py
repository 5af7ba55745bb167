"""Dense assembly of the Newton system of Eq. (linequil2ast) on tiny grids.

The projection G* and the tangent K are assembled as 9N x 9N matrices column
by column (G* from the oracle's projector applied to unit fields, K from its
block-diagonal voxel blocks), so that the linear and the nonlinear solves can
be repeated by dense LU and compared with the CG path.
"""
from __future__ import annotations

import numpy as np

from . import projector


def gstar_matrix(shape, mask):
    n = 9 * int(np.prod(shape))
    G = np.zeros((n, n))
    e = np.zeros(n)
    for col in range(n):
        e[:] = 0.0
        e[col] = 1.0
        G[:, col] = projector.apply(e.reshape((9,) + tuple(shape)), mask).ravel()
    return G


def k_matrix(K):
    """Block matrix of (K:x) with x flattened as [c, voxel]."""
    nv = K[0, 0].size
    Kv = K.reshape(9, 9, nv)
    M = np.zeros((9 * nv, 9 * nv))
    for c in range(9):
        for d in range(9):
            M[c * nv:(c + 1) * nv, d * nv:(d + 1) * nv] = np.diag(Kv[c, d])
    return M


def solve_projected(K, b, mask):
    """Solve G* K G* x = b on range(G*) by dense LU of
    (G* K G* + I - G*) x = b (the extra term is the identity on the
    complement of range(G*), making the matrix nonsingular there)."""
    shape = b.shape[1:]
    G = gstar_matrix(shape, mask)
    A = G @ k_matrix(K) @ G
    n = A.shape[0]
    x = np.linalg.solve(A + np.eye(n) - G, b.ravel())
    return x.reshape(b.shape), 1
