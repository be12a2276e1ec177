"""Euclidean gamma matrices in a chiral basis (oracle; test infrastructure only).

The paper states no Dirac basis.  We use hermitian gammas with
gamma5 = gamma_x gamma_y gamma_z gamma_t = diag(1, 1, -1, -1):

    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]   (k = x, y, z)
    gamma_t = [[0, 1], [1, 0]]

Index order mu = 0, 1, 2, 3 is x, y, z, t.
"""
from __future__ import annotations

import numpy as np

_SIGMA = np.array(
    [
        [[0, 1], [1, 0]],
        [[0, -1j], [1j, 0]],
        [[1, 0], [0, -1]],
    ],
    dtype=np.complex128,
)


def gamma_matrices() -> np.ndarray:
    """Array (4, 4, 4): gamma_mu for mu = x, y, z, t."""
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    z2 = np.zeros((2, 2), dtype=np.complex128)
    for k in range(3):
        g[k] = np.block([[z2, -1j * _SIGMA[k]], [1j * _SIGMA[k], z2]])
    g[3] = np.block([[z2, np.eye(2)], [np.eye(2), z2]])
    return g


def gamma5() -> np.ndarray:
    """gamma5 = gamma_x gamma_y gamma_z gamma_t (= diag(1, 1, -1, -1) in this basis)."""
    g = gamma_matrices()
    return g[0] @ g[1] @ g[2] @ g[3]
