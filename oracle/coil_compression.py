"""Coil compression (Methods, "Coil Compression"; Discussion): a compression matrix built from the
coil data maps the coil data and the coil sensitivity maps onto virtual coils ordered by
dominance, and the least dominant virtual coils are dropped.

Reading (the paper names the construction only by citation): the compression matrix is the
principal-component basis of the coil data.  With all coil-data samples stacked as Y (Nc x
samples), C = Y Y^H = V diag(s) V^H with s in descending order; the compression matrix is
A = V[:, :nv]^H (nv x Nc), virtual data y_v = A y, virtual maps S_v = A S.  Each virtual coil is
defined up to a unit phase (an eigenvector's), which changes neither the data term
sum_v S_v^H F^H R F S_v nor S_v^H y_v; comparisons use the projector A^H A.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def covariance(y: np.ndarray) -> np.ndarray:
    """C = Y Y^H over every sample of the coil data y [Nc, ...]."""
    Y = np.asarray(y, np.complex128).reshape(y.shape[0], -1)
    return Y @ Y.conj().T


def compression_matrix(y: np.ndarray, nv: int) -> tuple[np.ndarray, np.ndarray]:
    """(A, s): the nv x Nc compression matrix and the eigenvalues of C in descending order."""
    s, V = np.linalg.eigh(covariance(y))
    order = np.argsort(s)[::-1]
    return V[:, order[:nv]].conj().T, s[order]


def compress(y: np.ndarray, sens: np.ndarray, A: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Virtual coil data and maps: y_v = A y, S_v = A S (coil axis first)."""
    return np.tensordot(A, y, axes=(1, 0)), np.tensordot(A, sens, axes=(1, 0))
