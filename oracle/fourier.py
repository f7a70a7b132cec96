"""Unitary discrete Fourier transform F (Theory, "Parallel Imaging Reconstruction").

F is the multidimensional DFT over the image axes with forward sign negative and scaling
N^{-1/2}, so that F^H F = I (this identity is what the derivation of Eq. K uses).
Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def dft_matrix(n: int) -> np.ndarray:
    """The definition: F[k, j] = n^{-1/2} exp(-2 pi i k j / n), k, j = 0..n-1."""
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    return np.exp(-2j * np.pi * k * j / n) / np.sqrt(n)


def dft_naive(x: np.ndarray, ndim: int) -> np.ndarray:
    """Unitary DFT over the last ``ndim`` axes by explicit matrix products with ``dft_matrix``
    (slow; tiny grids only)."""
    y = np.asarray(x, np.complex128)
    for ax in range(-ndim, 0):
        m = dft_matrix(y.shape[ax])
        y = np.moveaxis(np.tensordot(m, np.moveaxis(y, ax, 0), axes=(1, 0)), 0, ax)
    return y


def fft(x: np.ndarray, ndim: int) -> np.ndarray:
    """F x over the last ``ndim`` axes (library FFT, unitary scaling)."""
    return np.fft.fftn(x, axes=tuple(range(-ndim, 0)), norm="ortho")


def ifft(x: np.ndarray, ndim: int) -> np.ndarray:
    """F^H x over the last ``ndim`` axes."""
    return np.fft.ifftn(x, axes=tuple(range(-ndim, 0)), norm="ortho")


def dense_F(shape: tuple[int, ...]) -> np.ndarray:
    """Dense N x N matrix of F for a C-ordered image of ``shape`` (Kronecker product of the 1D
    matrices, slowest axis first)."""
    m = np.ones((1, 1), np.complex128)
    for n in shape:
        m = np.kron(m, dft_matrix(n))
    return m
