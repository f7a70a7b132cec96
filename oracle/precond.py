"""The circulant preconditioner M^{-1} = F^H diag{k}^{-1} F (Eq. precon).

k = mu k_c + lambda k_d + gamma k_w (Eq. Kdiag) is the diagonal of K = F A F^H (Eq. K).

k_c, the data-fidelity part, follows the construction of "Efficient Implementation of the
Preconditioner" (Eq. diagonalelements): the diagonal of sum_i C_i^H R C_i with the BCCB
C_i = F S_i F^H is a circular correlation of the mask r with a sum of squared magnitudes of the
sensitivities' DFTs, evaluated with FFTs.  Worked out with unitary F (our reading of the printed
derivation, whose first-row / transpose / convolution bookkeeping is garbled):

    k_c[kappa] = sum_l r[l] g[l - kappa],    g = sum_i |DFT(s_i)|^2 / N^2,

with DFT the unnormalised transform and indices taken modulo the grid, i.e.
k_c = IDFT( DFT(r) * conj(DFT(g)) ) with IDFT including its 1/N.  ``k_diag_dense`` writes the
definition diag(F A F^H) out for tiny grids and the tests pin the two together.

k_d is the DFT of t_1, the first row of D_x^H D_x + D_y^H D_y (the stencil 2*ndim at the origin,
-1 at the 2*ndim periodic neighbours); k_w = 1.
Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import fourier, operators


def k_c(sens: np.ndarray, mask: np.ndarray, ndim: int) -> np.ndarray:
    """Diagonal of K_c = sum_i F S_i^H F^H R^H R F S_i F^H, by FFTs (Eq. diagonalelements)."""
    axes = tuple(range(-ndim, 0))
    n = mask.size
    s_hat = np.fft.fftn(sens, axes=axes)                       # unnormalised DFT of each s_i
    g = np.sum(np.abs(s_hat) ** 2, axis=0) / float(n) ** 2     # sum over coils
    r = mask.astype(np.float64)
    corr = np.fft.ifftn(np.fft.fftn(r) * np.conj(np.fft.fftn(g)))
    return corr.real


def first_row_tv(shape: tuple[int, ...]) -> np.ndarray:
    """t_1: the row of D_x^H D_x + D_y^H D_y (+ D_z^H D_z) belonging to pixel 0, as an image."""
    ndim = len(shape)
    e0 = np.zeros(shape)
    e0[(0,) * ndim] = 1.0
    # D^H D is real symmetric, so its first row equals its first column, (D^H D) e_0.
    return operators.tv_normal(e0, ndim)


def k_d(shape: tuple[int, ...]) -> np.ndarray:
    """k_d = DFT(t_1) (unnormalised DFT of a first row gives the eigenvalues of a BCCB matrix)."""
    return np.fft.fftn(first_row_tv(shape)).real


def k_diag(sens, mask, mu, lam, gam, ndim) -> np.ndarray:
    """k = mu k_c + lambda k_d + gamma k_w, k_w = 1 (Eq. Kdiag)."""
    return mu * k_c(sens, mask, ndim) + lam * k_d(mask.shape) + gam * np.ones(mask.shape)


def k_diag_dense(sens, mask, mu, lam, gam, ndim) -> np.ndarray:
    """The definition: diag(F A F^H) with dense F and A (tiny grids only)."""
    a = operators.dense_A(sens, mask, mu, lam, gam, ndim)
    f = fourier.dense_F(mask.shape)
    return np.real(np.diag(f @ a @ f.conj().T)).reshape(mask.shape)


def clamp_k(k: np.ndarray) -> np.ndarray:
    """Guard against a vanishing diagonal (never triggered when mu > 0 with a non-empty mask
    and lambda > 0 or gamma > 0): entries below 1e-12 * max(k) are raised to that floor."""
    floor = 1e-12 * float(np.max(k))
    return np.maximum(k, floor)


def apply_precond(r: np.ndarray, k: np.ndarray, ndim: int) -> np.ndarray:
    """M^{-1} r = F^H diag{k}^{-1} F r (Eq. precon): two FFTs and one diagonal scaling."""
    return fourier.ifft(fourier.fft(r, ndim) / k, ndim)


def jacobi_diag(sens, mask, mu, lam, gam, ndim) -> np.ndarray:
    """diag(A), the Jacobi preconditioner's diagonal (Preconditioning section).

    (S_i^H F^H R F S_i)_{jj} = |s_i[j]|^2 (F^H R F)_{jj} = |s_i[j]|^2 nnz(r)/N, and each
    D_a^H D_a contributes 2 on its diagonal."""
    frac = float(np.sum(mask)) / mask.size
    return (mu * frac * np.sum(np.abs(sens) ** 2, axis=0) + lam * 2.0 * ndim + gam).astype(np.float64)
