"""Textbook preconditioned conjugate gradients (Theory, "Complexity"; Saad, cited there).

The paper states PCG as the left-preconditioned system M^{-1} A x = M^{-1} b with HPD A and
HPD M^{-1}; preconditioned CG with the M^{-1}-inner product is the standard way to run it and
produces the same iterates.  Readings:
  * residual r = b - A x (the paper writes A x - b; the sign is immaterial);
  * stop when ||b - A x||_2 / ||b||_2 <= tol on the recurrence-updated residual (the
    "relative residual norm" of the Methods' Reconstruction paragraph), tested before the first
    iteration and after every residual update;
  * Re() of the complex inner products;
  * the iteration count is the number of A applications after the initial residual;
  * ``fixed_iters`` > 0 runs exactly that many iterations with no test;
  * ||b|| = 0 returns x = 0.
Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class PcgResult:
    x: np.ndarray
    iters: int
    rel_resid: float
    converged: bool


def _dot(u: np.ndarray, v: np.ndarray) -> float:
    return float(np.real(np.vdot(u, v)))


def pcg(apply_A, b: np.ndarray, x0: np.ndarray, apply_M=None, tol: float = 1e-3,
        maxit: int = 1000, fixed_iters: int = 0) -> PcgResult:
    """Solve A x = b from x0.  ``apply_M`` applies M^{-1} (None: plain CG)."""
    if apply_M is None:
        apply_M = lambda v: v  # noqa: E731
    bnorm = np.sqrt(_dot(b, b))
    if bnorm == 0.0:
        return PcgResult(np.zeros_like(b), 0, 0.0, True)
    x = np.array(x0, np.complex128, copy=True)
    r = b - apply_A(x)
    rel = np.sqrt(_dot(r, r)) / bnorm
    if fixed_iters <= 0 and rel <= tol:
        return PcgResult(x, 0, rel, True)
    z = apply_M(r)
    p = z.copy()
    rho = _dot(r, z)
    n_iter = fixed_iters if fixed_iters > 0 else maxit
    for it in range(1, n_iter + 1):
        q = apply_A(p)
        pq = _dot(p, q)
        if rho == 0.0 or not pq > 0.0:
            # exact solution reached (rho = 0) or loss of positivity: nothing left to do
            return PcgResult(x, it - 1, rel, rel <= tol or rho == 0.0)
        alpha = rho / pq
        x = x + alpha * p
        r = r - alpha * q
        rel = np.sqrt(_dot(r, r)) / bnorm
        if fixed_iters <= 0 and rel <= tol:
            return PcgResult(x, it, rel, True)
        z = apply_M(r)
        rho_new = _dot(r, z)
        beta = rho_new / rho
        p = z + beta * p
        rho = rho_new
    return PcgResult(x, n_iter, rel, fixed_iters > 0 or rel <= tol)
