"""Split Bregman iteration (Algorithm 1) around the PCG solve of Eq. system.

Readings of Algorithm 1 (the printed superscripts mix the inner index k and the outer index j):
  * x, the auxiliary variables d_* and the Bregman variables b_* persist across outer and inner
    iterations; each inner iteration solves A x = b warm-started from the current x (step 5);
  * shrink(z, t) = z/|z| max(|z| - t, 0) with shrink(0, t) = 0, on the complex modulus,
    component-wise (anisotropic TV: separate d_x, d_y (, d_z));
  * thresholds are 1/lambda (TV) and 1/gamma (wavelet) as printed in steps 6-8 unless the
    caller overrides them; lambda and gamma act as splitting penalties, as in Algorithm 1;
  * the wavelet term is skipped entirely when gamma == 0, the TV term when lambda == 0;
    all wavelet coefficients are shrunk, the coarsest approximation band included;
  * "Sum of Squares" initialisation (step 1) is the root-sum-of-squares coil combination
    x = sqrt(sum_i |F^H y_i|^2) (real, non-negative);
  * the outer data update (steps 12-14) is y_i <- y_i + y_i^[1] - R F S_i x, R included, so
    unsampled k-space stays zero.
Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import fourier, operators, pcg, precond


def shrink(z: np.ndarray, t: float) -> np.ndarray:
    """z/|z| * max(|z| - t, 0), 0 where z = 0."""
    mag = np.abs(z)
    scale = np.where(mag > 0, np.maximum(mag - t, 0.0) / np.where(mag > 0, mag, 1.0), 0.0)
    return z * scale


def rss(y: np.ndarray, ndim: int) -> np.ndarray:
    """Root-sum-of-squares combination of the coil images F^H y_i."""
    return np.sqrt(np.sum(np.abs(fourier.ifft(y, ndim)) ** 2, axis=0)).astype(np.complex128)


@dataclasses.dataclass
class SbResult:
    x: np.ndarray
    iters: list[int]          # PCG iterations of every solve, in order
    rel_resid: list[float]    # final relative residual of every solve
    shrink_nonzero: list[float] = dataclasses.field(default_factory=list)  # per solve: fraction of
    # non-zero shrink outputs (TV d's and wavelet d_w together), a record of how active steps 6-8 are


def split_bregman(y, sens, mask, mu, lam, gam, levels, ndim, n_outer, n_inner=1,
                  pcg_tol=1e-3, pcg_maxit=1000, fixed_iters=0, precond_kind="circulant",
                  tau_tv=None, tau_w=None, x0=None, wavelet="haar") -> SbResult:
    """Algorithm 1.  ``precond_kind``: 'circulant' (Eq. precon), 'jacobi' or 'none'; ``wavelet``:
    'haar' or 'daub4' (the paper's)."""
    y = np.asarray(y, np.complex128)
    sens = np.asarray(sens, np.complex128)
    mask = np.asarray(mask)
    if tau_tv is None or tau_tv <= 0:
        tau_tv = 1.0 / lam if lam > 0 else np.inf
    if tau_w is None or tau_w <= 0:
        tau_w = 1.0 / gam if gam > 0 else np.inf

    def apply_A(v):
        return operators.apply_A(v, sens, mask, mu, lam, gam, ndim)

    if precond_kind == "circulant":
        k = precond.clamp_k(precond.k_diag(sens, mask, mu, lam, gam, ndim))
        apply_M = lambda v: precond.apply_precond(v, k, ndim)  # noqa: E731
    elif precond_kind == "jacobi":
        jd = precond.jacobi_diag(sens, mask, mu, lam, gam, ndim)
        apply_M = lambda v: v / jd  # noqa: E731
    elif precond_kind == "none":
        apply_M = None
    else:
        raise ValueError(precond_kind)

    # step 1: initialisation
    y1 = y.copy()
    yj = y.copy()
    x = rss(y, ndim) if x0 is None else np.array(x0, np.complex128, copy=True)
    zero = np.zeros(mask.shape, np.complex128)
    d = [zero.copy() for _ in range(ndim)]
    bb = [zero.copy() for _ in range(ndim)]
    d_w = zero.copy()
    b_w = zero.copy()
    iters, resid, active = [], [], []
    for _j in range(n_outer):                                   # step 2
        for _k in range(n_inner):                               # step 3
            b = operators.rhs(yj, sens, mask, mu, lam, gam, d, bb, d_w, b_w, levels, ndim, wavelet)  # 4
            res = pcg.pcg(apply_A, b, x, apply_M, pcg_tol, pcg_maxit, fixed_iters)          # 5
            x = res.x
            iters.append(res.iters)
            resid.append(res.rel_resid)
            if lam != 0.0:
                dx = operators.grad(x, ndim)
                d = [shrink(g + bv, tau_tv) for g, bv in zip(dx, bb)]                        # 6-7
                bb = [bv + g - dv for bv, g, dv in zip(bb, dx, d)]                           # 9-10
            if gam != 0.0:
                wx = operators.wavelet(x, levels, ndim, wavelet)
                d_w = shrink(wx + b_w, tau_w)                                                # 8
                b_w = b_w + wx - d_w                                                         # 11
            outs = (d if lam != 0.0 else []) + ([d_w] if gam != 0.0 else [])
            active.append(float(np.mean([np.count_nonzero(v) / v.size for v in outs])) if outs else 0.0)
        yj = yj + y1 - operators.encode(x, sens, mask, ndim)                                 # 12-14
    return SbResult(x, iters, resid, active)
