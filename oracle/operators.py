"""Operators of the PI+CS problem, written from the paper's definitions.

* D_x, D_y (and D_z for volumes): first-order differences with periodic boundaries, Theory,
  "Parallel Imaging Reconstruction with Compressed Sensing": D_x(x)|_{i,j} = x_{i,j} - x_{i-1,j}
  with x_{0,j} := x_{m,j}; i indexes the x direction.  In our C-ordered arrays x is the last axis.
* W: a unitary wavelet transform (same paragraph); two are provided: the orthonormal Haar
  transform (pairs (a, b) -> ((a+b)/sqrt 2, (a-b)/sqrt 2)) and the periodic Daubechies
  four-tap transform, the wavelet of the paper's experiments (Methods, "Reconstruction").  Both
  are multilevel, Mallat layout, along x then y (then z) on the low-pass corner at each level,
  real, and act on real and imaginary parts alike.
* A = mu sum_i (R F S_i)^H R F S_i + lambda (D_x^H D_x + D_y^H D_y) + gamma W^H W  (Eq. system).
* b = mu sum_i (R F S_i)^H y_i + lambda [D_x^H (d_x - b_x) + D_y^H (d_y - b_y)]
      + gamma W^H (d_w - b_w)                                                       (Eq. system).
Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import fourier

SQRT_HALF = np.sqrt(0.5)


# ----------------------------------------------------------------------------- differences
def diff(x: np.ndarray, axis: int) -> np.ndarray:
    """D_a x: x[..., i, ...] - x[..., i-1, ...] along ``axis``, periodic (index -1 wraps)."""
    return x - np.roll(x, 1, axis=axis)


def diff_adj(v: np.ndarray, axis: int) -> np.ndarray:
    """D_a^H v = v[i] - v[i+1] (the transpose of the real circulant D_a), periodic."""
    return v - np.roll(v, -1, axis=axis)


def image_axes(ndim: int) -> list[int]:
    """Axes of an image in the paper's order x, y (, z): x is the last array axis."""
    return [-1, -2, -3][:ndim]


def grad(x: np.ndarray, ndim: int) -> list[np.ndarray]:
    """[D_x x, D_y x (, D_z x)]."""
    return [diff(x, ax) for ax in image_axes(ndim)]


def grad_adj(vs: list[np.ndarray], ndim: int) -> np.ndarray:
    """D_x^H v_x + D_y^H v_y (+ D_z^H v_z)."""
    return sum(diff_adj(v, ax) for v, ax in zip(vs, image_axes(ndim)))


def tv_normal(x: np.ndarray, ndim: int) -> np.ndarray:
    """(D_x^H D_x + D_y^H D_y (+ D_z^H D_z)) x."""
    return sum(diff_adj(diff(x, ax), ax) for ax in image_axes(ndim))


# ----------------------------------------------------------------------------- Haar wavelet
def _haar_step(c: np.ndarray, axis: int) -> np.ndarray:
    a = np.take(c, np.arange(0, c.shape[axis], 2), axis=axis)
    b = np.take(c, np.arange(1, c.shape[axis], 2), axis=axis)
    return np.concatenate([(a + b) * SQRT_HALF, (a - b) * SQRT_HALF], axis=axis)


def _haar_step_inv(c: np.ndarray, axis: int) -> np.ndarray:
    h = c.shape[axis] // 2
    lo = np.take(c, np.arange(0, h), axis=axis)
    hi = np.take(c, np.arange(h, 2 * h), axis=axis)
    out = np.empty_like(c)
    idx_even = [slice(None)] * c.ndim
    idx_odd = [slice(None)] * c.ndim
    idx_even[axis] = slice(0, None, 2)
    idx_odd[axis] = slice(1, None, 2)
    out[tuple(idx_even)] = (lo + hi) * SQRT_HALF
    out[tuple(idx_odd)] = (lo - hi) * SQRT_HALF
    return out


def haar(x: np.ndarray, levels: int, ndim: int) -> np.ndarray:
    """W x: ``levels``-level orthonormal Haar, Mallat layout (low-pass in the leading corner)."""
    c = np.array(x, dtype=np.result_type(x, np.float64), copy=True)
    shape = list(c.shape[-ndim:])
    for _ in range(levels):
        if any(s % 2 for s in shape):
            raise ValueError("image size not divisible by 2^levels")
        sl = (Ellipsis,) + tuple(slice(0, s) for s in shape)
        sub = c[sl]
        for ax in image_axes(ndim):
            sub = _haar_step(sub, ax)
        c[sl] = sub
        shape = [s // 2 for s in shape]
    return c


def haar_adj(c: np.ndarray, levels: int, ndim: int) -> np.ndarray:
    """W^H c (= W^{-1} c, W being orthonormal): undo the levels coarsest first."""
    x = np.array(c, dtype=np.result_type(c, np.float64), copy=True)
    full = list(x.shape[-ndim:])
    shapes = []
    shape = list(full)
    for _ in range(levels):
        shapes.append(shape)
        shape = [s // 2 for s in shape]
    for shape in reversed(shapes):
        sl = (Ellipsis,) + tuple(slice(0, s) for s in shape)
        sub = x[sl]
        for ax in reversed(image_axes(ndim)):
            sub = _haar_step_inv(sub, ax)
        x[sl] = sub
    return x


# ----------------------------------------------------------------------------- Daubechies-4
# Daubechies' orthonormal four-tap scaling filter (two vanishing moments), from its closed form
# h = (1 + sqrt 3, 3 + sqrt 3, 3 - sqrt 3, 1 - sqrt 3) / (4 sqrt 2), and the wavelet filter
# g_m = (-1)^m h_{3-m}.  One periodic analysis step along an axis of even length n >= 4:
#   a[k] = sum_m h_m x[(2k + m) mod n],   d[k] = sum_m g_m x[(2k + m) mod n],   k < n/2,
# with a in the first half of the axis and d in the second (Mallat layout).
_S3 = np.sqrt(3.0)
D4_H = np.array([1.0 + _S3, 3.0 + _S3, 3.0 - _S3, 1.0 - _S3]) / (4.0 * np.sqrt(2.0))
D4_G = np.array([D4_H[3], -D4_H[2], D4_H[1], -D4_H[0]])


def _d4_step(c: np.ndarray, axis: int) -> np.ndarray:
    n = c.shape[axis]
    if n < 4 or n % 2:
        raise ValueError("Daubechies-4 needs an even band length >= 4")
    v = np.moveaxis(c, axis, -1)
    k2 = np.arange(0, n, 2)
    a = sum(D4_H[m] * v[..., (k2 + m) % n] for m in range(4))
    d = sum(D4_G[m] * v[..., (k2 + m) % n] for m in range(4))
    return np.moveaxis(np.concatenate([a, d], axis=-1), -1, axis)


def _d4_step_inv(c: np.ndarray, axis: int) -> np.ndarray:
    """Transpose of _d4_step (its inverse, the step being orthogonal): every coefficient pair
    (a[k], d[k]) is spread back onto x[(2k + m) mod n] with weights h_m, g_m."""
    n = c.shape[axis]
    v = np.moveaxis(c, axis, -1)
    a, d = v[..., : n // 2], v[..., n // 2:]
    out = np.zeros_like(v)
    k2 = np.arange(0, n, 2)
    for m in range(4):
        out[..., (k2 + m) % n] += D4_H[m] * a + D4_G[m] * d
    return np.moveaxis(out, -1, axis)


def daub4(x: np.ndarray, levels: int, ndim: int) -> np.ndarray:
    """W x with the ``levels``-level periodic Daubechies-4 transform, Mallat layout."""
    c = np.array(x, dtype=np.result_type(x, np.float64), copy=True)
    shape = list(c.shape[-ndim:])
    for _ in range(levels):
        sl = (Ellipsis,) + tuple(slice(0, s) for s in shape)
        sub = c[sl]
        for ax in image_axes(ndim):
            sub = _d4_step(sub, ax)
        c[sl] = sub
        shape = [s // 2 for s in shape]
    return c


def daub4_adj(c: np.ndarray, levels: int, ndim: int) -> np.ndarray:
    """W^H c for the Daubechies-4 transform (coarsest level undone first)."""
    x = np.array(c, dtype=np.result_type(c, np.float64), copy=True)
    shapes, shape = [], list(x.shape[-ndim:])
    for _ in range(levels):
        shapes.append(shape)
        shape = [s // 2 for s in shape]
    for shape in reversed(shapes):
        sl = (Ellipsis,) + tuple(slice(0, s) for s in shape)
        sub = x[sl]
        for ax in reversed(image_axes(ndim)):
            sub = _d4_step_inv(sub, ax)
        x[sl] = sub
    return x


def wavelet(x: np.ndarray, levels: int, ndim: int, kind: str = "haar") -> np.ndarray:
    """W x for ``kind`` in {'haar', 'daub4'}."""
    return daub4(x, levels, ndim) if kind == "daub4" else haar(x, levels, ndim)


def wavelet_adj(c: np.ndarray, levels: int, ndim: int, kind: str = "haar") -> np.ndarray:
    """W^H c for ``kind`` in {'haar', 'daub4'}."""
    return daub4_adj(c, levels, ndim) if kind == "daub4" else haar_adj(c, levels, ndim)


# ----------------------------------------------------------------------------- encoding
def encode(x: np.ndarray, sens: np.ndarray, mask: np.ndarray, ndim: int) -> np.ndarray:
    """R F S_i x for every coil i (Eq. ill0): [Nc, ...] k-space, zero off the mask."""
    return mask[None] * fourier.fft(sens * x[None], ndim)


def encode_adj(y: np.ndarray, sens: np.ndarray, mask: np.ndarray, ndim: int) -> np.ndarray:
    """sum_i (R F S_i)^H y_i = sum_i S_i^H F^H R^H y_i."""
    return np.sum(np.conj(sens) * fourier.ifft(mask[None] * y, ndim), axis=0)


def apply_A(x: np.ndarray, sens: np.ndarray, mask: np.ndarray, mu: float, lam: float,
            gam: float, ndim: int) -> np.ndarray:
    """A x with A = mu sum_i (R F S_i)^H R F S_i + lambda sum_a D_a^H D_a + gamma W^H W.

    W^H W = I for the unitary wavelet (Theory, "Structure of the System Matrix A"), so the
    wavelet term is gamma x and W is not applied here."""
    data = encode_adj(encode(x, sens, mask, ndim), sens, mask, ndim)
    return mu * data + lam * tv_normal(x, ndim) + gam * x


def rhs(y: np.ndarray, sens: np.ndarray, mask: np.ndarray, mu: float, lam: float, gam: float,
        d: list[np.ndarray], bb: list[np.ndarray], d_w, b_w, levels: int, ndim: int,
        kind: str = "haar") -> np.ndarray:
    """Right-hand side b of Eq. system (step 4 of Algorithm 1).  ``d``/``bb`` hold the TV
    auxiliary and Bregman variables per axis (x, y (, z)); ``d_w``/``b_w`` the wavelet ones
    (ignored when gamma == 0)."""
    b = mu * encode_adj(y, sens, mask, ndim)
    b = b + lam * grad_adj([dd - bv for dd, bv in zip(d, bb)], ndim)
    if gam != 0.0:
        b = b + gam * wavelet_adj(d_w - b_w, levels, ndim, kind)
    return b


# ----------------------------------------------------------------------------- dense tools
def dense_operator(apply, shape: tuple[int, ...]) -> np.ndarray:
    """Dense matrix of the linear map ``apply`` on C-ordered images of ``shape`` (column j =
    apply(e_j)).  Tiny grids only."""
    n = int(np.prod(shape))
    m = np.empty((n, n), np.complex128)
    for j in range(n):
        e = np.zeros(n, np.complex128)
        e[j] = 1.0
        m[:, j] = apply(e.reshape(shape)).ravel()
    return m


def dense_A(sens, mask, mu, lam, gam, ndim) -> np.ndarray:
    shape = mask.shape
    return dense_operator(lambda v: apply_A(v, sens, mask, mu, lam, gam, ndim), shape)
