"""Pins of the oracle's F, D, W, A and b against definitions, closed forms and invariants.

F: the unitary DFT of the Parallel Imaging paragraph (F^H F = I is used for Eq. K).
D: periodic first-order differences of the PI+CS paragraph.  W: a unitary (orthonormal Haar)
wavelet.  A and b: Eq. system.  None of these tests re-calls the function under test to make its
expected value.
"""
import numpy as np
import pytest

from oracle import fourier, operators
from paper_1710_01758_gb300 import synth


@pytest.mark.parametrize("shape", [(8, 8), (6, 10), (4, 6, 5)])
def test_fft_matches_naive_dft(shape, rng):
    x = synth.random_complex(shape, rng)
    ndim = len(shape)
    np.testing.assert_allclose(fourier.fft(x, ndim), fourier.dft_naive(x, ndim), atol=1e-12)
    np.testing.assert_allclose(fourier.ifft(fourier.fft(x, ndim), ndim), x, atol=1e-12)


def test_fft_sign_and_scale():
    # F applied to exp(+2 pi i k0 j / n) is sqrt(n) at k0 and 0 elsewhere (forward sign -).
    n, k0 = 12, 5
    j = np.arange(n)
    f = fourier.fft(np.exp(2j * np.pi * k0 * j / n), 1)
    expect = np.zeros(n, complex)
    expect[k0] = np.sqrt(n)
    np.testing.assert_allclose(f, expect, atol=1e-12)
    # a delta maps to the constant n^{-1/2}
    d = np.zeros(n)
    d[0] = 1
    np.testing.assert_allclose(fourier.fft(d, 1), np.full(n, 1 / np.sqrt(n)), atol=1e-14)


def test_dense_F_unitary(rng):
    f = fourier.dense_F((4, 6))
    np.testing.assert_allclose(f.conj().T @ f, np.eye(24), atol=1e-12)
    x = synth.random_complex((4, 6), rng)
    np.testing.assert_allclose((f @ x.ravel()).reshape(4, 6), fourier.fft(x, 2), atol=1e-12)


def test_difference_matches_paper_indexing(rng):
    # D_x(x)|_{i,j} = x_{i,j} - x_{i-1,j} (i = 2..m), x_{1,j} - x_{m,j} at i = 1; i runs along x.
    m, n = 7, 5                                   # m along x, n along y
    x = synth.random_complex((n, m), rng)         # C order: [y, x]
    dx = np.empty_like(x)
    dy = np.empty_like(x)
    for j in range(n):
        for i in range(m):
            dx[j, i] = x[j, i] - x[j, i - 1 if i > 0 else m - 1]
    for j in range(n):
        for i in range(m):
            dy[j, i] = x[j, i] - x[j - 1 if j > 0 else n - 1, i]
    gx, gy = operators.grad(x, 2)
    np.testing.assert_allclose(gx, dx, atol=0)
    np.testing.assert_allclose(gy, dy, atol=0)


@pytest.mark.parametrize("axis", [-1, -2, -3])
def test_difference_adjoint(axis, rng):
    x = synth.random_complex((4, 5, 6), rng)
    v = synth.random_complex((4, 5, 6), rng)
    lhs = np.vdot(operators.diff(x, axis), v)
    rhs = np.vdot(x, operators.diff_adj(v, axis))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("shape", [(8, 8), (6, 10), (4, 6, 8)])
def test_tv_normal_eigenvalues_closed_form(shape):
    # D^H D is BCCB: each Fourier mode is an eigenvector with eigenvalue
    # sum_a (2 - 2 cos(2 pi kappa_a / n_a)).
    ndim = len(shape)
    grids = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    for kappa in [(1,) * ndim, tuple(s // 2 for s in shape), tuple(range(1, ndim + 1))]:
        phase = sum(2 * np.pi * k * g / s for k, g, s in zip(kappa, grids, shape))
        mode = np.exp(1j * phase)
        eig = sum(2 - 2 * np.cos(2 * np.pi * k / s) for k, s in zip(kappa, shape))
        np.testing.assert_allclose(operators.tv_normal(mode, ndim), eig * mode, atol=1e-12)


def test_haar_2x2_hand_values():
    a, b, c, d = 1.0, 2.0, 4.0, 8.0
    x = np.array([[a, b], [c, d]])               # row y = 0 holds a, b
    w = operators.haar(x, 1, 2)
    expect = np.array([[(a + b + c + d) / 2, (a - b + c - d) / 2],
                       [(a + b - c - d) / 2, (a - b - c + d) / 2]])
    np.testing.assert_allclose(w, expect, atol=1e-15)


@pytest.mark.parametrize("shape,levels", [((8, 8), 3), ((16, 8), 2), ((4, 4, 4), 2)])
def test_haar_orthonormal_dense(shape, levels):
    ndim = len(shape)
    wm = operators.dense_operator(lambda v: operators.haar(v, levels, ndim), shape).real
    n = wm.shape[0]
    np.testing.assert_allclose(wm.T @ wm, np.eye(n), atol=1e-14)
    np.testing.assert_allclose(wm @ wm.T, np.eye(n), atol=1e-14)
    wa = operators.dense_operator(lambda v: operators.haar_adj(v, levels, ndim), shape).real
    np.testing.assert_allclose(wa, wm.T, atol=1e-14)


def test_haar_constant_image():
    # a constant image has no detail; each 2D level multiplies the approximation by 2
    x = np.full((16, 16), 3.0)
    w = operators.haar(x, 4, 2)
    expect = np.zeros((16, 16))
    expect[0, 0] = 3.0 * 2 ** 4
    np.testing.assert_allclose(w, expect, atol=1e-12)


def _problem(rng, shape=(8, 10), nc=3, line=False):
    sens = synth.random_complex((nc,) + shape, rng)
    if line:
        mask = np.repeat((rng.random(shape[0]) < 0.5)[:, None], shape[1], 1).astype(np.uint8)
    else:
        mask = (rng.random(shape) < 0.4).astype(np.uint8)
    mask.flat[0] = 1
    return sens, mask


def test_A_data_term_matches_dense_matrix_formula(rng):
    # mu sum_i S_i^H F^H R F S_i with dense F from the DFT definition and diagonal S_i, R
    shape = (4, 6)
    sens, mask = _problem(rng, shape, nc=2)
    f = fourier.dense_F(shape)
    r = np.diag(mask.ravel().astype(float))
    a = sum(np.diag(s.ravel()).conj().T @ f.conj().T @ r @ f @ np.diag(s.ravel()) for s in sens)
    x = synth.random_complex(shape, rng)
    got = operators.apply_A(x, sens, mask, 1.0, 0.0, 0.0, 2)
    np.testing.assert_allclose(got.ravel(), a @ x.ravel(), atol=1e-12)


def test_A_self_adjoint(rng):
    sens, mask = _problem(rng)
    x = synth.random_complex(mask.shape, rng)
    y = synth.random_complex(mask.shape, rng)
    ax = operators.apply_A(x, sens, mask, 0.7, 0.3, 0.2, 2)
    ay = operators.apply_A(y, sens, mask, 0.7, 0.3, 0.2, 2)
    assert abs(np.vdot(ax, y) - np.vdot(x, ay)) < 1e-12 * abs(np.vdot(ax, y))


def test_A_hermitian_positive_definite(rng):
    sens, mask = _problem(rng, (8, 8), nc=2)
    a = operators.dense_A(sens, mask, 1.0, 0.05, 0.05, 2)
    np.testing.assert_allclose(a, a.conj().T, atol=1e-12)
    np.linalg.cholesky(a)                       # raises unless HPD
    assert np.min(np.linalg.eigvalsh(a)) > 0


def test_encode_adjoint_pair(rng):
    sens, mask = _problem(rng)
    x = synth.random_complex(mask.shape, rng)
    y = synth.random_complex(sens.shape, rng)
    lhs = np.vdot(operators.encode(x, sens, mask, 2), y)
    rhs = np.vdot(x, operators.encode_adj(y, sens, mask, 2))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("gam", [0.0, 0.3])
def test_normal_equations_match_split_objective(gam, rng):
    # A x = b is the stationarity condition of the l2 sub-problem of Algorithm 1:
    # J(x) = mu/2 sum_i ||R F S_i x - y_i||^2 + lam/2 sum_a ||D_a x - (d_a - b_a)||^2
    #        + gam/2 ||W x - (d_w - b_w)||^2.  Its directional derivative is Re<A x - b, v>.
    shape, levels = (8, 8), 2
    mu, lam = 0.8, 0.4
    sens, mask = _problem(rng, shape, nc=2)
    y = operators.encode(synth.random_complex(shape, rng), sens, mask, 2)
    d = [synth.random_complex(shape, rng) for _ in range(2)]
    bb = [synth.random_complex(shape, rng) for _ in range(2)]
    d_w, b_w = synth.random_complex(shape, rng), synth.random_complex(shape, rng)

    def J(x):
        v = mu / 2 * np.sum(np.abs(mask[None] * np.fft.fft2(sens * x, norm="ortho") - y) ** 2)
        for ax, dd, bv in zip([-1, -2], d, bb):
            v += lam / 2 * np.sum(np.abs(x - np.roll(x, 1, ax) - (dd - bv)) ** 2)
        if gam:
            v += gam / 2 * np.sum(np.abs(operators.haar(x, levels, 2) - (d_w - b_w)) ** 2)
        return v

    b = operators.rhs(y, sens, mask, mu, lam, gam, d, bb, d_w, b_w, levels, 2)
    x = synth.random_complex(shape, rng)
    g = operators.apply_A(x, sens, mask, mu, lam, gam, 2) - b
    for _ in range(4):
        v = synth.random_complex(shape, rng)
        eps = 1e-3
        fd = (J(x + eps * v) - J(x - eps * v)) / (2 * eps)
        assert abs(fd - np.real(np.vdot(g, v))) < 1e-7 * max(1.0, abs(fd))
