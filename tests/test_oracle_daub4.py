"""Pins of the oracle's Daubechies-4 wavelet (the wavelet of the paper's experiments, Methods,
"Reconstruction") against the filter's closed-form identities, textbook coefficient values,
orthogonality of the dense matrix, vanishing moments and a closed-form Split Bregman case.
None of these re-calls the function under test to make its expected value."""
import numpy as np
import pytest

from oracle import fourier, operators, split_bregman as sb
from paper_1710_01758_gb300 import synth

H = operators.D4_H
G = operators.D4_G


@pytest.fixture
def rng():
    return np.random.default_rng(4)


def test_filter_identities():
    # sum h = sqrt 2 (low-pass passes constants), unit energy, double-shift orthogonality;
    # the wavelet filter has two vanishing moments and is orthogonal to the scaling filter
    assert abs(H.sum() - np.sqrt(2.0)) < 1e-15
    assert abs((H ** 2).sum() - 1.0) < 1e-15
    assert abs(H[0] * H[2] + H[1] * H[3]) < 1e-15
    assert abs(G.sum()) < 1e-15
    assert abs((np.arange(4) * G).sum()) < 1e-15
    assert abs((G ** 2).sum() - 1.0) < 1e-15
    assert abs((H * G).sum()) < 1e-15 and abs(H[0] * G[2] + H[1] * G[3]) < 1e-15


def test_textbook_coefficients():
    # the published D4 coefficients (Daubechies 1988), to 15 digits
    np.testing.assert_allclose(H, [0.482962913144534, 0.836516303737808, 0.224143868042013,
                                   -0.129409522551260], atol=1e-14)


def test_one_step_hand_values():
    # x = e_0 (length 4): a[0] = h0, a[1] = h2 (x[(2 + 2) mod 4] = x[0]), d[0] = g0 = h3, d[1] = g2 = h1
    x = np.array([1.0, 0.0, 0.0, 0.0])
    w = operators.daub4(x, 1, 1)
    np.testing.assert_allclose(w, [0.482962913144534, 0.224143868042013, -0.129409522551260,
                                   0.836516303737808], atol=1e-14)


@pytest.mark.parametrize("shape,levels", [((16,), 3), ((8, 8), 2), ((8, 12), 1), ((8, 8, 8), 1)])
def test_dense_matrix_orthogonal(shape, levels):
    ndim = len(shape)
    wm = operators.dense_operator(lambda v: operators.daub4(v, levels, ndim), shape).real
    n = wm.shape[0]
    np.testing.assert_allclose(wm.T @ wm, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(wm @ wm.T, np.eye(n), atol=1e-13)
    wa = operators.dense_operator(lambda v: operators.daub4_adj(v, levels, ndim), shape).real
    np.testing.assert_allclose(wa, wm.T, atol=1e-13)


def test_adjoint_inverts_complex(rng):
    x = synth.random_complex((32, 64), rng)
    c = operators.daub4(x, 4, 2)
    np.testing.assert_allclose(operators.daub4_adj(c, 4, 2), x, atol=1e-12)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) < 1e-10 * np.linalg.norm(x)


def test_vanishing_moments_ramp():
    # a linear ramp has zero details wherever the filter window does not wrap (2k + 3 < n)
    n = 32
    x = np.arange(n, dtype=float) * 0.7 + 3.0
    w = operators.daub4(x, 1, 1)
    d = w[n // 2:]
    np.testing.assert_allclose(d[: n // 2 - 1], 0.0, atol=1e-12)
    assert abs(d[-1]) > 1.0  # the wrapping window sees the jump


def test_constant_image():
    x = np.full((32, 32), 0.5 + 0.25j)
    w = operators.daub4(x, 3, 2)
    expect = np.zeros_like(w)
    expect[:4, :4] = (0.5 + 0.25j) * 2.0 ** 3  # sqrt 2 per axis per level
    np.testing.assert_allclose(w, expect, atol=1e-13)


def test_differs_from_haar(rng):
    x = synth.random_complex((16, 16), rng)
    assert np.linalg.norm(operators.daub4(x, 2, 2) - operators.haar(x, 2, 2)) > 0.1


def test_sb_daub4_denoising_closed_form(rng):
    # full sampling, one unit coil, no TV: x = W^H shrink(W F^H y, 1/mu) with W = Daubechies-4
    x_true = synth.random_complex((16, 16), rng)
    sens = np.ones((1, 16, 16), complex)
    mask = np.ones((16, 16), np.uint8)
    y = fourier.fft(x_true[None], 2)
    mu, gam, levels = 2.0, 1.0, 2
    res = sb.split_bregman(y, sens, mask, mu, 0.0, gam, levels, 2, n_outer=1, n_inner=150, pcg_tol=1e-12,
                           pcg_maxit=50, x0=np.zeros((16, 16), complex), wavelet="daub4")
    u = fourier.ifft(y[0], 2)
    wd = operators.dense_operator(lambda v: operators.daub4(v, levels, 2), (16, 16)).real
    z = sb.shrink((wd @ u.ravel()), 1 / mu)
    expect = (wd.T @ z).reshape(16, 16)
    np.testing.assert_allclose(res.x, expect, atol=1e-8)
