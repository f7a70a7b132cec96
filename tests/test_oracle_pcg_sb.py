"""Pins of the oracle's PCG and Split Bregman (Complexity section; Algorithm 1).

PCG: finite termination on tiny systems, agreement with a dense direct solve, Jacobi = plain CG
when diag(A) is constant (the Results' observation that the system is invariant under scaling),
and the qualitative iteration reduction of the circulant preconditioner.
Split Bregman: shrink is the proximal map of t|.|; the inner loop converges to the minimiser of
the split objective (closed form for the orthonormal wavelet; first-order optimality for TV);
the outer loop recovers the image exactly from fully sampled noise-free data.
"""
import json
import os

import numpy as np
import pytest

from oracle import fourier, operators, pcg, precond, split_bregman as sb
from paper_1710_01758_gb300 import synth


def _problem(rng, shape, nc, frac=0.4, normalise=True):
    sens = synth.random_complex((nc,) + shape, rng)
    if normalise:
        sens /= np.sqrt(np.sum(np.abs(sens) ** 2, axis=0, keepdims=True))
    mask = (rng.random(shape) < frac).astype(np.uint8)
    mask.flat[0] = 1
    return sens, mask


def test_cg_terminates_within_n_steps(rng):
    shape = (4, 4)                                         # N = 16 unknowns
    sens, mask = _problem(rng, shape, 2)
    A = lambda v: operators.apply_A(v, sens, mask, 1.0, 0.05, 0.05, 2)  # noqa: E731
    b = synth.random_complex(shape, rng)
    res = pcg.pcg(A, b, np.zeros(shape, complex), tol=1e-10, maxit=16)
    assert res.converged and res.iters <= 16
    assert np.linalg.norm(b - A(res.x)) <= 1e-10 * np.linalg.norm(b)


def test_pcg_matches_direct_solve(rng):
    shape = (8, 8)
    sens, mask = _problem(rng, shape, 3)
    mu, lam, gam = 1.0, 0.05, 0.05
    a = operators.dense_A(sens, mask, mu, lam, gam, 2)
    b = synth.random_complex(shape, rng)
    k = precond.k_diag(sens, mask, mu, lam, gam, 2)
    res = pcg.pcg(lambda v: operators.apply_A(v, sens, mask, mu, lam, gam, 2), b,
                  synth.random_complex(shape, rng), lambda v: precond.apply_precond(v, k, 2),
                  tol=1e-13, maxit=200)
    np.testing.assert_allclose(res.x.ravel(), np.linalg.solve(a, b.ravel()), atol=1e-10)


def test_fixed_iters_and_zero_rhs(rng):
    shape = (8, 8)
    sens, mask = _problem(rng, shape, 2)
    A = lambda v: operators.apply_A(v, sens, mask, 1.0, 0.05, 0.05, 2)  # noqa: E731
    res = pcg.pcg(A, synth.random_complex(shape, rng), np.zeros(shape, complex), fixed_iters=7)
    assert res.iters == 7
    z = pcg.pcg(A, np.zeros(shape, complex), synth.random_complex(shape, rng))
    assert z.iters == 0 and not np.any(z.x)


def test_jacobi_equals_plain_cg_for_normalised_coils(rng):
    # sum_i |S_i|^2 = 1 makes diag(A) = mu nnz(r)/N + 4 lam + gam constant: Jacobi only rescales
    # the residual, so the PCG iterates coincide with plain CG.
    shape = (16, 16)
    sens, mask = _problem(rng, shape, 4)
    mu, lam, gam = 1.0, 0.05, 0.05
    A = lambda v: operators.apply_A(v, sens, mask, mu, lam, gam, 2)  # noqa: E731
    jd = precond.jacobi_diag(sens, mask, mu, lam, gam, 2)
    assert np.ptp(jd) < 1e-12
    b = synth.random_complex(shape, rng)
    x0 = np.zeros(shape, complex)
    plain = pcg.pcg(A, b, x0, None, tol=1e-6)
    jac = pcg.pcg(A, b, x0, lambda v: v / jd, tol=1e-6)
    assert plain.iters == jac.iters
    np.testing.assert_allclose(jac.x, plain.x, atol=1e-10)


def test_circulant_preconditioner_reduces_iterations():
    # Qualitative claims of the Results: with parameter set 1 (mu=1e-3, lambda=4e-3,
    # gamma=1e-3) the circulant preconditioner cuts the PCG iterations by a factor of about 5;
    # with set 2 (mu=1e-2) the gain is smaller (about threefold).
    wl = synth.Workload("t", 64, 64, 8, 4.0, 8, "uniform", 1.0, 0.05, 0.05, 3, 1, 1,
                        1e-3, 500, 0, seed=7)
    s = synth.make_slice(wl)
    b = operators.encode_adj(s.y, s.sens, s.mask, 2)
    x0 = np.zeros((64, 64), complex)
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                         "paper_results.json")))
    sets = golden["parameter_sets"]
    gains = []
    for mu, lam, gam in [tuple(sets[k][p] for p in ("mu", "lambda", "gamma"))
                         for k in ("set1", "set2")]:
        A = lambda v: operators.apply_A(v, s.sens, s.mask, mu, lam, gam, 2)  # noqa: E731
        k = precond.k_diag(s.sens, s.mask, mu, lam, gam, 2)
        plain = pcg.pcg(A, b, x0, None, tol=1e-3, maxit=500)
        pre = pcg.pcg(A, b, x0, lambda v: precond.apply_precond(v, k, 2), tol=1e-3, maxit=500)
        assert plain.converged and pre.converged
        gains.append(plain.iters / pre.iters)
    assert gains[0] >= 3.0 and gains[1] >= 1.5 and gains[0] > gains[1]


def test_shrink_is_prox_of_scaled_modulus(rng):
    z = synth.random_complex(200, rng)
    t = 0.8
    d = sb.shrink(z, t)
    obj = lambda v: t * np.abs(v) + 0.5 * np.abs(v - z) ** 2  # noqa: E731
    for _ in range(50):
        pert = 1e-3 * synth.random_complex(200, rng)
        assert np.all(obj(d) <= obj(d + pert) + 1e-15)
    np.testing.assert_allclose(np.abs(d), np.maximum(np.abs(z) - t, 0), atol=1e-15)
    big = np.abs(z) > t
    np.testing.assert_allclose(np.angle(d[big]), np.angle(z[big]), atol=1e-12)
    assert sb.shrink(np.zeros(3, complex), 1.0).tolist() == [0, 0, 0]


def test_rss_single_unit_coil():
    rng = np.random.default_rng(3)
    x = synth.random_complex((8, 8), rng)
    sens = np.exp(1j * rng.uniform(0, 6, (1, 8, 8)))
    y = fourier.fft(sens * x[None], 2)
    np.testing.assert_allclose(sb.rss(y, 2).real, np.abs(x), atol=1e-12)


def test_rss_several_coils_hand_values():
    """Step 1's root-sum-of-squares over several coils against values worked out by hand: coil
    images 3 and 4i give 5 (not 7 = |3| + |4i|, nor 25); images that differ per pixel combine per
    pixel; three constant coils 1, 2, -2 give 3."""
    shape = (4, 4)
    u = np.zeros((2,) + shape, complex)
    u[0] = 3.0
    u[1] = 4.0j
    np.testing.assert_allclose(sb.rss(fourier.fft(u, 2), 2).real, np.full(shape, 5.0), atol=1e-12)
    u = np.zeros((2,) + shape, complex)
    u[0, 0, 0], u[1, 0, 0] = 3.0, -4.0      # pixel (0, 0): sqrt(9 + 16) = 5
    u[1, 2, 1] = 1.0 - 1.0j                 # pixel (2, 1): sqrt(2), only coil 1
    u[0, 3, 3], u[1, 3, 3] = 0.6j, 0.8      # pixel (3, 3): sqrt(0.36 + 0.64) = 1
    want = np.zeros(shape)
    want[0, 0], want[2, 1], want[3, 3] = 5.0, np.sqrt(2.0), 1.0
    got = sb.rss(fourier.fft(u, 2), 2)
    np.testing.assert_allclose(got.real, want, atol=1e-12)
    np.testing.assert_allclose(got.imag, 0.0, atol=0)
    u = np.stack([np.full(shape, 1.0 + 0j), np.full(shape, 2.0 + 0j), np.full(shape, -2.0 + 0j)])
    np.testing.assert_allclose(sb.rss(fourier.fft(u, 2), 2).real, np.full(shape, 3.0), atol=1e-12)


def _denoise_setup(rng, shape=(16, 16)):
    x_true = synth.random_complex(shape, rng)
    sens = np.ones((1,) + shape, complex)
    mask = np.ones(shape, np.uint8)
    y = fourier.fft(x_true[None], 2)
    return x_true, sens, mask, y


def test_sb_wavelet_denoising_closed_form(rng):
    # Full sampling, one unit coil, no TV: the split problem is
    #   min_x mu/2 ||F x - y||^2 + ||W x||_1,
    # solved in closed form by x = W^H shrink(W F^H y, 1/mu) for unitary F and W.
    x_true, sens, mask, y = _denoise_setup(rng)
    mu, gam, levels = 2.0, 1.0, 2
    res = sb.split_bregman(y, sens, mask, mu, 0.0, gam, levels, 2, n_outer=1, n_inner=150,
                           pcg_tol=1e-12, pcg_maxit=50, x0=np.zeros((16, 16), complex))
    u = fourier.ifft(y[0], 2)
    expect = operators.haar_adj(sb.shrink(operators.haar(u, levels, 2), 1 / mu), levels, 2)
    np.testing.assert_allclose(res.x, expect, atol=1e-8)


def test_sb_tv_denoising_is_optimal(rng):
    # Full sampling, one unit coil, no wavelet: the inner loop converges to the minimiser of
    #   E(x) = mu/2 ||x - F^H y||^2 + ||D_x x||_1 + ||D_y x||_1  (complex modulus, anisotropic).
    x_true, sens, mask, y = _denoise_setup(rng, (12, 12))
    mu, lam = 1.5, 1.0
    res = sb.split_bregman(y, sens, mask, mu, lam, 0.0, 0, 2, n_outer=1, n_inner=600,
                           pcg_tol=1e-13, pcg_maxit=200, x0=np.zeros((12, 12), complex))
    u = fourier.ifft(y[0], 2)

    def E(x):
        return (mu / 2 * np.sum(np.abs(x - u) ** 2)
                + np.sum(np.abs(x - np.roll(x, 1, -1))) + np.sum(np.abs(x - np.roll(x, 1, -2))))

    e0 = E(res.x)
    assert e0 < E(u) and e0 < E(np.zeros_like(u))
    for eps in (1e-2, 1e-3):
        for _ in range(40):
            v = synth.random_complex(u.shape, rng)
            assert e0 <= E(res.x + eps * v / np.linalg.norm(v)) + 1e-7


def test_sb_exact_recovery_fully_sampled():
    # Fully sampled, noise-free, single coil S = 1: the Bregman add-back (steps 12-14) drives x
    # to the solution of min ||D x||_1 + ||W x||_1 subject to F x = y, which is the phantom itself.
    # Small shrink thresholds keep the l1 sub-problems active.
    rng = np.random.default_rng(11)
    shape = (32, 32)
    x_true = synth.ellipse_phantom(*shape, rng)
    sens = np.ones((1,) + shape, complex)
    mask = np.ones(shape, np.uint8)
    y = fourier.fft(x_true[None], 2)
    res = sb.split_bregman(y, sens, mask, 1.0, 0.05, 0.05, 2, 2, n_outer=60, pcg_tol=1e-12,
                           pcg_maxit=200, tau_tv=0.002, tau_w=0.002)
    err = np.linalg.norm(res.x - x_true) / np.linalg.norm(x_true)
    assert err <= 1e-6, err
