"""Pins of the oracle's circulant preconditioner (Eqs. K, Kdiag, precon, diagonalelements).

The FFT construction of k is pinned to the definition k = diag(F A F^H) by brute force on tiny
grids, to the closed form of k_d, and to the special cases the paper states: without
sensitivity encoding K is diagonal and M^{-1} = A^{-1} exactly (Structure of the System Matrix
section), full sampling with normalised sensitivities gives k_c = 1, and the trace identity.
"""
import numpy as np
import pytest

from oracle import operators, pcg, precond
from paper_1710_01758_gb300 import synth


def _sens(rng, nc, shape, normalise=False):
    s = synth.random_complex((nc,) + shape, rng)
    if normalise:
        s /= np.sqrt(np.sum(np.abs(s) ** 2, axis=0, keepdims=True))
    return s


@pytest.mark.parametrize("shape,kind", [((8, 8), "random"), ((6, 10), "random"),
                                        ((8, 8), "lines"), ((4, 4, 4), "random")])
def test_k_matches_dense_definition(shape, kind, rng):
    ndim = len(shape)
    sens = _sens(rng, 2, shape)
    if kind == "lines":
        mask = np.repeat((rng.random(shape[0]) < 0.5)[:, None], shape[1], 1).astype(np.uint8)
    else:
        mask = (rng.random(shape) < 0.4).astype(np.uint8)
    mask.flat[0] = 1
    mu, lam, gam = 0.9, 0.07, 0.03
    k_fft = precond.k_diag(sens, mask, mu, lam, gam, ndim)
    k_dense = precond.k_diag_dense(sens, mask, mu, lam, gam, ndim)
    np.testing.assert_allclose(k_fft, k_dense, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("shape", [(8, 8), (6, 10), (4, 6, 8)])
def test_k_d_closed_form(shape):
    grids = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    expect = sum(2 - 2 * np.cos(2 * np.pi * g / s) for g, s in zip(grids, shape))
    np.testing.assert_allclose(precond.k_d(shape), expect, atol=1e-12)


def test_constant_sensitivities_make_M_exact_inverse(rng):
    # S_i = s_i I with sum |s_i|^2 = 1: K is diagonal, k_c = r, and M^{-1} = A^{-1}.
    shape = (8, 12)
    s = synth.random_complex(3, rng)
    s /= np.linalg.norm(s)
    sens = s[:, None, None] * np.ones((3,) + shape)
    mask = (rng.random(shape) < 0.3).astype(np.uint8)
    mu, lam, gam = 1.0, 0.05, 0.02
    np.testing.assert_allclose(precond.k_c(sens, mask, 2), mask, atol=1e-12)
    k = precond.k_diag(sens, mask, mu, lam, gam, 2)
    b = synth.random_complex(shape, rng)
    x = precond.apply_precond(b, k, 2)
    np.testing.assert_allclose(operators.apply_A(x, sens, mask, mu, lam, gam, 2), b, atol=1e-11)
    res = pcg.pcg(lambda v: operators.apply_A(v, sens, mask, mu, lam, gam, 2), b,
                  np.zeros(shape, complex), lambda v: precond.apply_precond(v, k, 2), tol=1e-10)
    assert res.converged and res.iters == 1


def test_full_sampling_gives_unit_k_c(rng):
    shape = (10, 8)
    sens = _sens(rng, 4, shape, normalise=True)
    mask = np.ones(shape, np.uint8)
    np.testing.assert_allclose(precond.k_c(sens, mask, 2), np.ones(shape), atol=1e-12)


def test_k_c_trace_identity_and_positivity(rng):
    # sum_kappa k_c = trace(K_c) = trace(A_c) = nnz(r)/N * sum_j sum_i |S_ij|^2
    shape = (16, 12)
    sens = _sens(rng, 3, shape)
    mask = (rng.random(shape) < 0.3).astype(np.uint8)
    kc = precond.k_c(sens, mask, 2)
    expect = mask.sum() / mask.size * np.sum(np.abs(sens) ** 2)
    assert abs(kc.sum() - expect) < 1e-10 * expect
    assert np.all(kc > -1e-12)
    k = precond.k_diag(sens, mask, 1.0, 0.05, 0.05, 2)
    assert np.all(k > 0)


def test_jacobi_diag_matches_dense(rng):
    shape = (6, 8)
    sens = _sens(rng, 2, shape)
    mask = (rng.random(shape) < 0.5).astype(np.uint8)
    a = operators.dense_A(sens, mask, 0.8, 0.1, 0.05, 2)
    np.testing.assert_allclose(precond.jacobi_diag(sens, mask, 0.8, 0.1, 0.05, 2).ravel(),
                               np.real(np.diag(a)), atol=1e-12)
