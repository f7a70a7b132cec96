"""Pins of the oracle's helper functions that the other pins reach only through callers: each is
checked against a definition or hand values of its own (adjointness by inner products,
orthonormality, brute-force sums, hand-built stencils).  The DFT's sign and scale are pinned
against the library FFT in test_oracle_fourier_ops.py; here its unitarity and the Kronecker
assembly of the dense 2D matrix."""
import numpy as np
import pytest

from oracle import coil_compression, fourier, operators, precond

def cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def inner(a, b):
    return np.vdot(a, b)  # sum conj(a) b


@pytest.mark.parametrize("shape", [(6, 5), (4, 3, 5)])
def test_grad_adj_is_the_adjoint_of_grad(shape):
    rng = np.random.default_rng(1)
    ndim = len(shape)
    x = cplx(rng, shape)
    vs = [cplx(rng, shape) for _ in range(ndim)]
    lhs = sum(inner(g, v) for g, v in zip(operators.grad(x, ndim), vs))
    rhs = inner(x, operators.grad_adj(vs, ndim))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # the paper's x, y (, z) order: x is the last array axis
    assert operators.image_axes(2) == [-1, -2] and operators.image_axes(3) == [-1, -2, -3]


@pytest.mark.parametrize("kind,levels", [("haar", 2), ("daub4", 2), ("haar", 0)])
def test_wavelet_adj_inverts_wavelet(kind, levels):
    rng = np.random.default_rng(2)
    x = cplx(rng, (16, 16))
    c = operators.wavelet(x, levels, 2, kind)
    assert np.allclose(operators.wavelet_adj(c, levels, 2, kind), x, atol=1e-12)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) <= 1e-12 * np.linalg.norm(x)  # orthonormal


def test_clamp_k_floor():
    k = np.array([[0.0, 2.0], [1e-20, 5.0]])
    out = precond.clamp_k(k)
    assert out[0, 1] == 2.0 and out[1, 1] == 5.0
    assert out[0, 0] == pytest.approx(5e-12) and out[1, 0] == pytest.approx(5e-12)


def test_first_row_tv_hand_values():
    t = precond.first_row_tv((5, 6))
    expect = np.zeros((5, 6))
    expect[0, 0] = 4.0
    for i, j in [(0, 1), (0, 5), (1, 0), (4, 0)]:  # the four periodic neighbours of pixel 0
        expect[i, j] = -1.0
    assert np.array_equal(t, expect)
    t3 = precond.first_row_tv((4, 4, 4))
    assert t3[0, 0, 0] == 6.0 and np.count_nonzero(t3) == 7 and t3.sum() == 0.0


def test_covariance_brute_force():
    rng = np.random.default_rng(3)
    y = cplx(rng, (3, 4, 2))
    c = coil_compression.covariance(y)
    brute = np.zeros((3, 3), complex)
    for idx in np.ndindex(4, 2):
        v = y[(slice(None),) + idx]
        brute += np.outer(v, v.conj())
    assert np.allclose(c, brute, atol=1e-12)
    assert np.allclose(c, c.conj().T) and np.min(np.linalg.eigvalsh(c)) >= -1e-12


@pytest.mark.parametrize("n", [1, 4, 7])
def test_dft_matrix_definition_and_unitarity(n):
    F = fourier.dft_matrix(n)
    for k, j in {(0, 0), (min(1, n - 1), min(1, n - 1)), (n - 1, n - 1), (n - 1, 0)}:
        assert F[k, j] == pytest.approx(np.exp(-2j * np.pi * k * j / n) / np.sqrt(n))
    assert np.allclose(F.conj().T @ F, np.eye(n), atol=1e-12)


def test_dense_F_is_the_2d_transform():
    rng = np.random.default_rng(4)
    x = cplx(rng, (3, 4))
    F = fourier.dense_F((3, 4))
    assert np.allclose(F @ x.ravel(), fourier.dft_naive(x, 2).ravel(), atol=1e-12)
    assert np.allclose(F.conj().T @ F, np.eye(12), atol=1e-12)
