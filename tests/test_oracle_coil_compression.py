"""Pins of the oracle's coil compression (Methods, "Coil Compression") against exact invariants:
a full-rank compression leaves A and b's data term unchanged, data confined to an r-dimensional
coil subspace lose nothing at r virtual coils, the kept energy is the sum of the largest
eigenvalues and no other projection of the same rank keeps more, and an independent SVD of the
stacked data gives the same subspace."""
import numpy as np
import pytest

from oracle import coil_compression as cc, operators
from paper_1710_01758_gb300 import synth


@pytest.fixture
def rng():
    return np.random.default_rng(11)


def problem(rng, nc=6, shape=(16, 16)):
    sens = synth.coil_maps(*shape, nc, rng)
    mask = synth.line_mask(*shape, 2.0, 4, rng)
    x = synth.ellipse_phantom(*shape, rng)
    y = synth.acquire(x, sens, mask, 1e-3, rng)
    return sens, mask, y


def test_full_rank_compression_is_exact(rng):
    sens, mask, y = problem(rng)
    A, _ = cc.compression_matrix(y, sens.shape[0])
    np.testing.assert_allclose(A @ A.conj().T, np.eye(A.shape[0]), atol=1e-12)
    yv, sv = cc.compress(y, sens, A)
    v = synth.random_complex(mask.shape, rng)
    np.testing.assert_allclose(operators.apply_A(v, sv, mask, 1.0, 0.1, 0.1, 2),
                               operators.apply_A(v, sens, mask, 1.0, 0.1, 0.1, 2), atol=1e-12)
    np.testing.assert_allclose(operators.encode_adj(yv, sv, mask, 2), operators.encode_adj(y, sens, mask, 2),
                               atol=1e-12)


def test_rank_r_data_lose_nothing(rng):
    # Nc = 8 coils that are mixtures of r = 3 underlying coils: 3 virtual coils carry everything
    base_s, mask, base_y = problem(rng, nc=3)
    M = synth.random_complex((8, 3), rng)
    sens = np.tensordot(M, base_s, axes=(1, 0))
    y = np.tensordot(M, base_y, axes=(1, 0))
    A, s = cc.compression_matrix(y, 3)
    assert s[3] < 1e-9 * s[0]
    yv, sv = cc.compress(y, sens, A)
    v = synth.random_complex(mask.shape, rng)
    np.testing.assert_allclose(operators.apply_A(v, sv, mask, 1.0, 0.0, 0.0, 2),
                               operators.apply_A(v, sens, mask, 1.0, 0.0, 0.0, 2), atol=1e-9)
    np.testing.assert_allclose(operators.encode_adj(yv, sv, mask, 2), operators.encode_adj(y, sens, mask, 2),
                               atol=1e-9 * np.abs(y).max())


def test_kept_energy_is_maximal(rng):
    _, _, y = problem(rng, nc=6)
    A, s = cc.compression_matrix(y, 2)
    Y = y.reshape(6, -1)
    kept = np.linalg.norm(A @ Y) ** 2
    assert abs(kept - s[:2].sum()) < 1e-9 * s.sum()
    for _ in range(50):
        Q, _ = np.linalg.qr(synth.random_complex((6, 2), rng))
        assert np.linalg.norm(Q.conj().T @ Y) ** 2 <= kept * (1 + 1e-12)


def test_subspace_matches_svd(rng):
    _, _, y = problem(rng, nc=5)
    A, _ = cc.compression_matrix(y, 3)
    U, _, _ = np.linalg.svd(y.reshape(5, -1), full_matrices=False)
    P_eig = A.conj().T @ A
    P_svd = U[:, :3] @ U[:, :3].conj().T
    np.testing.assert_allclose(P_eig, P_svd, atol=1e-10)
