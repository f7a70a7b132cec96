"""FP64 CPU oracle for the circulant-preconditioned PCG inside Split Bregman
(arXiv 1710.01758, "Accelerating CS in Parallel Imaging Reconstructions Using an Efficient and
Effective Circulant Preconditioner").

TEST INFRASTRUCTURE ONLY.  This package is imported solely by ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of ``bench.py``.  The product
path (the CUDA library and its Python binding) never imports, links or executes anything here,
and nothing here imports the product path.  The two share no code; only the seeded synthetic
input generators feed both.

Everything is plain numpy in complex128 / float64, written step by step in the paper's order and
notation.  numpy's FFT serves as the library DFT primitive; ``fourier.dft_matrix`` writes the
definition out and the tests pin the one to the other.

Modules:
  fourier        unitary DFT F (the paper's Parallel Imaging section; F^H F = I is used in the
                 derivation of Eq. K)
  operators      D_x, D_y (finite differences with periodic boundaries), the orthonormal Haar and
                 Daubechies-4 W,
                 the system matrix A of Eq. system, the right-hand side b, dense tiny-grid tools
  precond        k = mu k_c + lambda k_d + gamma k_w (Eq. Kdiag) built by FFTs (Eq.
                 diagonalelements), its dense definition diag(F A F^H), M^{-1} (Eq. precon),
                 the Jacobi diagonal
  pcg            textbook preconditioned CG (the Complexity section)
  split_bregman  Algorithm 1 (Split Bregman Iteration), shrink, root-sum-of-squares start
  coil_compression  principal-component coil compression (Methods, "Coil Compression")

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py`` except the
paper's own iteration counts (they exist only in figures that are not in the text): parity
unpinned for those.
"""
from . import coil_compression, fourier, operators, precond, pcg, split_bregman  # noqa: F401
