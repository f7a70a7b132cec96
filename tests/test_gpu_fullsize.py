"""Parity at the benchmark's full size and launch configuration: a batch of 64 slices of
256x256 with 12 coils (R = 4 lines, 24 centre lines, TV + 4-level Haar, mu = 1, lambda = gamma =
0.05, 20 Split Bregman iterations, PCG to relative residual 1e-3), reconstructed in one call with
the library's default concurrent slice groups.  Sampled slices are recomputed one by one by the
FP64 oracle.

With a tolerance-driven stop the two implementations may stop a solve one iteration apart when a
relative residual lands within rounding of 1e-3; so per-solve iteration counts are compared to
within one, and the images to within 1e-3 relative L2 (the PCG tolerance: a solve stopped one
iteration earlier or later differs by less than its own remaining error, and the following
warm-started solves do not amplify it).  Every slice of the batch must satisfy the property that
holds at any size: finite output and every solve converged.
"""
import numpy as np
import pytest

from oracle import split_bregman as sb_oracle
from paper_1710_01758_gb300 import synth

pytestmark = pytest.mark.gpu


def test_benchmark_batch_sampled_slices():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_01758_gb300 import sb

    wl = synth.METRIC_256
    B = 64
    slices = synth.make_batch(wl, B, wl.seed)   # the inputs bench.py times on rank 0
    sens = torch.from_numpy(np.stack([s.sens for s in slices])).to(torch.complex64).cuda()
    mask = torch.from_numpy(np.stack([s.mask for s in slices])).cuda()
    y = torch.from_numpy(np.stack([s.y for s in slices])).to(torch.complex64).cuda()
    x = torch.zeros((B, wl.ny, wl.nx), dtype=torch.complex64, device="cuda")
    plan = sb.Plan(wl.nx, wl.ny, wl.ncoils, B, wl.mu, wl.lam, wl.gam, wl.wavelet_levels)
    plan.set_coils(sens)
    plan.set_mask(mask)
    st, iters, last = plan.split_bregman(y, x, wl.n_outer, wl.n_inner, tol=wl.pcg_tol, maxit=wl.pcg_maxit)
    assert st == sb.SB_OK
    xg = x.cpu().numpy()
    assert np.all(np.isfinite(xg))
    assert all(r[2] and r[1] <= wl.pcg_tol for r in last)
    for i in (0, 37, B - 1):
        s = slices[i]
        ref = sb_oracle.split_bregman(s.y, s.sens, s.mask, wl.mu, wl.lam, wl.gam, wl.wavelet_levels, 2,
                                      wl.n_outer, wl.n_inner, wl.pcg_tol, wl.pcg_maxit)
        diffs = [a - b for a, b in zip(iters[i], ref.iters)]
        assert all(abs(d) <= 1 for d in diffs), (i, iters[i], ref.iters)
        err = float(np.linalg.norm(xg[i] - ref.x) / np.linalg.norm(ref.x))
        assert err <= 1e-3, (i, err, diffs)
    plan.close()
