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
import functools

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


@pytest.mark.parametrize("prec,tol", [(2, 1e-3), (1, 2e-3)])
def test_benchmark_batch_split_precision_sampled_slice(prec, tol):
    """The same 64-slice batch in the split-precision modes (bench.py --prec split-fp16 /
    split-bf16): tensor-core DFT stages in every q = A p.  Slice 21 recomputed by the FP64
    oracle: iterations within one per solve, image within the PCG tolerance (split-fp16) or twice
    it (split-bf16, whose operator error is ~1e-5 relative)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_01758_gb300 import sb

    wl = synth.METRIC_256
    B = 64
    slices = synth.make_batch(wl, B, wl.seed)
    sens = torch.from_numpy(np.stack([s.sens for s in slices])).to(torch.complex64).cuda()
    mask = torch.from_numpy(np.stack([s.mask for s in slices])).cuda()
    y = torch.from_numpy(np.stack([s.y for s in slices])).to(torch.complex64).cuda()
    x = torch.zeros((B, wl.ny, wl.nx), dtype=torch.complex64, device="cuda")
    plan = sb.Plan(wl.nx, wl.ny, wl.ncoils, B, wl.mu, wl.lam, wl.gam, wl.wavelet_levels, prec=prec)
    plan.set_coils(sens)
    plan.set_mask(mask)
    st, iters, last = plan.split_bregman(y, x, wl.n_outer, wl.n_inner, tol=wl.pcg_tol, maxit=wl.pcg_maxit)
    assert st == sb.SB_OK
    xg = x.cpu().numpy()
    assert np.all(np.isfinite(xg)) and all(r[2] for r in last)
    i = 21
    ref = _oracle_recon(wl, slices[i])
    assert all(abs(a - b) <= 1 for a, b in zip(iters[i], ref.iters)), (iters[i], ref.iters)
    err = float(np.linalg.norm(xg[i] - ref.x) / np.linalg.norm(ref.x))
    assert err <= tol, err
    plan.close()


def test_volume_full_size_operators():
    """The 256 x 256 x 128 volume with 16 coils and (k_y, k_z) lines at R = 8 (24 x 24 centre):
    one application of A and of M^{-1}, and k, against the FP64 oracle over the whole volume."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import operators, precond
    from paper_1710_01758_gb300 import sb

    v = synth.VOLUME_256
    rng = np.random.default_rng(v.seed)
    sens = synth.coil_maps_3d(v.nz, v.ny, v.nx, v.ncoils, rng)
    mask = synth.readout_mask_3d(v.nz, v.ny, v.nx, v.accel, v.centre, rng)
    x = synth.random_complex((v.nz, v.ny, v.nx), rng)
    plan = sb.Plan(v.nx, v.ny, v.ncoils, 1, v.mu, v.lam, v.gam, v.wavelet_levels, nz=v.nz)
    d_sens = torch.from_numpy(sens[None].astype(np.complex64)).cuda()
    plan.set_coils(d_sens)
    plan.set_mask(torch.from_numpy(mask[None]).cuda())
    q = plan.apply_A(torch.from_numpy(x[None].astype(np.complex64)).cuda()).cpu().numpy()[0]
    z = plan.apply_precond(torch.from_numpy(x[None].astype(np.complex64)).cuda()).cpu().numpy()[0]
    kg = plan.k().cpu().numpy()[0]
    plan.close()
    del d_sens
    ref = operators.apply_A(x, sens, mask, v.mu, v.lam, v.gam, 3)
    assert np.linalg.norm(q - ref) / np.linalg.norm(ref) <= 1e-5
    kref = precond.k_diag(sens, mask, v.mu, v.lam, v.gam, 3)
    assert np.max(np.abs(kg - kref)) <= 1e-5 * np.max(kref)
    zref = precond.apply_precond(x, kref, 3)
    assert np.linalg.norm(z - zref) / np.linalg.norm(zref) <= 1e-5


def _oracle_recon(wl, s):
    return sb_oracle.split_bregman(s.y, s.sens, s.mask, wl.mu, wl.lam, wl.gam, wl.wavelet_levels, 2, wl.n_outer,
                                   wl.n_inner, wl.pcg_tol, wl.pcg_maxit)


@functools.lru_cache(maxsize=None)
def _large_512_reference(i):
    wl = synth.LARGE_512
    return _oracle_recon(wl, synth.make_batch(wl, 8, wl.seed)[i])


@pytest.mark.parametrize("prec,tol", [(0, 1e-3), (2, 1e-3), (1, 2e-3)])
def test_large_512_batch_sampled_slice(prec, tol):
    """512 x 512, 32 coils, R = 6 variable-density lines (the bench's --workload 512: 8 slices in
    one call), in FP32 and in the two split-precision modes (the precision sweep of this
    workload): slice 5 recomputed by the oracle; iterations within one per solve, image within
    the PCG tolerance (twice it for split-bf16)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_01758_gb300 import sb

    wl = synth.LARGE_512
    B = 8
    slices = synth.make_batch(wl, B, wl.seed)
    sens = torch.from_numpy(np.stack([s.sens for s in slices])).to(torch.complex64).cuda()
    mask = torch.from_numpy(np.stack([s.mask for s in slices])).cuda()
    y = torch.from_numpy(np.stack([s.y for s in slices])).to(torch.complex64).cuda()
    x = torch.zeros((B, wl.ny, wl.nx), dtype=torch.complex64, device="cuda")
    plan = sb.Plan(wl.nx, wl.ny, wl.ncoils, B, wl.mu, wl.lam, wl.gam, wl.wavelet_levels, prec=prec)
    plan.set_coils(sens)
    plan.set_mask(mask)
    st, iters, last = plan.split_bregman(y, x, wl.n_outer, wl.n_inner, tol=wl.pcg_tol, maxit=wl.pcg_maxit)
    assert st == sb.SB_OK
    xg = x.cpu().numpy()
    assert np.isfinite(xg).all() and all(r[2] for r in last)
    ref = _large_512_reference(5)
    assert all(abs(a - b) <= 1 for a, b in zip(iters[5], ref.iters)), (iters[5], ref.iters)
    assert np.linalg.norm(xg[5] - ref.x) / np.linalg.norm(ref.x) <= tol
    plan.close()


def test_uneven_batch_full_size_sampled_slices():
    """The 64-slice uneven batch (the bench's --workload uneven64): all geometries reconstructed
    concurrently with sb_split_bregman_many; one slice of each image size recomputed by the
    oracle, iterations within one per solve, images within the PCG tolerance."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import collections
    from paper_1710_01758_gb300 import sb

    wls = synth.uneven_workloads()
    groups = collections.defaultdict(list)
    for i, w in enumerate(wls):
        groups[(w.nx, w.ny, w.ncoils)].append(i)
    plans, ys, xs, keep, members = [], [], [], [], []
    for (nx, ny, nc), ids in sorted(groups.items()):
        sl = [synth.uneven_slice(wls, i) for i in ids]
        w = wls[ids[0]]
        s_ = torch.from_numpy(np.stack([s.sens for s in sl])).to(torch.complex64).cuda()
        m_ = torch.from_numpy(np.stack([s.mask for s in sl])).cuda()
        ys.append(torch.from_numpy(np.stack([s.y for s in sl])).to(torch.complex64).cuda())
        xs.append(torch.zeros((len(ids), ny, nx), dtype=torch.complex64, device="cuda"))
        torch.cuda.synchronize()
        p = sb.Plan(nx, ny, nc, len(ids), w.mu, w.lam, w.gam, w.wavelet_levels, stream=torch.cuda.Stream())
        p.set_coils(s_)
        p.set_mask(m_)
        keep.append(s_)
        plans.append(p)
        members.append((ids, sl))
    torch.cuda.synchronize()
    w0 = wls[0]
    st, iters, last = sb.split_bregman_many(plans, ys, xs, w0.n_outer, w0.n_inner, tol=w0.pcg_tol,
                                            maxit=w0.pcg_maxit)
    assert st == sb.SB_OK
    seen = set()
    for (ids, sl), x, it, la in zip(members, xs, iters, last):
        xg = x.cpu().numpy()
        assert np.isfinite(xg).all() and all(r[2] for r in la)
        w = wls[ids[0]]
        if (w.nx, w.ny) in seen:
            continue
        seen.add((w.nx, w.ny))
        ref = _oracle_recon(w, sl[0])
        assert all(abs(a - b) <= 1 for a, b in zip(it[0], ref.iters)), (w.name, it[0], ref.iters)
        assert np.linalg.norm(xg[0] - ref.x) / np.linalg.norm(ref.x) <= 1e-3, w.name
    assert len(seen) == 4
    for p in plans:
        p.close()
