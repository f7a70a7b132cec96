"""The uneven batch (slices of different sizes, coil counts and accelerations): one plan per
geometry, all reconstructed concurrently by sb_split_bregman_many, against the FP64 oracle and
against each plan run on its own."""
import collections

import numpy as np
import pytest

from oracle import split_bregman as sb_oracle
from paper_1710_01758_gb300 import synth

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def build(torch, sb, wls, idx):
    """Plans (one per (nx, ny, ncoils)), their device inputs, and the slice list per plan."""
    groups = collections.defaultdict(list)
    for i in idx:
        groups[(wls[i].nx, wls[i].ny, wls[i].ncoils)].append(i)
    plans, ys, members, keep = [], [], [], []
    for (nx, ny, nc), ids in sorted(groups.items()):
        sl = [synth.uneven_slice(wls, i) for i in ids]
        w = wls[ids[0]]
        stream = torch.cuda.Stream()
        plan = sb.Plan(nx, ny, nc, len(ids), w.mu, w.lam, w.gam, w.wavelet_levels, stream=stream)
        sens = torch.from_numpy(np.stack([s.sens for s in sl])).to(torch.complex64).cuda()
        mask = torch.from_numpy(np.stack([s.mask for s in sl])).cuda()
        torch.cuda.synchronize()  # the plan works on its own stream
        plan.set_coils(sens)
        plan.set_mask(mask)
        keep.append(sens)
        ys.append(torch.from_numpy(np.stack([s.y for s in sl])).to(torch.complex64).cuda())
        plans.append(plan)
        members.append((ids, sl))
    torch.cuda.synchronize()
    return plans, ys, members, keep


def test_uneven_batch_concurrent_plans(torch):
    from paper_1710_01758_gb300 import sb
    wls = synth.uneven_workloads()
    idx = list(range(12))
    plans, ys, members, _keep = build(torch, sb, wls, idx)
    assert len(plans) >= 4
    n_outer, fixed, tau = 3, 6, 0.02
    xs = [torch.zeros((p.nbatch,) + p.shape[1:], dtype=torch.complex64, device="cuda") for p in plans]
    torch.cuda.synchronize()
    st, iters, _ = sb.split_bregman_many(plans, ys, xs, n_outer, tau_tv=tau, tau_w=tau, fixed_iters=fixed)
    assert st == sb.SB_OK
    assert all(all(all(k == fixed for k in row) for row in it) for it in iters)
    # each plan alone gives bit-identical images
    for p, y, x in zip(plans, ys, xs):
        x1 = torch.zeros_like(x)
        torch.cuda.synchronize()
        st1, _, _ = p.split_bregman(y, x1, n_outer, tau_tv=tau, tau_w=tau, fixed_iters=fixed)
        assert st1 == sb.SB_OK
        assert torch.equal(x1, x)
    # sampled slices against the oracle: the first slice of every size present
    seen = set()
    for (ids, sl), x in zip(members, xs):
        w = wls[ids[0]]
        if (w.nx, w.ny) in seen:
            continue
        seen.add((w.nx, w.ny))
        s = sl[0]
        ref = sb_oracle.split_bregman(s.y, s.sens, s.mask, w.mu, w.lam, w.gam, w.wavelet_levels, 2, n_outer,
                                      1, w.pcg_tol, w.pcg_maxit, fixed, "circulant", tau, tau)
        assert rel(x[0].cpu().numpy(), ref.x) <= IMG_TOL, w.name
    assert len(seen) >= 3
    with pytest.raises(sb.SbError) as ei:
        sb.split_bregman_many([plans[0], plans[0]], [ys[0], ys[0]], [xs[0], xs[0]], 1, fixed_iters=2)
    assert ei.value.status == sb.SB_ERR_INVALID_ARG
    for p in plans:
        p.close()
