"""GPU parity of the split-precision modes (the radix-16 and radix-32 DFT stages of q = A p on the tensor cores,
operands split in two bf16 or fp16 terms, FP32 accumulation) against the FP64 oracle.

Stated tolerances, per mode (relative L2):
  split-fp16: one operator application <= 1e-5, a fixed PCG / Split Bregman schedule <= 1e-4
              (the FP32 bars: the two fp16 terms carry 22 significant bits);
  split-bf16: one operator application <= 1e-4, a fixed schedule <= 1e-3 (16 significant bits).
"""
import dataclasses

import numpy as np
import pytest

from oracle import operators, pcg, precond, split_bregman as sb_oracle
from paper_1710_01758_gb300 import synth

pytestmark = pytest.mark.gpu

MODES = {"fp16": (2, 1e-5, 1e-4), "bf16": (1, 1e-4, 1e-3)}  # prec, operator tol, image tol


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def sbm(torch):
    from paper_1710_01758_gb300 import sb
    return sb


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(torch, a):
    dt = torch.complex64 if np.iscomplexobj(a) else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()


def problem(nx, ny, nc, nb, seed, accel=4.0, n_centre=24):
    rng = np.random.default_rng(seed)
    sens = np.stack([synth.coil_maps(ny, nx, nc, rng) for _ in range(nb)])
    mask = np.stack([synth.line_mask(ny, nx, accel, n_centre, rng) for _ in range(nb)])
    return sens, mask, rng


def make_plan(sbm, torch, sens, mask, mu, lam, gam, prec, levels=0):
    nb, nc, ny, nx = sens.shape
    plan = sbm.Plan(nx, ny, nc, nb, mu, lam, gam, levels, prec=prec)
    plan.set_coils(to_dev(torch, sens))
    plan.set_mask(torch.from_numpy(mask).cuda())
    return plan


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("nx,ny,nc,nb", [(256, 256, 12, 2), (64, 256, 3, 3), (512, 256, 4, 1), (32, 256, 1, 2),
                                         (512, 512, 6, 1), (64, 512, 3, 2), (192, 512, 2, 1)])
def test_split_apply_A(torch, sbm, mode, nx, ny, nc, nb):
    prec, op_tol, _ = MODES[mode]
    sens, mask, rng = problem(nx, ny, nc, nb, seed=nx + ny + nc, n_centre=32 if ny == 512 else 24)
    mu, lam, gam = 1.0, 0.05, 0.05
    plan = make_plan(sbm, torch, sens, mask, mu, lam, gam, prec)
    x = synth.random_complex((nb, ny, nx), rng)
    q = plan.apply_A(to_dev(torch, x)).cpu().numpy()
    for b in range(nb):
        ref = operators.apply_A(x[b], sens[b], mask[b], mu, lam, gam, 2)
        assert rel(q[b], ref) <= op_tol, (mode, b, rel(q[b], ref))
    # the data term alone (lambda = gamma = 0), where the tensor-core stages are all of A
    plan0 = make_plan(sbm, torch, sens, mask, mu, 0.0, 0.0, prec)
    q0 = plan0.apply_A(to_dev(torch, x)).cpu().numpy()
    for b in range(nb):
        ref = operators.apply_A(x[b], sens[b], mask[b], mu, 0.0, 0.0, 2)
        assert rel(q0[b], ref) <= op_tol, (mode, b, rel(q0[b], ref))


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("ny", [256, 512])
def test_split_scale_invariance_and_zero(torch, sbm, mode, ny):
    """A is linear: A (2^-70 x) and A (2^60 x) are 2^-70 A x and 2^60 A x to the same tolerance
    (fp16 keeps its range by exact power-of-two scaling of each tile), and A 0 = 0."""
    prec, op_tol, _ = MODES[mode]
    nx, nc, nb = 64, 4, 2
    sens, mask, rng = problem(nx, ny, nc, nb, seed=9)
    mu = 1.0
    plan = make_plan(sbm, torch, sens, mask, mu, 0.0, 0.0, prec)
    x = synth.random_complex((nb, ny, nx), rng)
    for f in (2.0 ** -70, 2.0 ** 60):
        q = plan.apply_A(to_dev(torch, x * f)).cpu().numpy().astype(np.complex128) / f
        for b in range(nb):
            ref = operators.apply_A(x[b], sens[b], mask[b], mu, 0.0, 0.0, 2)
            assert rel(q[b], ref) <= op_tol, (f, b, rel(q[b], ref))
    z = plan.apply_A(to_dev(torch, np.zeros((nb, ny, nx), complex))).cpu().numpy()
    assert not np.any(z)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("nx,ny", [(128, 256), (64, 512)])
def test_split_pcg_fixed_iterations(torch, sbm, mode, nx, ny):
    prec, _, img_tol = MODES[mode]
    nc, nb = 6, 2
    sens, mask, rng = problem(nx, ny, nc, nb, seed=41)
    mu, lam, gam = 1.0, 0.05, 0.05
    plan = make_plan(sbm, torch, sens, mask, mu, lam, gam, prec)
    b = synth.random_complex((nb, ny, nx), rng)
    x0 = synth.random_complex((nb, ny, nx), rng) * 0.1
    xd = to_dev(torch, x0)
    st, res = plan.pcg_solve(to_dev(torch, b), xd, fixed_iters=12, precond=sbm.SB_PRECOND_CIRCULANT)
    assert st == sbm.SB_OK and all(r[0] == 12 for r in res)
    xg = xd.cpu().numpy()
    for i in range(nb):
        A = lambda v: operators.apply_A(v, sens[i], mask[i], mu, lam, gam, 2)  # noqa: E731
        k = precond.k_diag(sens[i], mask[i], mu, lam, gam, 2)
        ref = pcg.pcg(A, b[i], x0[i], lambda v: precond.apply_precond(v, k, 2), fixed_iters=12)
        assert rel(xg[i], ref.x) <= img_tol, (mode, i, rel(xg[i], ref.x))


@pytest.mark.parametrize("mode", list(MODES))
def test_split_bregman_metric_config(torch, sbm, mode):
    """The 256 x 256, 12-coil, TV + 4-level Haar workload, 20 Split Bregman iterations with a fixed
    schedule of 3 PCG iterations each, against the FP64 oracle."""
    prec, _, img_tol = MODES[mode]
    wl = synth.METRIC_256
    s = synth.make_slice(wl, wl.seed * 1000)
    plan = make_plan(sbm, torch, s.sens[None], s.mask[None], wl.mu, wl.lam, wl.gam, prec, wl.wavelet_levels)
    xd = torch.zeros((1, wl.ny, wl.nx), dtype=torch.complex64, device="cuda")
    st, _, _ = plan.split_bregman(to_dev(torch, s.y[None]), xd, wl.n_outer, wl.n_inner, fixed_iters=3,
                                  tol=wl.pcg_tol, maxit=wl.pcg_maxit)
    assert st == sbm.SB_OK
    ref = sb_oracle.split_bregman(s.y, s.sens, s.mask, wl.mu, wl.lam, wl.gam, wl.wavelet_levels, 2, wl.n_outer,
                                  wl.n_inner, wl.pcg_tol, wl.pcg_maxit, 3, "circulant", None, None)
    err = rel(xd.cpu().numpy()[0], ref.x)
    assert err <= img_tol, (mode, err)


def test_split_tolerance_run_matches_fp32_iteration_counts(torch, sbm):
    """PCG to 1e-3 in split-fp16 takes the FP32 mode's iteration counts (within one) on the metric
    workload's first solve."""
    wl = dataclasses.replace(synth.METRIC_256, n_outer=1)
    s = synth.make_slice(wl, wl.seed * 1000 + 1)
    its = {}
    for prec in (0, 2):
        plan = make_plan(sbm, torch, s.sens[None], s.mask[None], wl.mu, wl.lam, wl.gam, prec, wl.wavelet_levels)
        xd = torch.zeros((1, wl.ny, wl.nx), dtype=torch.complex64, device="cuda")
        st, iters, _ = plan.split_bregman(to_dev(torch, s.y[None]), xd, 1, 1, tol=wl.pcg_tol, maxit=wl.pcg_maxit)
        assert st == sbm.SB_OK
        its[prec] = np.asarray(iters).ravel()
    assert np.all(np.abs(its[0] - its[2]) <= 1), its


def test_split_unsupported(torch, sbm):
    for nx, ny in [(128, 128), (384, 384), (256, 320), (32, 192)]:  # the stages factor 256 and 512 only
        with pytest.raises(sbm.SbError) as ei:
            sbm.Plan(nx, ny, 2, 1, 1.0, 0.1, 0.1, 0, prec=sbm.SB_PREC_SPLIT_BF16)
        assert ei.value.status == sbm.SB_ERR_UNSUPPORTED
    with pytest.raises(sbm.SbError) as ei:
        sbm.Plan(64, 64, 2, 1, 1.0, 0.1, 0.1, 0, nz=64, prec=sbm.SB_PREC_SPLIT_FP16)
    assert ei.value.status == sbm.SB_ERR_UNSUPPORTED
    with pytest.raises(sbm.SbError) as ei:
        sbm.Plan(64, 256, 2, 1, 1.0, 0.1, 0.1, 0, prec=7)
    assert ei.value.status == sbm.SB_ERR_INVALID_ARG
    # a mask that varies along x needs the general (FP32) path
    nx, ny = 64, 256
    rng = np.random.default_rng(2)
    sens = synth.coil_maps(ny, nx, 2, rng)[None]
    mask = (rng.random((1, ny, nx)) < 0.3).astype(np.uint8)
    plan = sbm.Plan(nx, ny, 2, 1, 1.0, 0.1, 0.1, 0, prec=sbm.SB_PREC_SPLIT_FP16)
    plan.set_coils(to_dev(torch, sens))
    with pytest.raises(sbm.SbError) as ei:
        plan.set_mask(torch.from_numpy(mask).cuda())
    assert ei.value.status == sbm.SB_ERR_UNSUPPORTED
