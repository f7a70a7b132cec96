"""The bounded device waits run out into an error status, not a hang (failure detection).

Every wait of a coil-tile kernel for its TMA tile polls an mbarrier a bounded number of times.
Here the plan's coil-tile kernels withhold their tile requests (sb_set_wait_check), so nothing is
ever in flight and each wait gives up after a short poll limit: the solve must come back with
SB_ERR_TIMEOUT, the CUDA context must stay usable, and the same plan (check switched off again)
and a fresh plan must then reproduce the FP64 oracle.  Nothing faults and nothing waits forever.
"""
import numpy as np
import pytest

from oracle import operators, pcg, precond
from paper_1710_01758_gb300 import synth

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
IMG_TOL = 1e-4
SHORT_POLLS = 1024


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _problem(nx=128, ny=128, nc=4, nb=2, seed=4242):
    rng = np.random.default_rng(seed)
    sens = np.stack([synth.coil_maps(ny, nx, nc, rng) for _ in range(nb)])
    mask = np.stack([synth.line_mask(ny, nx, 4.0, 8, rng) for _ in range(nb)])
    return sens, mask, rng


def _plan(torch, sb, sens, mask, mu, lam, gam):
    nb, nc, ny, nx = sens.shape
    plan = sb.Plan(nx, ny, nc, nb, mu, lam, gam, 0)
    d_sens = torch.from_numpy(sens).to(torch.complex64).cuda()
    plan.set_coils(d_sens)
    plan.set_mask(torch.from_numpy(mask).cuda())
    return plan


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("nx,ny", [(128, 128), (64, 256)])
def test_withheld_tiles_give_timeout_and_context_survives(torch, nx, ny):
    from paper_1710_01758_gb300 import sb

    mu, lam, gam = 1.0, 0.05, 0.05
    sens, mask, rng = _problem(nx=nx, ny=ny)
    nb, nc, ny, nx = sens.shape
    b = synth.random_complex((nb, ny, nx), rng)
    d_b = torch.from_numpy(b).to(torch.complex64).cuda()

    plan = _plan(torch, sb, sens, mask, mu, lam, gam)
    plan.set_wait_check(SHORT_POLLS, withhold_coil_tiles=True)
    x = torch.zeros_like(d_b)
    st, _ = sb.sb_pcg_solve(plan.handle, d_b.data_ptr(), x.data_ptr(), sb.pcg_opts(fixed_iters=8), nb,
                            allow=(sb.SB_ERR_TIMEOUT,))
    assert st == sb.SB_ERR_TIMEOUT
    assert "bounded device wait" in sb._lib.sb_plan_last_error(sb._P(plan.handle)).decode()
    # Split Bregman (right-hand side kernel and PCG) reports the same
    y = torch.from_numpy(synth.random_complex((nb, nc, ny, nx), rng)).to(torch.complex64).cuda()
    st2, _, _ = sb.sb_split_bregman(plan.handle, y.data_ptr(), x.data_ptr(), 1, 1, sb.pcg_opts(fixed_iters=4), nb,
                                    allow=(sb.SB_ERR_TIMEOUT,))
    assert st2 == sb.SB_ERR_TIMEOUT
    torch.cuda.synchronize()  # the context is still usable: no sticky error

    # the same plan with the check off: a fixed PCG schedule matches the oracle again
    plan.set_wait_check(0, withhold_coil_tiles=False)
    x = torch.zeros_like(d_b)
    st3, _ = sb.sb_pcg_solve(plan.handle, d_b.data_ptr(), x.data_ptr(), sb.pcg_opts(fixed_iters=8), nb)
    assert st3 == sb.SB_OK
    xs = x.cpu().numpy()
    for s in range(nb):
        k = precond.clamp_k(precond.k_diag(sens[s], mask[s], mu, lam, gam, 2))
        A = lambda v, s=s: operators.apply_A(v, sens[s], mask[s], mu, lam, gam, 2)  # noqa: E731
        ref = pcg.pcg(A, b[s], np.zeros((ny, nx), complex), lambda v: precond.apply_precond(v, k, 2),
                      fixed_iters=8).x
        assert _rel(xs[s], ref) <= IMG_TOL, (s, _rel(xs[s], ref))
    plan.close()

    # a fresh plan: one application of A matches the oracle
    plan2 = _plan(torch, sb, sens, mask, mu, lam, gam)
    p = synth.random_complex((nb, ny, nx), rng)
    q = plan2.apply_A(torch.from_numpy(p).to(torch.complex64).cuda()).cpu().numpy()
    for s in range(nb):
        ref = operators.apply_A(p[s], sens[s], mask[s], mu, lam, gam, 2)
        assert _rel(q[s], ref) <= OP_TOL
    plan2.close()


def test_short_poll_limit_alone_changes_nothing(torch):
    """With the tiles requested as usual, a shorter poll limit than the default still leaves
    ample time for a tile to land: the solve is unchanged, bit for bit."""
    from paper_1710_01758_gb300 import sb

    mu, lam, gam = 1.0, 0.05, 0.05
    sens, mask, rng = _problem(seed=99)
    nb, nc, ny, nx = sens.shape
    d_b = torch.from_numpy(synth.random_complex((nb, ny, nx), rng)).to(torch.complex64).cuda()
    out = []
    for polls in (0, 1 << 16):
        plan = _plan(torch, sb, sens, mask, mu, lam, gam)
        plan.set_wait_check(polls, withhold_coil_tiles=False)
        x = torch.zeros_like(d_b)
        st, _ = sb.sb_pcg_solve(plan.handle, d_b.data_ptr(), x.data_ptr(), sb.pcg_opts(fixed_iters=6), nb)
        assert st == sb.SB_OK
        out.append(x.clone())
        plan.close()
    assert torch.equal(out[0], out[1])
