"""Launch-configuration tuning on the GPU: every column-pass tile width gives bitwise the same
M^{-1} r and the same PCG result (up to the FP64 summation order of rho); the poll interval and
graph replay change no result; unfit tiles are refused; the autotuner returns a valid choice and
caches it."""
import numpy as np
import pytest

from oracle import operators, precond
from paper_1710_01758_gb300 import synth

pytestmark = pytest.mark.gpu


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


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.complex64 if np.iscomplexobj(a) else torch.uint8).cuda()


def setup(sbm, torch, nx, ny, nc, nb, seed, groups=0, stream=None):
    rng = np.random.default_rng(seed)
    sens = np.stack([synth.coil_maps(ny, nx, nc, rng) for _ in range(nb)])
    mask = np.stack([synth.line_mask(ny, nx, 4.0, 8, rng) for _ in range(nb)])
    plan = sbm.Plan(nx, ny, nc, nb, 1.0, 0.05, 0.05, 0, groups=groups, stream=stream)
    plan.set_coils(dev(torch, sens))
    plan.set_mask(dev(torch, mask))
    torch.cuda.synchronize()
    return plan, sens, mask, rng


@pytest.mark.parametrize("nx,ny", [(256, 256), (64, 128), (512, 512), (320, 320)])
def test_col_tiles_bitwise_and_oracle(torch, sbm, nx, ny):
    from paper_1710_01758_gb300 import autotune
    nb = 2
    plan, sens, mask, rng = setup(sbm, torch, nx, ny, 2, nb, seed=nx + ny)
    r = synth.random_complex((nb, ny, nx), rng)
    rd = dev(torch, r)
    outs = {}
    for ct in (8, 16, 32):
        if not autotune.col_tile_fits(ny, nx, ct):
            with pytest.raises(sbm.SbError) as ei:
                plan.set_tuning(col_tile=ct)
            assert ei.value.status == sbm.SB_ERR_UNSUPPORTED
            continue
        plan.set_tuning(col_tile=ct)
        assert plan.tuning()["col_tile"] == ct
        z = plan.apply_precond(rd)
        torch.cuda.synchronize()
        outs[ct] = z.cpu().numpy()
    assert len(outs) >= 2
    for ct, z in outs.items():
        assert np.array_equal(z, outs[16]), ct
    kref = precond.k_diag(sens[0], mask[0], 1.0, 0.05, 0.05, 2)
    zref = precond.apply_precond(r[0], kref, 2)
    assert np.linalg.norm(outs[16][0] - zref) / np.linalg.norm(zref) <= 1e-5


def test_tuning_keeps_pcg_results(torch, sbm):
    nx = ny = 128
    nb = 6
    plan, sens, mask, rng = setup(sbm, torch, nx, ny, 3, nb, seed=3, groups=2, stream=torch.cuda.Stream())
    b = dev(torch, synth.random_complex((nb, ny, nx), rng))
    res = {}
    for ct, pe, graphs in [(16, 4, False), (8, 2, True), (32, 8, True), (16, 1, True), (16, 4, True)]:
        plan.set_tuning(col_tile=ct, poll_every=pe)
        plan.set_graphs(graphs)
        x = torch.zeros((nb, ny, nx), dtype=torch.complex64, device="cuda")
        torch.cuda.synchronize()
        st, r = plan.pcg_solve(b, x, tol=1e-4, maxit=100)
        assert st == sbm.SB_OK
        res[(ct, pe, graphs)] = (x.cpu().numpy(), [i[0] for i in r])
    base_x, base_it = res[(16, 4, False)]
    assert np.array_equal(res[(16, 4, True)][0], base_x)  # graphs: bitwise
    for k, (xk, itk) in res.items():
        assert itk == base_it, k
        assert np.linalg.norm(xk - base_x) / np.linalg.norm(base_x) <= 1e-6, k
    with pytest.raises(sbm.SbError) as ei:
        plan.set_tuning(poll_every=65)
    assert ei.value.status == sbm.SB_ERR_INVALID_ARG
    with pytest.raises(sbm.SbError) as ei:
        plan.set_tuning(col_tile=12)
    assert ei.value.status == sbm.SB_ERR_UNSUPPORTED


def test_autotuner_choice_and_cache(torch, sbm, tmp_path):
    from paper_1710_01758_gb300 import autotune
    nx, ny, nc, nb = 128, 128, 3, 4
    rng = np.random.default_rng(8)
    sens = dev(torch, np.stack([synth.coil_maps(ny, nx, nc, rng) for _ in range(nb)]))
    mask = dev(torch, np.stack([synth.line_mask(ny, nx, 4.0, 8, rng) for _ in range(nb)]))

    def make(g):
        p = sbm.Plan(nx, ny, nc, nb, 1.0, 0.05, 0.05, 0, groups=g, stream=torch.cuda.Stream())
        p.set_coils(sens)
        p.set_mask(mask)
        torch.cuda.synchronize()
        return p

    path = str(tmp_path / "tune.json")
    t = autotune.tune(make, nx, ny, nc, nb, reps=1, path=path)
    assert not t["cached"] and (t["groups"], t["col_tile"], t["poll_every"]) in autotune.candidates(nx, ny, nb)
    assert t["ms"] > 0 and t["ms"] <= t["default_ms"]
    t2 = autotune.tune(make, nx, ny, nc, nb, reps=1, path=path)
    assert t2["cached"] and t2["col_tile"] == t["col_tile"] and t2["groups"] == t["groups"]


@pytest.mark.parametrize("ny", [256, 512])
def test_apply_tile_kernels_agree(torch, sbm, ny):
    """The two q = A p kernels at 256 and 512 rows (8 columns per CTA with tensor-memory state, 16
    columns with register state) compute the same values: one application bitwise; a PCG solve to
    the same iterates up to the order of the FP64 partial sums of p^H q."""
    nx, nc, nb = 64, 5, 3
    plan, sens, mask, rng = setup(sbm, torch, nx, ny, nc, nb, seed=21)
    p = dev(torch, synth.random_complex((nb, ny, nx), rng))
    q = {}
    xs = {}
    for at in (8, 16):
        plan.set_tuning(apply_tile=at)
        assert plan.tuning()["apply_tile"] == at
        q[at] = plan.apply_A(p).cpu().numpy()
        x = torch.zeros((nb, ny, nx), dtype=torch.complex64, device="cuda")
        st, _ = plan.pcg_solve(p, x, fixed_iters=6)
        assert st == sbm.SB_OK
        xs[at] = x.cpu().numpy()
    assert np.array_equal(q[8], q[16])
    assert np.linalg.norm(xs[8] - xs[16]) / np.linalg.norm(xs[16]) <= 1e-6
    for s in range(nb):
        ref = operators.apply_A(p[s].cpu().numpy().astype(np.complex128), sens[s], mask[s], 1.0, 0.05, 0.05, 2)
        assert np.linalg.norm(q[8][s] - ref) / np.linalg.norm(ref) <= 1e-5
    with pytest.raises(sbm.SbError) as ei:
        plan.set_tuning(apply_tile=12)
    assert ei.value.status == sbm.SB_ERR_INVALID_ARG
