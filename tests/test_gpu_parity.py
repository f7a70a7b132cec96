"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on the same seeded
inputs.  Tolerances: one operator application <= 1e-5 relative L2; a fixed PCG / Split Bregman
schedule <= 1e-4 relative L2 on the image (complex64 vectors, FP64 CG scalars)."""
import numpy as np
import pytest

from oracle import operators, pcg, precond, split_bregman as sb_oracle
from paper_1710_01758_gb300 import synth

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
IMG_TOL = 1e-4


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


def oracle_M(kind, sens, mask, mu, lam, gam, k):
    if kind == "circulant":
        return lambda v: precond.apply_precond(v, k, 2)
    if kind == "jacobi":
        jd = precond.jacobi_diag(sens, mask, mu, lam, gam, 2)
        return lambda v: v / jd
    return None


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(torch, a, dtype=None):
    if dtype is None:
        dtype = torch.complex64 if np.iscomplexobj(a) else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def problem(nx, ny, nc, nb, seed, accel=4.0, n_centre=4):
    rng = np.random.default_rng(seed)
    sens = np.stack([synth.coil_maps(ny, nx, nc, rng) for _ in range(nb)])
    mask = np.stack([synth.line_mask(ny, nx, accel, min(n_centre, int(round(ny / accel))), rng)
                     for _ in range(nb)])
    return sens, mask, rng


def make_plan(sbm, torch, sens, mask, mu, lam, gam, levels=0, passes=0):
    nb, nc, ny, nx = sens.shape
    plan = sbm.Plan(nx, ny, nc, nb, mu, lam, gam, levels, precond_passes=passes)
    s_dev = to_dev(torch, sens)
    plan.set_coils(s_dev)
    plan.set_mask(torch.from_numpy(mask).cuda())
    return plan


SHAPES = [(32, 64, 3, 2), (64, 32, 2, 3), (128, 128, 4, 1), (256, 256, 12, 1), (256, 128, 5, 2), (32, 256, 3, 2),
          (64, 512, 3, 2),
          (512, 512, 32, 1), (512, 128, 3, 2),
          # mixed-radix lengths 16 x {12, 14, 20, 24}
          (192, 192, 8, 2), (256, 224, 12, 1), (320, 320, 16, 1), (384, 320, 32, 1), (224, 384, 3, 1)]


@pytest.mark.parametrize("nx,ny,nc,nb", SHAPES)
def test_apply_A(torch, sbm, nx, ny, nc, nb):
    sens, mask, rng = problem(nx, ny, nc, nb, seed=nx * 7 + ny + nc)
    mu, lam, gam = 1.0, 0.05, 0.05
    plan = make_plan(sbm, torch, sens, mask, mu, lam, gam)
    x = synth.random_complex((nb, ny, nx), rng)
    q = plan.apply_A(to_dev(torch, x)).cpu().numpy()
    for b in range(nb):
        ref = operators.apply_A(x[b], sens[b], mask[b], mu, lam, gam, 2)
        assert rel(q[b], ref) <= OP_TOL


@pytest.mark.parametrize("nx,ny,nc,nb", SHAPES)
def test_k_and_precond(torch, sbm, nx, ny, nc, nb):
    sens, mask, rng = problem(nx, ny, nc, nb, seed=nx + ny * 3 + nc)
    mu, lam, gam = 1.0, 0.05, 0.05
    plan = make_plan(sbm, torch, sens, mask, mu, lam, gam)
    kg = plan.k().cpu().numpy()
    r = synth.random_complex((nb, ny, nx), rng)
    z = plan.apply_precond(to_dev(torch, r)).cpu().numpy()
    for b in range(nb):
        kref = precond.k_diag(sens[b], mask[b], mu, lam, gam, 2)
        assert np.max(np.abs(kg[b] - kref)) <= OP_TOL * np.max(kref)
        zref = precond.apply_precond(r[b], kref, 2)
        assert rel(z[b], zref) <= OP_TOL


def test_precond_in_place_and_edge_masks(torch, sbm):
    # a single sampled line, full sampling, and one coil
    nx = ny = 64
    rng = np.random.default_rng(5)
    sens = np.stack([synth.coil_maps(ny, nx, 1, rng), synth.coil_maps(ny, nx, 1, rng)])
    mask = np.zeros((2, ny, nx), np.uint8)
    mask[0, 3] = 1
    mask[1] = 1
    plan = make_plan(sbm, torch, sens, mask, 1.0, 0.1, 0.02)
    r = synth.random_complex((2, ny, nx), rng)
    rd = to_dev(torch, r)
    plan.apply_precond(rd, rd)
    x = synth.random_complex((2, ny, nx), rng)
    q = plan.apply_A(to_dev(torch, x)).cpu().numpy()
    for b in range(2):
        kref = precond.k_diag(sens[b], mask[b], 1.0, 0.1, 0.02, 2)
        assert rel(rd[b].cpu().numpy(), precond.apply_precond(r[b], kref, 2)) <= OP_TOL
        assert rel(q[b], operators.apply_A(x[b], sens[b], mask[b], 1.0, 0.1, 0.02, 2)) <= OP_TOL


@pytest.mark.parametrize("kind", ["circulant", "none", "jacobi"])
def test_pcg_fixed_iterations(torch, sbm, kind):
    nx, ny, nc, nb = 128, 128, 4, 2
    sens, mask, rng = problem(nx, ny, nc, nb, seed=21)
    mu, lam, gam = 1.0, 0.05, 0.05
    plan = make_plan(sbm, torch, sens, mask, mu, lam, gam)
    b = synth.random_complex((nb, ny, nx), rng)
    x0 = synth.random_complex((nb, ny, nx), rng) * 0.1
    xd = to_dev(torch, x0)
    pc = {"circulant": sbm.SB_PRECOND_CIRCULANT, "none": sbm.SB_PRECOND_NONE, "jacobi": sbm.SB_PRECOND_JACOBI}[kind]
    st, res = plan.pcg_solve(to_dev(torch, b), xd, fixed_iters=12, precond=pc)
    assert st == sbm.SB_OK and all(r[0] == 12 for r in res)
    xg = xd.cpu().numpy()
    for i in range(nb):
        A = lambda v: operators.apply_A(v, sens[i], mask[i], mu, lam, gam, 2)  # noqa: E731
        k = precond.k_diag(sens[i], mask[i], mu, lam, gam, 2)
        M = oracle_M(kind, sens[i], mask[i], mu, lam, gam, k)
        ref = pcg.pcg(A, b[i], x0[i], M, fixed_iters=12)
        assert rel(xg[i], ref.x) <= IMG_TOL


def test_jacobi_weights_follow_new_coils_and_mask(torch, sbm):
    """The Jacobi weights are built by the first Jacobi solve after sb_set_mask: a solve after
    new coils (not normalised, so diag(A) changes) and after a new mask must use the new
    weights, checked against the oracle's Jacobi PCG each time."""
    nx, ny, nc, nb = 128, 128, 4, 2
    sens, mask, rng = problem(nx, ny, nc, nb, seed=29)
    mu, lam, gam = 1.0, 0.05, 0.05
    plan = make_plan(sbm, torch, sens, mask, mu, lam, gam)
    b = synth.random_complex((nb, ny, nx), rng)
    yy, xx = np.mgrid[0:ny, 0:nx]
    gain = 1.0 + 0.8 * np.cos(2 * np.pi * xx / nx) * np.sin(2 * np.pi * yy / ny)  # |S| no longer normalised
    sens2 = sens * gain
    mask2 = np.stack([synth.line_mask(ny, nx, 3.0, 8, rng) for _ in range(nb)])

    def check(s, m):
        xd = torch.zeros((nb, ny, nx), dtype=torch.complex64, device="cuda")
        st, res = plan.pcg_solve(to_dev(torch, b), xd, fixed_iters=10, precond=sbm.SB_PRECOND_JACOBI)
        assert st == sbm.SB_OK and all(r[0] == 10 for r in res)
        xg = xd.cpu().numpy()
        for i in range(nb):
            A = lambda v: operators.apply_A(v, s[i], m[i], mu, lam, gam, 2)  # noqa: E731
            M = oracle_M("jacobi", s[i], m[i], mu, lam, gam, None)
            ref = pcg.pcg(A, b[i], np.zeros((ny, nx), complex), M, fixed_iters=10)
            assert rel(xg[i], ref.x) <= IMG_TOL

    check(sens, mask)
    s2 = to_dev(torch, sens2)
    plan.set_coils(s2)  # new coils need sb_set_mask again before a solve (k depends on both)
    plan.set_mask(torch.from_numpy(mask).cuda())
    check(sens2, mask)
    plan.set_mask(torch.from_numpy(mask2).cuda())
    check(sens2, mask2)


@pytest.mark.parametrize("kind", ["circulant", "none", "jacobi"])
def test_pcg_tolerance_iteration_counts(torch, sbm, kind):
    nx, ny, nc, nb = 256, 256, 8, 2
    sens, mask, rng = problem(nx, ny, nc, nb, seed=33, n_centre=16)
    mu, lam, gam = 1e-3, 4e-3, 1e-3        # the paper's parameter set 1
    plan = make_plan(sbm, torch, sens, mask, mu, lam, gam)
    b = synth.random_complex((nb, ny, nx), rng)
    xd = torch.zeros((nb, ny, nx), dtype=torch.complex64, device="cuda")
    pc = {"circulant": sbm.SB_PRECOND_CIRCULANT, "none": sbm.SB_PRECOND_NONE, "jacobi": sbm.SB_PRECOND_JACOBI}[kind]
    st, res = plan.pcg_solve(to_dev(torch, b), xd, tol=1e-3, maxit=300, precond=pc)
    assert st == sbm.SB_OK
    xg = xd.cpu().numpy()
    for i in range(nb):
        A = lambda v: operators.apply_A(v, sens[i], mask[i], mu, lam, gam, 2)  # noqa: E731
        k = precond.k_diag(sens[i], mask[i], mu, lam, gam, 2)
        M = oracle_M(kind, sens[i], mask[i], mu, lam, gam, k)
        ref = pcg.pcg(A, b[i], np.zeros((ny, nx), complex), M, tol=1e-3, maxit=300)
        assert abs(res[i][0] - ref.iters) <= 1, (res[i], ref.iters)
        assert res[i][1] <= 1e-3 and res[i][2]
        assert rel(xg[i], ref.x) <= 2e-3


def test_pcg_zero_rhs_and_converged_start(torch, sbm):
    nx = ny = 64
    sens, mask, rng = problem(nx, ny, 2, 2, seed=3)
    plan = make_plan(sbm, torch, sens, mask, 1.0, 0.05, 0.05)
    b = np.zeros((2, ny, nx), complex)
    b[1] = synth.random_complex((ny, nx), rng)
    xd = to_dev(torch, synth.random_complex((2, ny, nx), rng))
    st, res = plan.pcg_solve(to_dev(torch, b), xd, tol=1e-3, maxit=100)
    assert st == sbm.SB_OK
    assert res[0][0] == 0 and res[0][2] and not torch.any(xd[0]).item()
    # restart from the converged solution: zero iterations
    st, res2 = plan.pcg_solve(to_dev(torch, b), xd, tol=1e-2, maxit=100)
    assert res2[1][0] == 0


def run_sb_both(torch, sbm, wl, nb, seed, tau=0.0, fixed=20, levels=None, n_outer=None):
    levels = wl.wavelet_levels if levels is None else levels
    n_outer = wl.n_outer if n_outer is None else n_outer
    slices = [synth.make_slice(wl, seed * 1000 + i) for i in range(nb)]
    sens = np.stack([s.sens for s in slices])
    mask = np.stack([s.mask for s in slices])
    y = np.stack([s.y for s in slices])
    plan = make_plan(sbm, torch, sens, mask, wl.mu, wl.lam, wl.gam, levels)
    xd = torch.zeros((nb, wl.ny, wl.nx), dtype=torch.complex64, device="cuda")
    st, iters, _ = plan.split_bregman(to_dev(torch, y), xd, n_outer, wl.n_inner, tau_tv=tau, tau_w=tau,
                                      fixed_iters=fixed, tol=wl.pcg_tol, maxit=wl.pcg_maxit)
    assert st == sbm.SB_OK
    xg = xd.cpu().numpy()
    refs = [sb_oracle.split_bregman(s.y, s.sens, s.mask, wl.mu, wl.lam, wl.gam, levels, 2, n_outer,
                                    wl.n_inner, wl.pcg_tol, wl.pcg_maxit, fixed, "circulant",
                                    tau if tau > 0 else None, tau if tau > 0 else None) for s in slices]
    return xg, refs, iters


def test_split_bregman_small_config(torch, sbm):
    # 128x128, 4 coils, TV only, 10 SB x 20 fixed PCG iterations
    wl = synth.SMALL_128
    xg, refs, _ = run_sb_both(torch, sbm, wl, 1, wl.seed, fixed=wl.pcg_fixed_iters)
    assert rel(xg[0], refs[0].x) <= IMG_TOL


@pytest.mark.parametrize("tau", [0.0, 0.02])
def test_split_bregman_tv_haar_active_shrink(torch, sbm, tau):
    wl = synth.Workload("64x64 Nc6 TV+Haar", 64, 64, 6, 4.0, 8, "uniform", 1.0, 0.05, 0.05, 4, 6, 1,
                        1e-3, 100, 0, seed=91)
    xg, refs, _ = run_sb_both(torch, sbm, wl, 2, wl.seed, tau=tau, fixed=15)
    for b in range(2):
        assert rel(xg[b], refs[b].x) <= IMG_TOL


def test_split_bregman_inner_loops_and_levels(torch, sbm):
    wl = synth.Workload("64x32 Nc3 TV+Haar2 inner2", 32, 64, 3, 4.0, 4, "uniform", 1.0, 0.1, 0.05, 2, 3, 2,
                        1e-3, 100, 0, seed=17)
    xg, refs, _ = run_sb_both(torch, sbm, wl, 1, wl.seed, tau=0.03, fixed=10)
    assert rel(xg[0], refs[0].x) <= IMG_TOL


def test_concurrent_groups_are_bitwise_identical(torch, sbm):
    # slices are independent: running the batch as 3 concurrent groups must give exactly the
    # result of one group, and both must match the oracle
    wl = synth.Workload("64x64 Nc4 TV+Haar groups", 64, 64, 4, 4.0, 8, "uniform", 1.0, 0.05, 0.05, 3, 3, 1,
                        1e-3, 100, 0, seed=5)
    nb = 5
    slices = [synth.make_slice(wl, 77 * 1000 + i) for i in range(nb)]
    sens = to_dev(torch, np.stack([s.sens for s in slices]))
    mask = torch.from_numpy(np.stack([s.mask for s in slices])).cuda()
    y = to_dev(torch, np.stack([s.y for s in slices]))
    out = []
    for groups in (1, 3):
        plan = sbm.Plan(wl.nx, wl.ny, wl.ncoils, nb, wl.mu, wl.lam, wl.gam, wl.wavelet_levels, groups=groups)
        plan.set_coils(sens)
        plan.set_mask(mask)
        x = torch.zeros((nb, wl.ny, wl.nx), dtype=torch.complex64, device="cuda")
        st, iters, _ = plan.split_bregman(y, x, wl.n_outer, tol=wl.pcg_tol, maxit=wl.pcg_maxit)
        assert st == sbm.SB_OK
        b = to_dev(torch, synth.random_complex((nb, wl.ny, wl.nx), np.random.default_rng(1)))
        xs = torch.zeros_like(b)
        st2, res = plan.pcg_solve(b, xs, tol=1e-4, maxit=100)
        assert st2 == sbm.SB_OK
        out.append((x.cpu().numpy(), iters, xs.cpu().numpy(), [r[0] for r in res]))
        plan.close()
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2]) and out[0][3] == out[1][3]
    for i in (0, nb - 1):
        s = slices[i]
        ref = sb_oracle.split_bregman(s.y, s.sens, s.mask, wl.mu, wl.lam, wl.gam, wl.wavelet_levels, 2, wl.n_outer,
                                      1, wl.pcg_tol, wl.pcg_maxit)
        assert rel(out[1][0][i], ref.x) <= 5e-3
        assert all(abs(a - b) <= 1 for a, b in zip(out[1][1][i], ref.iters))


@pytest.mark.parametrize("prec,groups", [(0, 3), (2, 3), (0, 1)])
def test_graph_replay_is_bitwise_identical(torch, sbm, prec, groups):
    """PCG iteration blocks replayed from CUDA graphs give exactly the direct launches' results
    (tolerance-stopped and fixed schedules, three concurrent slice groups, repeated calls that
    reuse the captured graphs, and a second coil buffer whose maps need their own capture)."""
    wl = synth.Workload("256x256 Nc4 TV+Haar graphs", 256, 256, 4, 4.0, 16, "uniform", 1.0, 0.05, 0.05, 3, 4, 1,
                        1e-3, 100, 0, seed=6)
    nb = 5
    slices = [synth.make_slice(wl, 88 * 1000 + i) for i in range(nb)]
    sens = to_dev(torch, np.stack([s.sens for s in slices]))
    mask = torch.from_numpy(np.stack([s.mask for s in slices])).cuda()
    y = to_dev(torch, np.stack([s.y for s in slices]))
    out = []
    for graphs in (False, True):
        # one group runs on the plan's stream: a stream of its own (the default stream is never captured)
        stream = torch.cuda.Stream() if groups == 1 else None
        torch.cuda.synchronize()
        plan = sbm.Plan(wl.nx, wl.ny, wl.ncoils, nb, wl.mu, wl.lam, wl.gam, wl.wavelet_levels, groups=groups,
                        prec=prec, stream=stream)
        plan.set_graphs(graphs)
        plan.set_coils(sens)
        plan.set_mask(mask)
        runs = []
        for rep, kw in enumerate([{"tol": wl.pcg_tol, "maxit": wl.pcg_maxit}, {"fixed_iters": 6},
                                  {"tol": wl.pcg_tol, "maxit": wl.pcg_maxit}]):
            x = torch.zeros((nb, wl.ny, wl.nx), dtype=torch.complex64, device="cuda")
            torch.cuda.synchronize()
            st, iters, _ = plan.split_bregman(y, x, wl.n_outer, **kw)
            assert st == sbm.SB_OK
            runs.append((x.cpu().numpy(), iters))
        sens2 = sens.clone()  # same coils at another address, then back to the first buffer
        for sd in (sens2, sens):
            plan.set_coils(sd)
            plan.set_mask(mask)
            x = torch.zeros((nb, wl.ny, wl.nx), dtype=torch.complex64, device="cuda")
            torch.cuda.synchronize()
            st, iters, _ = plan.split_bregman(y, x, wl.n_outer, tol=wl.pcg_tol, maxit=wl.pcg_maxit)
            assert st == sbm.SB_OK
            runs.append((x.cpu().numpy(), iters))
        out.append(runs)
        plan.close()
    for (xa, ia), (xb, ib) in zip(out[0], out[1]):
        assert np.array_equal(xa, xb) and ia == ib
    for k in (2, 3, 4):
        assert np.array_equal(out[1][0][0], out[1][k][0])


def test_unsupported_inputs(torch, sbm):
    with pytest.raises(sbm.SbError) as ei:
        sbm.Plan(48, 64, 2, 1, 1.0, 0.1, 0.1, 0)
    assert ei.value.status == sbm.SB_ERR_UNSUPPORTED
    with pytest.raises(sbm.SbError) as ei:  # Haar blocks larger than the update tiles
        sbm.Plan(64, 64, 2, 1, 1.0, 0.1, 0.1, 6)
    assert ei.value.status == sbm.SB_ERR_UNSUPPORTED
    with pytest.raises(sbm.SbError) as ei:  # a 512 x 512 slice does not fit one cluster
        sbm.Plan(512, 512, 2, 1, 1.0, 0.1, 0.1, 0, precond_passes=1)
    assert ei.value.status == sbm.SB_ERR_UNSUPPORTED
    with pytest.raises(sbm.SbError) as ei:
        sbm.Plan(64, 64, 2, 1, 1.0, 0.1, 0.1, 0, precond_passes=2)
    assert ei.value.status == sbm.SB_ERR_INVALID_ARG
    nx = ny = 32
    sens, mask, rng = problem(nx, ny, 2, 1, seed=1)
    plan = sbm.Plan(nx, ny, 2, 1, 1.0, 0.1, 0.1, 0)
    plan.set_coils(to_dev(torch, sens))
    with pytest.raises(sbm.SbError) as ei:  # k was not built: operators refuse
        plan.apply_A(to_dev(torch, np.zeros((1, ny, nx), complex)))
    assert ei.value.status == sbm.SB_ERR_NOT_READY
    plan.set_mask(torch.from_numpy(mask).cuda())
    y = to_dev(torch, np.zeros((1, 2, ny, nx), complex))
    buf = torch.zeros(ny * nx + 1, dtype=torch.complex64, device="cuda")
    x_off = buf[1:].view(1, ny, nx)  # 8 bytes past a 16-byte boundary
    with pytest.raises(sbm.SbError) as ei:
        plan.split_bregman(y, x_off, 1, 1)
    assert ei.value.status == sbm.SB_ERR_INVALID_ARG


def test_parameter_sets_preconditioner_comparison(torch, sbm):
    # The comparison of the Results on synthetic data: for the paper's parameter sets 1-3 the
    # circulant preconditioner needs fewer PCG iterations than plain CG, and Jacobi needs the
    # same number as plain CG (normalised coils make diag(A) constant).  GPU counts match the
    # oracle's within one iteration.
    nx = ny = 128
    nb, nc = 2, 8
    sens, mask, rng = problem(nx, ny, nc, nb, seed=404, n_centre=12)
    b = synth.random_complex((nb, ny, nx), rng)
    sets = [(1e-3, 4e-3, 1e-3), (1e-2, 4e-3, 1e-3), (1e-3, 4e-3, 4e-3)]
    for mu, lam, gam in sets:
        plan = make_plan(sbm, torch, sens, mask, mu, lam, gam)
        counts = {}
        for kind, pc in [("circulant", sbm.SB_PRECOND_CIRCULANT), ("none", sbm.SB_PRECOND_NONE),
                         ("jacobi", sbm.SB_PRECOND_JACOBI)]:
            xd = torch.zeros((nb, ny, nx), dtype=torch.complex64, device="cuda")
            st, res = plan.pcg_solve(to_dev(torch, b), xd, tol=1e-3, maxit=500, precond=pc)
            assert st == sbm.SB_OK
            counts[kind] = [r[0] for r in res]
            for i in range(nb):
                A = lambda v: operators.apply_A(v, sens[i], mask[i], mu, lam, gam, 2)  # noqa: E731
                k = precond.k_diag(sens[i], mask[i], mu, lam, gam, 2)
                ref = pcg.pcg(A, b[i], np.zeros((ny, nx), complex), oracle_M(kind, sens[i], mask[i], mu, lam, gam, k),
                              tol=1e-3, maxit=500)
                assert abs(res[i][0] - ref.iters) <= 1, (mu, lam, gam, kind, res[i][0], ref.iters)
        for i in range(nb):
            assert counts["circulant"][i] < counts["none"][i]
            assert abs(counts["jacobi"][i] - counts["none"][i]) <= 1
        plan.close()


def test_split_bregman_512_variable_density(torch, sbm):
    # 512x512 (three-stage transforms), R = 6 variable-density lines with 32 centre lines,
    # TV + 4-level Haar, fixed schedule against the oracle
    wl = synth.Workload("512x512 Nc6 R6 vd TV+Haar4", 512, 512, 6, 6.0, 32, "variable", 1.0, 0.05, 0.05, 4, 3, 1,
                        1e-3, 100, 0, seed=synth.SEED_BASE + 3)
    xg, refs, _ = run_sb_both(torch, sbm, wl, 1, wl.seed, tau=0.02, fixed=6)
    assert rel(xg[0], refs[0].x) <= IMG_TOL


def test_split_bregman_five_haar_levels(torch, sbm):
    # the deepest Haar tree the 32 x 32 update tiles hold (5 levels), active shrinkage
    wl = synth.Workload("64x64 Nc4 TV+Haar5", 64, 64, 4, 4.0, 8, "uniform", 1.0, 0.05, 0.05, 5, 4, 1,
                        1e-3, 100, 0, seed=29)
    xg, refs, _ = run_sb_both(torch, sbm, wl, 2, wl.seed, tau=0.02, fixed=10)
    for b in range(2):
        assert rel(xg[b], refs[b].x) <= IMG_TOL


@pytest.mark.parametrize("nx,ny,nc,nb", [(256, 256, 6, 3), (128, 256, 3, 2), (256, 64, 2, 2), (32, 32, 2, 2),
                                         (128, 128, 4, 2)])
@pytest.mark.parametrize("passes", [1, 3])
def test_pcg_precond_schedules(torch, sbm, nx, ny, nc, nb, passes):
    # the circulant M^{-1} inside PCG as one cluster launch (1) or three HBM passes (3): both
    # against the oracle, for a fixed count and to the tolerance
    sens, mask, rng = problem(nx, ny, nc, nb, seed=nx + 3 * ny + nc, n_centre=8)
    mu, lam, gam = 1.0, 0.05, 0.05
    plan = make_plan(sbm, torch, sens, mask, mu, lam, gam, passes=passes)
    b = synth.random_complex((nb, ny, nx), rng)
    x0 = synth.random_complex((nb, ny, nx), rng) * 0.1
    xd = to_dev(torch, x0)
    st, res = plan.pcg_solve(to_dev(torch, b), xd, fixed_iters=9)
    assert st == sbm.SB_OK and all(r[0] == 9 for r in res)
    xt = to_dev(torch, x0)
    st, rest = plan.pcg_solve(to_dev(torch, b), xt, tol=1e-4, maxit=200)
    assert st == sbm.SB_OK
    xg, xtg = xd.cpu().numpy(), xt.cpu().numpy()
    for i in range(nb):
        A = lambda v: operators.apply_A(v, sens[i], mask[i], mu, lam, gam, 2)  # noqa: E731
        k = precond.k_diag(sens[i], mask[i], mu, lam, gam, 2)
        M = lambda v: precond.apply_precond(v, k, 2)  # noqa: E731
        ref = pcg.pcg(A, b[i], x0[i], M, fixed_iters=9)
        assert rel(xg[i], ref.x) <= IMG_TOL
        reft = pcg.pcg(A, b[i], x0[i], M, tol=1e-4, maxit=200)
        assert abs(rest[i][0] - reft.iters) <= 1, (rest[i], reft.iters)
        assert rest[i][1] <= 1e-4 and rest[i][2]
        assert rel(xtg[i], reft.x) <= 1e-3


def test_split_bregman_mixed_radix_sizes(torch, sbm):
    # 224 x 192 (x by y): radix-16 x 2 x 7 along x, 16 x 4 x 3 along y; TV + 4-level Haar with
    # active shrinkage, R = 3 lines
    wl = synth.Workload("192x224 Nc8 R3 TV+Haar4", 192, 224, 8, 3.0, 16, "uniform", 1.0, 0.05, 0.05, 4, 4, 1,
                        1e-3, 100, 0, seed=4242)
    xg, refs, _ = run_sb_both(torch, sbm, wl, 2, wl.seed, tau=0.02, fixed=8)
    for b in range(2):
        assert rel(xg[b], refs[b].x) <= IMG_TOL


def random_mask_problem(nx, ny, nc, nb, seed, accel=3.0, centre=8):
    rng = np.random.default_rng(seed)
    sens = np.stack([synth.coil_maps(ny, nx, nc, rng) for _ in range(nb)])
    mask = np.stack([synth.random_mask(ny, nx, accel, centre, rng) for _ in range(nb)])
    return sens, mask, rng


@pytest.mark.parametrize("nx,ny,nc,nb", [(64, 64, 4, 2), (128, 64, 3, 1), (192, 224, 6, 1), (256, 256, 8, 1)])
def test_random_mask_operators(torch, sbm, nx, ny, nc, nb):
    # the paper's second sampling scheme: points drawn at random in (k_y, k_x)
    sens, mask, rng = random_mask_problem(nx, ny, nc, nb, seed=nx + 5 * ny + nc)
    mu, lam, gam = 1.0, 0.05, 0.05
    plan = make_plan(sbm, torch, sens, mask, mu, lam, gam)
    x = synth.random_complex((nb, ny, nx), rng)
    q = plan.apply_A(to_dev(torch, x)).cpu().numpy()
    kg = plan.k().cpu().numpy()
    z = plan.apply_precond(to_dev(torch, x)).cpu().numpy()
    for b in range(nb):
        assert rel(q[b], operators.apply_A(x[b], sens[b], mask[b], mu, lam, gam, 2)) <= OP_TOL
        kref = precond.k_diag(sens[b], mask[b], mu, lam, gam, 2)
        assert np.max(np.abs(kg[b] - kref)) <= OP_TOL * np.max(kref)
        assert rel(z[b], precond.apply_precond(x[b], kref, 2)) <= OP_TOL


@pytest.mark.parametrize("nx,ny,nc,nb", [(256, 256, 6, 3), (64, 128, 3, 2), (256, 64, 2, 2), (128, 128, 12, 1)])
def test_random_mask_cluster_and_three_passes(torch, sbm, nx, ny, nc, nb):
    # the general path's q = A p as one cluster launch (spectra in distributed shared memory) and
    # as three passes through the coil scratch: both against the oracle, one application and a
    # fixed PCG schedule (p^H q and alpha in the cluster kernel)
    sens, mask, rng = random_mask_problem(nx, ny, nc, nb, seed=3 * nx + ny + nc)
    mu, lam, gam = 1.0, 0.05, 0.05
    plan = make_plan(sbm, torch, sens, mask, mu, lam, gam)
    x = synth.random_complex((nb, ny, nx), rng)
    b = synth.random_complex((nb, ny, nx), rng)
    out = {}
    for passes in (1, 3):
        plan.set_tuning(general_passes=passes)
        assert plan.tuning()["general_passes"] == passes
        q = plan.apply_A(to_dev(torch, x)).cpu().numpy()
        xd = torch.zeros((nb, ny, nx), dtype=torch.complex64, device="cuda")
        st, _ = plan.pcg_solve(to_dev(torch, b), xd, fixed_iters=6)
        assert st == sbm.SB_OK
        out[passes] = (q, xd.cpu().numpy())
    for s_ in range(nb):
        qref = operators.apply_A(x[s_], sens[s_], mask[s_], mu, lam, gam, 2)
        k = precond.clamp_k(precond.k_diag(sens[s_], mask[s_], mu, lam, gam, 2))
        A = lambda v, s_=s_: operators.apply_A(v, sens[s_], mask[s_], mu, lam, gam, 2)  # noqa: E731
        xref = pcg.pcg(A, b[s_], np.zeros((ny, nx), complex), lambda v: precond.apply_precond(v, k, 2),
                       fixed_iters=6).x
        for passes in (1, 3):
            assert rel(out[passes][0][s_], qref) <= OP_TOL, (passes, s_)
            assert rel(out[passes][1][s_], xref) <= IMG_TOL, (passes, s_)
    with pytest.raises(sbm.SbError) as ei:
        plan.set_tuning(general_passes=2)
    assert ei.value.status == sbm.SB_ERR_INVALID_ARG


@pytest.mark.parametrize("kind", ["circulant", "jacobi"])
def test_random_mask_pcg_and_mixed_batch(torch, sbm, kind):
    # slice 0 random points, slice 1 Cartesian lines: one plan in the general mode
    nx = ny = 64
    rng = np.random.default_rng(8)
    sens = np.stack([synth.coil_maps(ny, nx, 4, rng) for _ in range(2)])
    mask = np.stack([synth.random_mask(ny, nx, 3.0, 8, rng), synth.line_mask(ny, nx, 4.0, 8, rng)])
    mu, lam, gam = 1.0, 0.05, 0.05
    plan = make_plan(sbm, torch, sens, mask, mu, lam, gam)
    b = synth.random_complex((2, ny, nx), rng)
    pc = sbm.SB_PRECOND_CIRCULANT if kind == "circulant" else sbm.SB_PRECOND_JACOBI
    xd = torch.zeros((2, ny, nx), dtype=torch.complex64, device="cuda")
    st, res = plan.pcg_solve(to_dev(torch, b), xd, tol=1e-4, maxit=300, precond=pc)
    assert st == sbm.SB_OK
    for i in range(2):
        A = lambda v: operators.apply_A(v, sens[i], mask[i], mu, lam, gam, 2)  # noqa: E731
        k = precond.k_diag(sens[i], mask[i], mu, lam, gam, 2)
        M = oracle_M(kind, sens[i], mask[i], mu, lam, gam, k)
        ref = pcg.pcg(A, b[i], np.zeros((ny, nx), complex), M, tol=1e-4, maxit=300)
        assert abs(res[i][0] - ref.iters) <= 1, (res[i], ref.iters)
        assert rel(xd[i].cpu().numpy(), ref.x) <= 1e-3


@pytest.mark.parametrize("tau", [0.0, 0.02])
def test_random_mask_split_bregman(torch, sbm, tau):
    nx, ny, nc, nb = 64, 64, 4, 2
    rng = np.random.default_rng(1234)
    mu, lam, gam, levels = 1.0, 0.05, 0.05, 3
    sl = []
    for _ in range(nb):
        xt = synth.ellipse_phantom(ny, nx, rng)
        s_ = synth.coil_maps(ny, nx, nc, rng)
        m_ = synth.random_mask(ny, nx, 3.0, 8, rng)
        sl.append((s_, m_, synth.acquire(xt, s_, m_, 1e-3, rng)))
    sens = np.stack([a for a, _, _ in sl])
    mask = np.stack([m for _, m, _ in sl])
    y = np.stack([c for _, _, c in sl])
    plan = make_plan(sbm, torch, sens, mask, mu, lam, gam, levels)
    xd = torch.zeros((nb, ny, nx), dtype=torch.complex64, device="cuda")
    st, _, _ = plan.split_bregman(to_dev(torch, y), xd, 4, tau_tv=tau, tau_w=tau, fixed_iters=8)
    assert st == sbm.SB_OK
    for i in range(nb):
        ref = sb_oracle.split_bregman(y[i], sens[i], mask[i], mu, lam, gam, levels, 2, 4, 1, 1e-3, 100, 8,
                                      "circulant", tau if tau > 0 else None, tau if tau > 0 else None)
        assert rel(xd[i].cpu().numpy(), ref.x) <= IMG_TOL


@pytest.mark.parametrize("nx,ny,levels,tau,density", [(64, 64, 3, 0.02, "uniform"), (128, 64, 1, 0.02, "uniform"),
                                                      (64, 64, 4, 0.0, "uniform"), (512, 256, 4, 0.02, "uniform"),
                                                      (64, 64, 2, 0.02, "random")])
def test_split_bregman_daubechies4(torch, sbm, nx, ny, levels, tau, density):
    # the paper's wavelet: W = periodic Daubechies-4 in steps 4, 8 and 11
    wl = synth.Workload("D4", ny, nx, 4, 4.0, 8, density, 1.0, 0.05, 0.05, levels, 4, 1, 1e-3, 100, 0, seed=606)
    nb = 2
    slices = [synth.make_slice(wl, wl.seed * 1000 + i) for i in range(nb)]
    sens = np.stack([s.sens for s in slices])
    mask = np.stack([s.mask for s in slices])
    y = np.stack([s.y for s in slices])
    plan = sbm.Plan(nx, ny, 4, nb, wl.mu, wl.lam, wl.gam, levels, wavelet=sbm.SB_WAVELET_DAUB4)
    plan.set_coils(to_dev(torch, sens))
    plan.set_mask(torch.from_numpy(mask).cuda())
    xd = torch.zeros((nb, ny, nx), dtype=torch.complex64, device="cuda")
    st, _, _ = plan.split_bregman(to_dev(torch, y), xd, wl.n_outer, tau_tv=tau, tau_w=tau, fixed_iters=8)
    assert st == sbm.SB_OK
    for i, s in enumerate(slices):
        ref = sb_oracle.split_bregman(s.y, s.sens, s.mask, wl.mu, wl.lam, wl.gam, levels, 2, wl.n_outer, 1, 1e-3, 100,
                                      8, "circulant", tau if tau > 0 else None, tau if tau > 0 else None,
                                      wavelet="daub4")
        assert rel(xd[i].cpu().numpy(), ref.x) <= IMG_TOL
    plan.close()


def test_daubechies4_unsupported(torch, sbm):
    with pytest.raises(sbm.SbError) as ei:  # coarsest band 2 wide
        sbm.Plan(32, 32, 2, 1, 1.0, 0.1, 0.1, 5, wavelet=sbm.SB_WAVELET_DAUB4)
    assert ei.value.status == sbm.SB_ERR_UNSUPPORTED
    with pytest.raises(sbm.SbError) as ei:  # volumes use Haar
        sbm.Plan(32, 32, 2, 1, 1.0, 0.1, 0.1, 2, nz=32, wavelet=sbm.SB_WAVELET_DAUB4)
    assert ei.value.status == sbm.SB_ERR_UNSUPPORTED
    with pytest.raises(sbm.SbError) as ei:
        sbm.Plan(32, 32, 2, 1, 1.0, 0.1, 0.1, 2, wavelet=7)
    assert ei.value.status == sbm.SB_ERR_INVALID_ARG


def test_coil_compression(torch, sbm):
    # Methods, "Coil Compression": 12 coils to 6 virtual coils, then Split Bregman on the virtual
    # coils; compared with the oracle's compression through phase-invariant quantities
    from oracle import coil_compression as cc
    wl = synth.Workload("cc 64x64 Nc12", 64, 64, 12, 4.0, 8, "uniform", 1.0, 0.05, 0.05, 2, 3, 1, 1e-3, 100, 0,
                        seed=77)
    nb, nv = 2, 6
    slices = [synth.make_slice(wl, wl.seed * 1000 + i) for i in range(nb)]
    y = np.stack([s.y for s in slices])
    sens = np.stack([s.sens for s in slices])
    mask = np.stack([s.mask for s in slices])
    yv, sv, mat, eig = sbm.coil_compress(to_dev(torch, y), to_dev(torch, sens), nv)
    yv_h, sv_h = yv.cpu().numpy(), sv.cpu().numpy()
    refs = []
    for b in range(nb):
        A_o, s_o = cc.compression_matrix(y[b], nv)
        np.testing.assert_allclose(eig[b], s_o, rtol=1e-4, atol=1e-6 * s_o[0])
        gap = s_o[nv - 1] - s_o[nv]
        P_g = mat[b].astype(np.complex128).conj().T @ mat[b].astype(np.complex128)
        assert np.abs(P_g - A_o.conj().T @ A_o).max() <= 1e-5 + 1e-5 * s_o[0] / gap
        yo, so = cc.compress(y[b], sens[b], A_o)
        refs.append((yo, so))
        bp_g = operators.encode_adj(yv_h[b], sv_h[b], mask[b], 2)
        bp_o = operators.encode_adj(yo, so, mask[b], 2)
        assert rel(bp_g, bp_o) <= 1e-4
    plan = sbm.Plan(wl.nx, wl.ny, nv, nb, wl.mu, wl.lam, wl.gam, wl.wavelet_levels)
    plan.set_coils(sv)
    plan.set_mask(torch.from_numpy(mask).cuda())
    xd = torch.zeros((nb, wl.ny, wl.nx), dtype=torch.complex64, device="cuda")
    st, _, _ = plan.split_bregman(yv, xd, wl.n_outer, tau_tv=0.02, tau_w=0.02, fixed_iters=8)
    assert st == sbm.SB_OK
    for b in range(nb):
        yo, so = refs[b]
        ref = sb_oracle.split_bregman(yo, so, mask[b], wl.mu, wl.lam, wl.gam, wl.wavelet_levels, 2, wl.n_outer, 1,
                                      1e-3, 100, 8, "circulant", 0.02, 0.02)
        assert rel(xd[b].cpu().numpy(), ref.x) <= IMG_TOL
    plan.close()
