"""GPU parity for volumes (ndim = 3, readout x fully sampled, sampled (k_y, k_z) lines): the
CUDA library through its C ABI against the FP64 oracle (which implements the 3D operators from
their definitions).  Tolerances as in the 2D tests: one operator <= 1e-5, fixed schedules <= 1e-4
relative L2."""
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(torch, a):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a).to(torch.complex64 if np.iscomplexobj(a) else torch.float32).cuda()


def volume_problem(nz, ny, nx, nc, nb, seed, accel=4.0, centre=6):
    rng = np.random.default_rng(seed)
    sens = np.stack([synth.coil_maps_3d(nz, ny, nx, nc, rng) for _ in range(nb)])
    mask = np.stack([synth.readout_mask_3d(nz, ny, nx, accel, centre, rng) for _ in range(nb)])
    return sens, mask, rng


def vplan(sbm, torch, sens, mask, mu, lam, gam, levels=0):
    nb, nc, nz, ny, nx = sens.shape
    plan = sbm.Plan(nx, ny, nc, nb, mu, lam, gam, levels, nz=nz)
    plan.set_coils(dev(torch, sens))
    plan.set_mask(torch.from_numpy(np.ascontiguousarray(mask)).cuda())
    return plan


VSHAPES = [(32, 32, 32, 3, 2), (32, 64, 32, 2, 1), (64, 32, 64, 4, 1), (32, 32, 64, 1, 1)]


@pytest.mark.parametrize("nz,ny,nx,nc,nb", VSHAPES)
def test_volume_apply_A_k_precond(torch, sbm, nz, ny, nx, nc, nb):
    sens, mask, rng = volume_problem(nz, ny, nx, nc, nb, seed=nz + 3 * ny + 7 * nx + nc)
    mu, lam, gam = 1.0, 0.05, 0.05
    plan = vplan(sbm, torch, sens, mask, mu, lam, gam)
    x = synth.random_complex((nb, nz, ny, nx), rng)
    q = plan.apply_A(dev(torch, x)).cpu().numpy()
    kg = plan.k().cpu().numpy()
    r = synth.random_complex((nb, nz, ny, nx), rng)
    z = plan.apply_precond(dev(torch, r)).cpu().numpy()
    for b in range(nb):
        assert rel(q[b], operators.apply_A(x[b], sens[b], mask[b], mu, lam, gam, 3)) <= OP_TOL
        kref = precond.k_diag(sens[b], mask[b], mu, lam, gam, 3)
        assert np.max(np.abs(kg[b] - kref)) <= OP_TOL * np.max(kref)
        assert rel(z[b], precond.apply_precond(r[b], kref, 3)) <= OP_TOL
    plan.close()


@pytest.mark.parametrize("kind", ["circulant", "none", "jacobi"])
def test_volume_pcg(torch, sbm, kind):
    nz, ny, nx, nc, nb = 32, 32, 32, 4, 2
    sens, mask, rng = volume_problem(nz, ny, nx, nc, nb, seed=77)
    mu, lam, gam = 1.0, 0.05, 0.05
    plan = vplan(sbm, torch, sens, mask, mu, lam, gam)
    b = synth.random_complex((nb, nz, ny, nx), rng)
    x0 = synth.random_complex((nb, nz, ny, nx), rng) * 0.1
    pc = {"circulant": sbm.SB_PRECOND_CIRCULANT, "none": sbm.SB_PRECOND_NONE, "jacobi": sbm.SB_PRECOND_JACOBI}[kind]
    xd = dev(torch, x0)
    st, res = plan.pcg_solve(dev(torch, b), xd, fixed_iters=10, precond=pc)
    assert st == sbm.SB_OK and all(r[0] == 10 for r in res)
    xt = dev(torch, x0)
    st, rest = plan.pcg_solve(dev(torch, b), xt, tol=1e-4, maxit=300, precond=pc)
    assert st == sbm.SB_OK
    for i in range(nb):
        A = lambda v: operators.apply_A(v, sens[i], mask[i], mu, lam, gam, 3)  # noqa: E731
        if kind == "circulant":
            k = precond.k_diag(sens[i], mask[i], mu, lam, gam, 3)
            M = lambda v: precond.apply_precond(v, k, 3)  # noqa: E731
        elif kind == "jacobi":
            jd = precond.jacobi_diag(sens[i], mask[i], mu, lam, gam, 3)
            M = lambda v: v / jd  # noqa: E731
        else:
            M = None
        ref = pcg.pcg(A, b[i], x0[i], M, fixed_iters=10)
        assert rel(xd[i].cpu().numpy(), ref.x) <= IMG_TOL
        reft = pcg.pcg(A, b[i], x0[i], M, tol=1e-4, maxit=300)
        assert abs(rest[i][0] - reft.iters) <= 1, (rest[i], reft.iters)
        assert rest[i][1] <= 1e-4 and rest[i][2]
        assert rel(xt[i].cpu().numpy(), reft.x) <= 1e-3
    plan.close()


@pytest.mark.parametrize("levels,tau", [(2, 0.02), (4, 0.02), (0, 0.0)])
def test_volume_split_bregman(torch, sbm, levels, tau):
    v = synth.Volume("32x32x32 Nc4", 32, 32, 32, 4, 4.0, 6, 1.0, 0.05, 0.05, levels, 4, 1, 1e-3, 100, 0, seed=314)
    nb = 2
    vols = [synth.make_volume(v, v.seed * 1000 + i) for i in range(nb)]
    sens = np.stack([s.sens for s in vols])
    mask = np.stack([s.mask for s in vols])
    y = np.stack([s.y for s in vols])
    plan = vplan(sbm, torch, sens, mask, v.mu, v.lam, v.gam, levels)
    xd = torch.zeros((nb, v.nz, v.ny, v.nx), dtype=torch.complex64, device="cuda")
    st, iters, _ = plan.split_bregman(dev(torch, y), xd, v.n_outer, tau_tv=tau, tau_w=tau, fixed_iters=8)
    assert st == sbm.SB_OK
    xg = xd.cpu().numpy()
    for i, s in enumerate(vols):
        ref = sb_oracle.split_bregman(s.y, s.sens, s.mask, v.mu, v.lam, v.gam, levels, 3, v.n_outer, 1,
                                      v.pcg_tol, v.pcg_maxit, 8, "circulant", tau if tau > 0 else None,
                                      tau if tau > 0 else None)
        assert rel(xg[i], ref.x) <= IMG_TOL
    plan.close()


def test_volume_split_bregman_tolerance_mode(torch, sbm):
    v = synth.Volume("32x32x32 Nc3", 32, 32, 32, 3, 4.0, 8, 1.0, 0.05, 0.05, 3, 3, 1, 1e-3, 100, 0, seed=99)
    s = synth.make_volume(v)
    plan = vplan(sbm, torch, s.sens[None], s.mask[None], v.mu, v.lam, v.gam, v.wavelet_levels)
    xd = torch.zeros((1, v.nz, v.ny, v.nx), dtype=torch.complex64, device="cuda")
    st, iters, _ = plan.split_bregman(dev(torch, s.y[None]), xd, v.n_outer, tau_tv=0.02, tau_w=0.02,
                                      tol=v.pcg_tol, maxit=v.pcg_maxit)
    assert st == sbm.SB_OK
    ref = sb_oracle.split_bregman(s.y, s.sens, s.mask, v.mu, v.lam, v.gam, v.wavelet_levels, 3, v.n_outer, 1,
                                  v.pcg_tol, v.pcg_maxit, 0, "circulant", 0.02, 0.02)
    assert all(abs(a - b) <= 1 for a, b in zip(iters[0], ref.iters)), (iters[0], ref.iters)
    assert rel(xd[0].cpu().numpy(), ref.x) <= 1e-3
    plan.close()


def test_volume_unsupported(torch, sbm):
    for (nz, levels, passes) in [(48, 0, 0), (16, 0, 0), (32, 5, 0), (32, 0, 1)]:
        desc = sbm.plan_desc(32, 32, 2, 1, 1.0, 0.1, 0.1, levels, precond_passes=passes, nz=nz)
        with pytest.raises(sbm.SbError) as ei:
            sbm.sb_plan_create(desc, 0)
        assert ei.value.status == sbm.SB_ERR_UNSUPPORTED


def random_volume_mask(nz, ny, nx, frac, rng):
    """An arbitrary 3D sampling pattern: points drawn independently in (k_z, k_y, k_x), DC kept."""
    m = (rng.random((nz, ny, nx)) < frac).astype(np.uint8)
    m[0, 0, 0] = 1
    return m


@pytest.mark.parametrize("nz,ny,nx,nc,nb", [(32, 32, 32, 2, 2), (64, 32, 64, 3, 1)])
def test_volume_arbitrary_mask_operators(torch, sbm, nz, ny, nx, nc, nb):
    # a mask that varies along x too: the general path in five passes (DFT_y, DFT_z, the x pass
    # with the per-point mask, IDFT_z, IDFT_y and combine)
    rng = np.random.default_rng(nz + ny + nx + nc)
    sens = np.stack([synth.coil_maps_3d(nz, ny, nx, nc, rng) for _ in range(nb)])
    mask = np.stack([random_volume_mask(nz, ny, nx, 0.3, rng) for _ in range(nb)])
    mu, lam, gam = 1.0, 0.05, 0.05
    plan = vplan(sbm, torch, sens, mask, mu, lam, gam)
    x = synth.random_complex((nb, nz, ny, nx), rng)
    q = plan.apply_A(dev(torch, x)).cpu().numpy()
    kg = plan.k().cpu().numpy()
    z = plan.apply_precond(dev(torch, x)).cpu().numpy()
    b = synth.random_complex((nb, nz, ny, nx), rng)
    xd = torch.zeros((nb, nz, ny, nx), dtype=torch.complex64, device="cuda")
    st, _ = plan.pcg_solve(dev(torch, b), xd, fixed_iters=6)
    assert st == sbm.SB_OK
    for i in range(nb):
        assert rel(q[i], operators.apply_A(x[i], sens[i], mask[i], mu, lam, gam, 3)) <= OP_TOL
        kref = precond.k_diag(sens[i], mask[i], mu, lam, gam, 3)
        assert np.max(np.abs(kg[i] - kref)) <= OP_TOL * np.max(kref)
        assert rel(z[i], precond.apply_precond(x[i], kref, 3)) <= OP_TOL
        A = lambda v, i=i: operators.apply_A(v, sens[i], mask[i], mu, lam, gam, 3)  # noqa: E731
        kc = precond.clamp_k(kref)
        ref = pcg.pcg(A, b[i], np.zeros((nz, ny, nx), complex), lambda v: precond.apply_precond(v, kc, 3),
                      fixed_iters=6)
        assert rel(xd[i].cpu().numpy(), ref.x) <= IMG_TOL
    plan.close()


@pytest.mark.parametrize("tau", [0.0, 0.02])
def test_volume_arbitrary_mask_split_bregman(torch, sbm, tau):
    # Algorithm 1 on volumes with an arbitrary mask: the right-hand side and the back-projection of
    # the start take the same five passes, the k-space data kept whole
    nz, ny, nx, nc, levels = 32, 32, 32, 3, 2
    rng = np.random.default_rng(2718)
    x_true = synth.ellipsoid_phantom(nz, ny, nx, rng)
    sens = synth.coil_maps_3d(nz, ny, nx, nc, rng)
    mask = random_volume_mask(nz, ny, nx, 0.35, rng)
    y = synth.acquire_nd(x_true, sens, mask, 1e-3, rng)
    mu, lam, gam = 1.0, 0.05, 0.05
    plan = vplan(sbm, torch, sens[None], mask[None], mu, lam, gam, levels)
    xd = torch.zeros((1, nz, ny, nx), dtype=torch.complex64, device="cuda")
    st, _, _ = plan.split_bregman(dev(torch, y[None]), xd, 3, tau_tv=tau, tau_w=tau, fixed_iters=6)
    assert st == sbm.SB_OK
    ref = sb_oracle.split_bregman(y, sens, mask, mu, lam, gam, levels, 3, 3, 1, 1e-3, 100, 6, "circulant",
                                  tau if tau > 0 else None, tau if tau > 0 else None)
    assert rel(xd[0].cpu().numpy(), ref.x) <= IMG_TOL
    plan.close()
