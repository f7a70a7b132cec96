"""Seeded synthetic inputs for PI+CS reconstruction problems.

This module only *simulates an acquisition*: a piecewise-constant ellipse phantom, smooth
Gaussian-profile coil sensitivities normalised to sum(|S_c|^2) = 1 (the normalisation of the
"Coil sensitivity maps" paragraph of the paper's Methods), Cartesian phase-encode line masks
(Methods, "Undersampling"), and noisy undersampled k-space y_c = R (F S_c x + n_c) (the data model
of Eq. ill0).  It holds none of the reconstruction method's arithmetic: no system matrix, no
preconditioner, no CG, no Split Bregman.  Both the FP64 oracle and the CUDA path consume its
arrays; neither is used to produce them.

Conventions shared by every consumer:
  * images are C-ordered ``[ny, nx]`` (2D) with x fastest;
  * coil sensitivities are ``[Nc, ny, nx]``;
  * the mask is ``uint8 [ny, nx]`` in DFT (unshifted) order, 1 = sampled;
  * k-space is ``[Nc, ny, nx]`` in DFT order with zeros off the mask;
  * F is the unitary 2D DFT (forward sign negative).
All arrays are returned in complex128 / float64; a consumer casts them to its own precision.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Seeds of the workloads: seed = SEED_BASE + workload number.
SEED_BASE = 1710017580


def _grid(ny: int, nx: int):
    """Pixel-centre coordinates in [-1, 1) along x and y, shaped [ny, nx]."""
    xs = -1.0 + 2.0 * np.arange(nx) / nx
    ys = -1.0 + 2.0 * np.arange(ny) / ny
    return np.meshgrid(ys, xs, indexing="ij")[::-1]  # (X, Y)


def ellipse_phantom(ny: int, nx: int, rng: np.random.Generator, n_ellipses: int = 12) -> np.ndarray:
    """Piecewise-constant phantom: ``n_ellipses`` ellipses painted in order, each overwriting the
    pixels it covers with an intensity drawn from U[0, 1]; background 0.  Centres U[-0.7, 0.7],
    semi-axes U[0.05, 0.5], rotation U[0, pi).  The magnitude image is multiplied by the smooth
    phase exp(i*pi*(a*x + b*y)), a, b ~ U[-0.5, 0.5]."""
    X, Y = _grid(ny, nx)
    img = np.zeros((ny, nx), np.float64)
    for _ in range(n_ellipses):
        cx, cy = rng.uniform(-0.7, 0.7, 2)
        a, b = rng.uniform(0.05, 0.5, 2)
        th = rng.uniform(0.0, math.pi)
        val = rng.uniform(0.0, 1.0)
        xr = (X - cx) * math.cos(th) + (Y - cy) * math.sin(th)
        yr = -(X - cx) * math.sin(th) + (Y - cy) * math.cos(th)
        img[(xr / a) ** 2 + (yr / b) ** 2 <= 1.0] = val
    pa, pb = rng.uniform(-0.5, 0.5, 2)
    return img * np.exp(1j * math.pi * (pa * X + pb * Y))


def coil_maps(ny: int, nx: int, nc: int, rng: np.random.Generator) -> np.ndarray:
    """Smooth complex coil sensitivities ``[nc, ny, nx]``.

    Coil c sits at angle theta_c = 2*pi*c/nc + theta_0 (theta_0 ~ U[0, 2*pi/nc), one draw per
    slice) on a ring of radius 1.2 around the field of view [-1, 1]^2, with profile
    exp(-|r - r_c|^2 / (2 * 0.6^2)) * exp(i*theta_c).  The maps are then normalised pointwise so
    that sum_c |S_c|^2 = 1 everywhere."""
    X, Y = _grid(ny, nx)
    theta0 = rng.uniform(0.0, 2.0 * math.pi / nc)
    maps = np.empty((nc, ny, nx), np.complex128)
    for c in range(nc):
        th = 2.0 * math.pi * c / nc + theta0
        xc, yc = 1.2 * math.cos(th), 1.2 * math.sin(th)
        prof = np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / (2.0 * 0.6 ** 2))
        maps[c] = prof * np.exp(1j * th)
    maps /= np.sqrt(np.sum(np.abs(maps) ** 2, axis=0, keepdims=True))
    return maps


def line_mask(ny: int, nx: int, accel: float, n_centre: int, rng: np.random.Generator,
              density: str = "uniform") -> np.ndarray:
    """Cartesian mask of fully sampled readout (x) lines at random phase-encode (y) positions.

    round(ny/accel) lines in total, of which the ``n_centre`` lines around k_y = 0 are always
    taken; the rest are drawn without replacement, uniformly (``density='uniform'``) or with
    probability proportional to (1 - |k|/k_max)^2 (``'variable'``).  Returned in DFT order."""
    n_lines = int(round(ny / accel))
    if not (0 < n_centre <= n_lines <= ny):
        raise ValueError("need 0 < n_centre <= round(ny/accel) <= ny")
    kc = np.arange(ny) - ny // 2                      # centred k_y coordinate of each slot
    centre = np.zeros(ny, bool)
    lo = ny // 2 - n_centre // 2
    centre[lo:lo + n_centre] = True
    cand = np.flatnonzero(~centre)
    if density == "uniform":
        p = np.ones(cand.size)
    elif density == "variable":
        p = (1.0 - np.abs(kc[cand]) / (ny / 2.0)) ** 2 + 1e-12
    else:
        raise ValueError(density)
    pick = rng.choice(cand, size=n_lines - n_centre, replace=False, p=p / p.sum())
    lines_centred = centre.copy()
    lines_centred[pick] = True
    lines = np.fft.ifftshift(lines_centred)           # centred order -> DFT order
    return np.repeat(lines[:, None], nx, axis=1).astype(np.uint8)


def random_mask(ny: int, nx: int, accel: float, centre: int, rng: np.random.Generator) -> np.ndarray:
    """Fully random 2D variable-density mask (the paper's second sampling scheme): a fully
    sampled ``centre`` x ``centre`` block plus points drawn with probability proportional to
    (1 - r/r_max)^2, round(ny*nx/accel) points in total.  DFT order."""
    n_pts = int(round(ny * nx / accel))
    ky = (np.arange(ny) - ny // 2)[:, None] / (ny / 2.0)
    kx = (np.arange(nx) - nx // 2)[None, :] / (nx / 2.0)
    rad = np.sqrt(ky ** 2 + kx ** 2) / math.sqrt(2.0)
    m = np.zeros((ny, nx), bool)
    cy, cx = ny // 2 - centre // 2, nx // 2 - centre // 2
    m[cy:cy + centre, cx:cx + centre] = True
    cand = np.flatnonzero(~m.ravel())
    p = (1.0 - rad.ravel()[cand]) ** 2 + 1e-12
    pick = rng.choice(cand, size=max(0, n_pts - int(m.sum())), replace=False, p=p / p.sum())
    m.ravel()[pick] = True
    return np.fft.ifftshift(m).astype(np.uint8)


def acquire(x: np.ndarray, sens: np.ndarray, mask: np.ndarray, sigma: float,
            rng: np.random.Generator) -> np.ndarray:
    """Simulated undersampled acquisition y_c = R (F S_c x + n_c), n_c complex Gaussian with
    independent N(0, sigma^2) real and imaginary parts (data model of Eq. ill0)."""
    coil_imgs = sens * x[None]
    k = np.fft.fft2(coil_imgs, norm="ortho")
    noise = sigma * (rng.standard_normal(k.shape) + 1j * rng.standard_normal(k.shape))
    return (k + noise) * mask[None].astype(np.float64)


def _grid3(nz: int, ny: int, nx: int):
    """Voxel-centre coordinates in [-1, 1) along x, y and z, shaped [nz, ny, nx]."""
    xs = -1.0 + 2.0 * np.arange(nx) / nx
    ys = -1.0 + 2.0 * np.arange(ny) / ny
    zs = -1.0 + 2.0 * np.arange(nz) / nz
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return X, Y, Z


def ellipsoid_phantom(nz: int, ny: int, nx: int, rng: np.random.Generator, n_ellipsoids: int = 12) -> np.ndarray:
    """3D counterpart of ``ellipse_phantom``: ellipsoids painted in order with U[0, 1] intensities
    (centres U[-0.7, 0.7]^3, semi-axes U[0.05, 0.5]^3, orientation from three angles U[0, pi)),
    background 0, times the smooth phase exp(i*pi*(a*x + b*y + c*z)), a, b, c ~ U[-0.5, 0.5]."""
    X, Y, Z = _grid3(nz, ny, nx)
    img = np.zeros((nz, ny, nx), np.float64)
    for _ in range(n_ellipsoids):
        c = rng.uniform(-0.7, 0.7, 3)
        ax = rng.uniform(0.05, 0.5, 3)
        a1, a2, a3 = rng.uniform(0.0, math.pi, 3)
        val = rng.uniform(0.0, 1.0)
        rz = np.array([[math.cos(a1), -math.sin(a1), 0], [math.sin(a1), math.cos(a1), 0], [0, 0, 1]])
        ry = np.array([[math.cos(a2), 0, math.sin(a2)], [0, 1, 0], [-math.sin(a2), 0, math.cos(a2)]])
        rx = np.array([[1, 0, 0], [0, math.cos(a3), -math.sin(a3)], [0, math.sin(a3), math.cos(a3)]])
        rot = rz @ ry @ rx
        d = np.stack([X - c[0], Y - c[1], Z - c[2]], axis=-1) @ rot
        img[np.sum((d / ax) ** 2, axis=-1) <= 1.0] = val
    pa, pb, pc = rng.uniform(-0.5, 0.5, 3)
    return img * np.exp(1j * math.pi * (pa * X + pb * Y + pc * Z))


def coil_maps_3d(nz: int, ny: int, nx: int, nc: int, rng: np.random.Generator) -> np.ndarray:
    """Smooth 3D coil sensitivities ``[nc, nz, ny, nx]``: coils alternate between two rings of
    radius 1.2 at z = -0.5 and z = +0.5, coil c at angle 2*pi*c/nc + theta_0, with the profile
    and phase of ``coil_maps``; normalised pointwise to sum_c |S_c|^2 = 1."""
    X, Y, Z = _grid3(nz, ny, nx)
    theta0 = rng.uniform(0.0, 2.0 * math.pi / nc)
    maps = np.empty((nc, nz, ny, nx), np.complex128)
    for c in range(nc):
        th = 2.0 * math.pi * c / nc + theta0
        xc, yc, zc = 1.2 * math.cos(th), 1.2 * math.sin(th), (-0.5 if c % 2 == 0 else 0.5)
        prof = np.exp(-((X - xc) ** 2 + (Y - yc) ** 2 + (Z - zc) ** 2) / (2.0 * 0.6 ** 2))
        maps[c] = prof * np.exp(1j * th)
    maps /= np.sqrt(np.sum(np.abs(maps) ** 2, axis=0, keepdims=True))
    return maps


def readout_mask_3d(nz: int, ny: int, nx: int, accel: float, centre: int, rng: np.random.Generator) -> np.ndarray:
    """3D Cartesian mask with the readout (x) fully sampled: round(ny*nz/accel) (k_y, k_z) lines,
    a ``centre`` x ``centre`` block around the origin always, the rest drawn without replacement
    with probability proportional to (1 - r/r_max)^2 (variable density); DFT order, [nz, ny, nx]."""
    return np.repeat(random_mask(nz, ny, accel, centre, rng)[:, :, None], nx, axis=2)


def acquire_nd(x: np.ndarray, sens: np.ndarray, mask: np.ndarray, sigma: float,
               rng: np.random.Generator) -> np.ndarray:
    """``acquire`` for images of any dimension (unitary DFT over all image axes)."""
    axes = tuple(range(1, sens.ndim))
    k = np.fft.fftn(sens * x[None], axes=axes, norm="ortho")
    noise = sigma * (rng.standard_normal(k.shape) + 1j * rng.standard_normal(k.shape))
    return (k + noise) * mask[None].astype(np.float64)


@dataclasses.dataclass
class Volume:
    """A 3D PI+CS reconstruction workload (readout along x fully sampled)."""
    name: str
    nz: int
    ny: int
    nx: int
    ncoils: int
    accel: float
    centre: int
    mu: float
    lam: float
    gam: float
    wavelet_levels: int
    n_outer: int
    n_inner: int
    pcg_tol: float
    pcg_maxit: int
    pcg_fixed_iters: int
    sigma: float = 1e-3
    seed: int = SEED_BASE + 5


# 256 x 256 x 128 volume, 16 coils, (k_y, k_z) lines at R = 8 with a 24 x 24 centre, 3D TV +
# 3-level 3D Haar, 15 SB iterations, PCG to 1e-3.
VOLUME_256 = Volume("256x256x128 Nc16 R8 TV+Haar3 15SB PCG-tol1e-3", 128, 256, 256, 16, 8.0, 24,
                    1.0, 0.05, 0.05, 3, 15, 1, 1e-3, 200, 0)


def make_volume(v: Volume, seed: int | None = None) -> "Slice":
    """One seeded volume of ``v`` (arrays [nz, ny, nx] / [Nc, nz, ny, nx])."""
    rng = np.random.default_rng(v.seed if seed is None else seed)
    x = ellipsoid_phantom(v.nz, v.ny, v.nx, rng)
    s = coil_maps_3d(v.nz, v.ny, v.nx, v.ncoils, rng)
    m = readout_mask_3d(v.nz, v.ny, v.nx, v.accel, v.centre, rng)
    y = acquire_nd(x, s, m, v.sigma, rng)
    return Slice(x, s, m, y)


@dataclasses.dataclass
class Workload:
    """A 2D PI+CS reconstruction workload (geometry, regularisation and iteration schedule)."""
    name: str
    ny: int
    nx: int
    ncoils: int
    accel: float
    n_centre: int
    density: str
    mu: float
    lam: float
    gam: float
    wavelet_levels: int
    n_outer: int
    n_inner: int
    pcg_tol: float
    pcg_maxit: int
    pcg_fixed_iters: int          # > 0: run exactly this many PCG iterations per solve
    sigma: float = 1e-3
    seed: int = SEED_BASE
    tau: float = 0.0              # shrink thresholds of steps 6-8; <= 0: 1/lambda and 1/gamma


# 128x128, 4 coils, R=4 lines + 16 centre lines, TV only, 10 SB x 20 fixed PCG iterations.
SMALL_128 = Workload("128x128 Nc4 R4 TV-only 10SBx20PCG", 128, 128, 4, 4.0, 16, "uniform",
                     1.0, 0.1, 0.0, 0, 10, 1, 1e-3, 20, 20, seed=SEED_BASE + 1)
# 256x256, 12 coils, R=4 lines + 24 centre lines, TV + 4-level Haar, 20 SB, PCG to 1e-3.
METRIC_256 = Workload("256x256 Nc12 R4 TV+Haar4 20SB PCG-tol1e-3", 256, 256, 12, 4.0, 24, "uniform",
                      1.0, 0.05, 0.05, 4, 20, 1, 1e-3, 200, 0, seed=SEED_BASE + 2)


# 256x256, 12 coils, random 2D variable-density points at R=4 with a 24 x 24 centre, TV + 4-level
# Haar, 20 SB, PCG to 1e-3 (the paper's second sampling scheme).
RANDOM_256 = Workload("256x256 Nc12 R4 random-2D TV+Haar4 20SB PCG-tol1e-3", 256, 256, 12, 4.0, 24, "random",
                      1.0, 0.05, 0.05, 4, 20, 1, 1e-3, 200, 0, seed=SEED_BASE + 6)
# The benchmark geometry with active shrinkage: thresholds 0.02 instead of 1/lambda = 1/gamma = 20
# (at which, for images in [0, 1], every shrink output stays zero and steps 6-11 do no work).
SHRINK_256 = dataclasses.replace(METRIC_256, name="256x256 Nc12 R4 TV+Haar4 tau0.02 20SB PCG-tol1e-3",
                                 tau=0.02, seed=SEED_BASE + 7)
# The paper's parameter sets 1-3 (Methods, "Reconstruction") on the benchmark geometry, thresholds
# 0.02 so that shrinkage is active on these synthetic images.
PARAM_SETS = {"set1": (1e-3, 4e-3, 1e-3), "set2": (1e-2, 4e-3, 1e-3), "set3": (1e-3, 4e-3, 4e-3)}
PARAM_256 = {k: dataclasses.replace(METRIC_256, name=f"256x256 Nc12 R4 TV+Haar4 {k} mu{mu:g} lam{lam:g} gam{gam:g} "
                                                     "tau0.02 20SB PCG-tol1e-3",
                                    mu=mu, lam=lam, gam=gam, tau=0.02, seed=SEED_BASE + 8 + i)
             for i, (k, (mu, lam, gam)) in enumerate(PARAM_SETS.items())}
# 512x512, 32 coils, R=6 variable-density lines + 32 centre lines, TV + 4-level Haar, 20 SB.
LARGE_512 = Workload("512x512 Nc32 R6vd TV+Haar4 20SB PCG-tol1e-3", 512, 512, 32, 6.0, 32, "variable",
                     1.0, 0.05, 0.05, 4, 20, 1, 1e-3, 200, 0, seed=SEED_BASE + 3)

# The uneven batch: per slice a seeded choice of image size, coil count and acceleration.
# Sizes are (ny, nx): 192 x 192, 256 x 224 (x by y), 320 x 320 and 384 x 320 (x by y).
UNEVEN_SIZES = ((192, 192), (224, 256), (320, 320), (320, 384))
UNEVEN_COILS = (8, 12, 16, 32)
UNEVEN_ACCEL = (3.0, 4.0, 6.0)
UNEVEN_SEED = SEED_BASE + 4


def uneven_workloads(n: int = 64, seed: int = UNEVEN_SEED) -> list[Workload]:
    """Workloads of the ``n`` slices of the uneven batch: size, coils and R drawn per slice
    (uniform over UNEVEN_SIZES x UNEVEN_COILS x UNEVEN_ACCEL), 16 centre lines, uniform line
    density, TV + 4-level Haar and the weights and schedule of METRIC_256."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        ny, nx = UNEVEN_SIZES[int(rng.integers(len(UNEVEN_SIZES)))]
        nc = UNEVEN_COILS[int(rng.integers(len(UNEVEN_COILS)))]
        accel = UNEVEN_ACCEL[int(rng.integers(len(UNEVEN_ACCEL)))]
        out.append(Workload(f"{nx}x{ny} Nc{nc} R{accel:g} TV+Haar4", ny, nx, nc, accel, 16, "uniform",
                            1.0, 0.05, 0.05, 4, 20, 1, 1e-3, 200, 0, seed=seed))
    return out


def uneven_slice(wls: list[Workload], i: int) -> "Slice":
    """Slice i of the uneven batch (seed = batch seed * 1000 + i)."""
    return make_slice(wls[i], wls[i].seed * 1000 + i)


@dataclasses.dataclass
class Slice:
    x_true: np.ndarray    # complex128 [ny, nx]
    sens: np.ndarray      # complex128 [Nc, ny, nx]
    mask: np.ndarray      # uint8 [ny, nx], DFT order
    y: np.ndarray         # complex128 [Nc, ny, nx], zeros off-mask


def make_slice(wl: Workload, seed: int | None = None) -> Slice:
    """One seeded slice of workload ``wl`` (seed defaults to ``wl.seed``)."""
    rng = np.random.default_rng(wl.seed if seed is None else seed)
    x = ellipse_phantom(wl.ny, wl.nx, rng)
    s = coil_maps(wl.ny, wl.nx, wl.ncoils, rng)
    if wl.density == "random":  # random 2D points with an n_centre x n_centre centre block
        m = random_mask(wl.ny, wl.nx, wl.accel, wl.n_centre, rng)
    else:
        m = line_mask(wl.ny, wl.nx, wl.accel, wl.n_centre, rng, wl.density)
    y = acquire(x, s, m, wl.sigma, rng)
    return Slice(x, s, m, y)


def make_batch(wl: Workload, nbatch: int, seed: int | None = None) -> list[Slice]:
    """``nbatch`` independent slices; slice i uses seed (seed or wl.seed) * 1000 + i."""
    base = wl.seed if seed is None else seed
    return [make_slice(wl, base * 1000 + i) for i in range(nbatch)]


def random_complex(shape, rng: np.random.Generator) -> np.ndarray:
    """Standard complex Gaussian test vector (real and imaginary parts N(0, 1))."""
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
