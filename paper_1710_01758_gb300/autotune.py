"""Autotuner for a plan's launch configuration, with a JSON cache per device and geometry.

Choices (none changes the arithmetic of a slice, only the launch shapes and the schedule):
  groups      concurrent slice groups (streams + host threads) of a batch, fixed at plan creation;
  col_tile    columns per CTA of the preconditioner's column pass (the length-ny DFTs of
              M^{-1} = F^H diag(k)^{-1} F): 8, 16 or 32, where they fit;
  poll_every  PCG iterations between convergence polls (and per replayed CUDA-graph block);
  apply_tile  columns per CTA of q = A p where the library has two kernels (2D line masks in
              FP32 at ny = 256 and 512): 8 (p and the accumulator in tensor memory) or 16
              (registers, a two-stage coil-tile ring); tuned after the other three, with their
              best values.
The objective is the wall time of a PCG solve to a relative residual of 1e-3 from x = 0 on the
caller's coils and mask (q = A p and the preconditioner are the whole PCG iteration; the call
returns when the solve has finished), best of `reps` after a warm-up.  Results are cached under
$SB_AUTOTUNE_CACHE (default ~/.cache/paper_1710_01758_gb300/autotune.json), keyed by device name,
geometry, batch and precision mode.
"""
from __future__ import annotations

import json
import os
import tempfile
import time

COL_TILES = (8, 16, 32)
APPLY_TILES = (8, 16)
POLLS = (2, 4, 8)
GROUPS = (1, 2, 4, 8)


def cache_path() -> str:
    p = os.environ.get("SB_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1710_01758_gb300", "autotune.json")


def cache_key(device: str, nx: int, ny: int, ncoils: int, nbatch: int, prec: int = 0, nz: int = 1) -> str:
    shape = f"{nx}x{ny}" + (f"x{nz}" if nz > 1 else "")
    return f"{device}|{shape}|nc{ncoils}|nb{nbatch}|prec{prec}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(data: dict, path: str | None = None) -> None:
    """Atomic replace, so concurrent tuners never leave a torn file."""
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(path) or ".", suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def col_tile_fits(ny: int, nx: int, ct: int) -> bool:
    """The library's rule for the column pass: ct divides nx, at most 1024 threads (ct ny / 16)
    and 160 KB of exchange buffers (2 ny ct complex64 values)."""
    return ct in COL_TILES and nx % ct == 0 and ct * ny // 16 <= 1024 and 2 * ny * ct * 8 <= 160 * 1024


def candidates(nx: int, ny: int, nbatch: int, nz: int = 1):
    """Every (groups, col_tile, poll_every) the library accepts for this geometry."""
    groups = [g for g in GROUPS if g <= nbatch]
    tiles = [ct for ct in COL_TILES if col_tile_fits(ny, nx, ct)] if nz == 1 else [16]
    return [(g, ct, pe) for g in groups for ct in tiles for pe in POLLS]


def apply_tiles(nx: int, ny: int, prec: int = 0, nz: int = 1) -> list:
    """q = A p tiles the library offers for this geometry (the default alone where there is one
    kernel)."""
    return list(APPLY_TILES) if (ny in (256, 512) and nz == 1 and prec == 0) else [APPLY_TILES[0]]


def default_groups(nbatch: int) -> int:
    """The library's choice for groups = 0: one group per 8 slices, at most 4."""
    return max(1, min(4, nbatch // 8, nbatch))


def select(timings: dict) -> tuple:
    """The fastest candidate; ties go to the earlier (smaller) configuration."""
    return min(sorted(timings), key=lambda c: timings[c])


def tune(make_plan, nx: int, ny: int, ncoils: int, nbatch: int, prec: int = 0, nz: int = 1, reps: int = 3,
         use_cache: bool = True, path: str | None = None) -> dict:
    """Time every candidate and return {"groups", "col_tile", "poll_every", "apply_tile", "ms",
    "cached"}.

    make_plan(groups) must return a Plan (paper_1710_01758_gb300.sb.Plan) of this geometry with
    its coils and mask set; the tuner sets the tuning fields itself and closes the plans it made.
    """
    import torch

    device = torch.cuda.get_device_name()
    key = cache_key(device, nx, ny, ncoils, nbatch, prec, nz)
    data = load_cache(path) if use_cache else {}
    if use_cache and key in data:
        return dict(data[key], cached=True)
    shape = (nbatch, nz, ny, nx) if nz > 1 else (nbatch, ny, nx)
    gen = torch.Generator(device="cuda").manual_seed(1710)
    b = torch.complex(torch.randn(shape, device="cuda", generator=gen),
                      torch.randn(shape, device="cuda", generator=gen)).to(torch.complex64)
    timings = {}
    by_groups = {}

    def solve_ms(plan):
        best = None
        for r in range(reps + 1):
            x = torch.zeros(shape, dtype=torch.complex64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            plan.pcg_solve(b, x, tol=1e-3, maxit=200)  # returns after the solve has finished
            ms = 1e3 * (time.perf_counter() - t0)
            if r > 0:  # the first run is the warm-up (graph capture, attributes)
                best = ms if best is None else min(best, ms)
        return best

    for g, ct, pe in candidates(nx, ny, nbatch, nz):
        by_groups.setdefault(g, []).append((ct, pe))
    for g, rest in by_groups.items():
        plan = make_plan(g)
        try:
            for ct, pe in rest:
                plan.set_tuning(col_tile=ct, poll_every=pe, apply_tile=APPLY_TILES[0])
                timings[(g, ct, pe)] = solve_ms(plan)
        finally:
            plan.close()
    g, ct, pe = select(timings)
    at, ms = APPLY_TILES[0], timings[(g, ct, pe)]
    tiles = apply_tiles(nx, ny, prec, nz)
    if len(tiles) > 1:
        plan = make_plan(g)
        try:
            t_at = {APPLY_TILES[0]: ms}
            for a in tiles[1:]:
                plan.set_tuning(col_tile=ct, poll_every=pe, apply_tile=a)
                t_at[a] = solve_ms(plan)
        finally:
            plan.close()
        at = min(sorted(t_at), key=lambda a: t_at[a])
        ms = t_at[at]
    out = {"groups": g, "col_tile": ct, "poll_every": pe, "apply_tile": at, "ms": ms,
           "default_ms": timings.get((default_groups(nbatch), 16, 4))}
    if use_cache:
        store(key, out, path)
    return dict(out, cached=False)


def store(key: str, entry: dict, path: str | None = None) -> bool:
    """Add one entry to the cache file; False when the location cannot be written (the tuning
    result is still used, just not kept)."""
    data = load_cache(path)
    data[key] = entry
    try:
        save_cache(data, path)
    except OSError:
        return False
    return True
