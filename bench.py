#!/usr/bin/env python
"""Throughput of batched PI+CS reconstruction with circulant-preconditioned PCG inside Split
Bregman (arXiv 1710.01758) on one node.

Workload (one "step"): a batch of independent 256x256 slices, 12 coils each, Cartesian line
masks at R = 4 with 24 fully sampled centre lines, TV + 4-level Haar, mu = 1, lambda = gamma =
0.05, 20 Split Bregman iterations with PCG to relative residual 1e-3.  A step runs the whole
hot path: k construction from the coils and mask (sb_set_mask), then Split Bregman
(sb_split_bregman: right-hand sides, PCG solves, shrink / Bregman updates, data add-back).
Inputs are seeded synthetic phantoms, coil maps and masks, resident in HBM before timing; the
batch (about 0.9 GB of coil maps and k-space) is larger than L2.

Metric: PCG iterations per second summed over the batch (value) and reconstructions per second;
the dominant kernel's achieved HBM bandwidth against the measured peak; the image error against
the FP64 oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload 256|128|512|uneven64]

The default workload is the one above; --workload selects further measurement lines: 512 x 128
slices of 128x128 x 4 coils (TV only, 10 Split Bregman x 20 fixed PCG iterations), 8 slices of
512x512 x 32 coils (R = 6 variable-density lines), or 64 uneven slices (sizes 192x192 to 384x320,
8-32 coils, R = 3/4/6) solved as one plan per geometry, concurrently.

Multi-GPU (torchrun): each rank reconstructs its own batch (weak scaling, no collective on the
data path); rank 0 prints one JSON line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PCG iters/s and recon/s at 256²×12 coils; HBM GB/s vs peak; err vs FP64"
UNIT = "PCG iter/s"
HBM_FALLBACK_GBS = 6800.0
# FP32 lanes per SM (the FP32 CUDA-core peak is SMs x lanes x 2 flops (FMA) x the SM clock)
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) of one q = A p launch (k_apply_A8) over the full 64-slice 256x256x12
# batch: an ncu capture of a 32-slice launch (231.76 MB read + 10.52 MB written) scaled by the
# slices processed.  Set to None whenever the kernel changes until it is captured again.
TRAFFIC_K1 = 2 * (231.76e6 + 10.52e6)
# --prec: (sb_precision, dtype label of the JSON line)
PRECS = {"fp32": (0, "fp32"), "split-bf16": (1, "bf16x2 split, fp32 accumulate (tensor-core DFT stages)"),
         "split-fp16": (2, "fp16x2 split, fp32 accumulate (tensor-core DFT stages)")}
# workloads: name -> (synth workload attribute, default batch).  The default is the headline
# configuration; the others are further measurement lines (batches sized above L2).
WORKLOADS = {"256": ("METRIC_256", 64), "128": ("SMALL_128", 512), "512": ("LARGE_512", 8),
             "random256": ("RANDOM_256", 64), "shrink256": ("SHRINK_256", 64),
             "set1": ("PARAM_256:set1", 64), "set2": ("PARAM_256:set2", 64), "set3": ("PARAM_256:set3", 64)}


def workload_of(synth, name):
    """The synth workload behind a --workload name (``ATTR`` or ``ATTR:key`` of a dict)."""
    attr = WORKLOADS[name][0]
    if ":" in attr:
        a, k = attr.split(":")
        return getattr(synth, a)[k]
    return getattr(synth, attr)


def sm_count(dev) -> int:
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["uneven64", "volume"], default="256",
                    help="256: 256x256x12 (default); 128: 128x128x4; 512: 512x512x32; uneven64: 64 slices "
                         "of mixed size / coils / R, one plan per geometry, solved concurrently; volume: "
                         "256x256x128 x 16 coils, (ky, kz) lines at R 8; random256: 256x256x12 with random "
                         "2D k-space points; shrink256: the default with shrink thresholds 0.02 (active "
                         "shrinkage); set1..set3: the paper's weight sets on the default geometry, "
                         "thresholds 0.02")
    ap.add_argument("--batch", type=int, default=0, help="slices per step (0 = the workload's default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-loop", action="store_true", help="uneven64: skip the per-slice loop comparison")
    ap.add_argument("--no-pcg-iter", action="store_true",
                    help="skip the standalone PCG-iteration measurement after the timed region")
    ap.add_argument("--autotune", action="store_true",
                    help="choose slice groups, the preconditioner's column tile and the poll interval with the "
                         "library's autotuner (timed before the measured region, cached per geometry)")
    ap.add_argument("--groups", type=int, default=0, help="concurrent slice groups (0 = library default)")
    ap.add_argument("--general-passes", type=int, choices=[0, 1, 3], default=0,
                    help="random-mask workloads: q = A p as one cluster launch (1) or three passes through a coil "
                         "scratch (3); 0 = library default")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch the PCG iteration blocks directly instead of replaying captured CUDA graphs")
    ap.add_argument("--prec", choices=list(PRECS), default="fp32",
                    help="fp32, or a split-precision mode: the radix-16 DFT stages of q = A p on the tensor cores "
                         "with operands split in two bf16 / fp16 terms and FP32 accumulation (ny = 256 or 512)")
    ap.add_argument("--wavelet", choices=["haar", "daub4"], default="haar",
                    help="W of Algorithm 1 (daub4: the paper's Daubechies-4; 2D workloads)")
    ap.add_argument("--compress", type=int, default=0,
                    help="coil compression to this many virtual coils inside every step (0 = off)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while active; only the rows
    written after start() returns (the timed region) are summarised."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.skip = 0

    def _rows_written(self) -> int:
        with open(self.path) as fh:
            return sum(1 for _ in fh)

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # nvidia-smi takes a moment to start: wait for its first row, so that the rows written
            # from here on fall inside the timed region that follows
            t0 = time.time()
            while time.time() - t0 < 3.0 and self.proc.poll() is None and self._rows_written() == 0:
                time.sleep(0.02)
            self.skip = self._rows_written()
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if len(rows) > self.skip:  # else keep every row (a region shorter than one interval)
            rows = rows[self.skip:]
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        smax = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(rows)}


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s batch: every rank reconstructs its own independent slices (weak
    scaling over ranks, no data exchanged); rank 0 uses the workload's own seed."""
    return seed + 7919 * rank


def reduce_over_ranks(dist, device, elapsed: float, units: int):
    """(max over ranks of the elapsed time, sum over ranks of the work units)."""
    import torch
    t = torch.tensor([elapsed, float(units)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), int(round(float(t[1])))


def make_inputs(wl, nbatch, seed):
    import numpy as np
    from paper_1710_01758_gb300 import synth
    slices = synth.make_batch(wl, nbatch, seed)
    sens = np.ascontiguousarray(np.stack([s.sens for s in slices]).astype(np.complex64))
    mask = np.ascontiguousarray(np.stack([s.mask for s in slices]))
    y = np.ascontiguousarray(np.stack([s.y for s in slices]).astype(np.complex64))
    return slices, sens, mask, y


def oracle_recon(wl, s, n_outer=None, wavelet="haar", nv=0, with_active=False):
    """The FP64 oracle on one slice (coil-compressed to nv virtual coils by the oracle's own
    compression if 0 < nv < Nc); returns (x, total PCG iterations, seconds) and, with
    ``with_active``, the mean fraction of non-zero shrink outputs over the solves."""
    from oracle import coil_compression as cc, split_bregman as sbo
    t0 = time.perf_counter()
    y, sens = s.y, s.sens
    if 0 < nv < sens.shape[0]:
        A, _ = cc.compression_matrix(y, nv)
        y, sens = cc.compress(y, sens, A)
    tau = getattr(wl, "tau", 0.0)
    r = sbo.split_bregman(y, sens, s.mask, wl.mu, wl.lam, wl.gam, wl.wavelet_levels, 2,
                          wl.n_outer if n_outer is None else n_outer, wl.n_inner, wl.pcg_tol, wl.pcg_maxit,
                          wl.pcg_fixed_iters, wavelet=wavelet, tau_tv=tau if tau > 0 else None,
                          tau_w=tau if tau > 0 else None)
    secs = time.perf_counter() - t0
    if with_active:
        return r.x, int(sum(r.iters)), secs, (float(sum(r.shrink_nonzero) / len(r.shrink_nonzero))
                                              if r.shrink_nonzero else 0.0)
    return r.x, int(sum(r.iters)), secs


def _oracle_worker(job):
    """One slice through the oracle in a spawned worker process (no CUDA in the worker)."""
    wl, s, n_outer, wavelet, nv = job
    return oracle_recon(wl, s, n_outer, wavelet=wavelet, nv=nv, with_active=True)


def _oracle_warm(_):
    import numpy  # noqa: F401
    from oracle import split_bregman  # noqa: F401
    return 0


def oracle_pool(n):
    """n spawned worker processes for the oracle, started and warmed (imports done) before any
    timing; numpy's own thread pools are pinned to one thread per process."""
    import multiprocessing as mp
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"  # inherited by the spawned workers
    pool = mp.get_context("spawn").Pool(n)
    pool.map(_oracle_warm, range(n), chunksize=1)
    return pool


def oracle_parallel(pool, wl, slices, n_outer=None, wavelet="haar", nv=0):
    """The oracle, as it stands, on several slices at once, one per worker process.  Returns (x of
    the first slice, total PCG iterations, wall seconds, summed per-process seconds, slices, mean
    fraction of non-zero shrink outputs)."""
    t0 = time.perf_counter()
    res = pool.map(_oracle_worker, [(wl, s, n_outer, wavelet, nv) for s in slices], chunksize=1)
    wall = time.perf_counter() - t0
    return (res[0][0], sum(r[1] for r in res), wall, sum(r[2] for r in res), len(slices),
            sum(r[3] for r in res) / len(res))


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def host_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return 1


def workload_config(wl, nbatch, extra=None):
    cfg = {"workload": f"{nbatch} x [{wl.name}]", "nx": wl.nx, "ny": wl.ny, "ncoils": wl.ncoils,
           "batch_slices": nbatch, "accel": wl.accel, "centre_lines": wl.n_centre, "mu": wl.mu,
           "lambda": wl.lam, "gamma": wl.gam, "haar_levels": wl.wavelet_levels, "n_outer": wl.n_outer,
           "n_inner": wl.n_inner, "pcg_tol": wl.pcg_tol, "precond": "circulant",
           "shrink_thresholds": (wl.tau if getattr(wl, "tau", 0.0) > 0 else "1/lambda, 1/gamma"),
           "l2": "inputs larger than L2 (coil maps + k-space of the batch)"}
    if extra:
        cfg.update(extra)
    return cfg


# --------------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The FP64 oracle, as it stands, timed on the host cores on a bounded sample of the workload
    (one slice per host core, one worker process each, the first 4 Split Bregman iterations, per
    step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1710_01758_gb300 import synth
    wl = synth.METRIC_256
    cores = max(1, min(host_cores(), 64))
    slices = [synth.make_slice(wl, wl.seed * 1000 + i) for i in range(cores)]
    n_outer = 4
    iters, secs = 0, 0.0
    with oracle_pool(cores) as pool:
        for _ in range(args.warmup):
            oracle_parallel(pool, wl, slices, n_outer)
        for _ in range(args.steps):
            _, it, wall, _, _, _ = oracle_parallel(pool, wl, slices, n_outer)
            iters += it
            secs += wall
    value = iters / secs
    sample = (f"{cores} slices of the batch, one per process on {cores} host cores, first {n_outer} of "
              f"{wl.n_outer} Split Bregman iterations per step")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(wl, WORKLOADS["256"][1], {"sample": sample}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1710_01758_gb300 import build as build_mod
    build_mod.build()
    from paper_1710_01758_gb300 import sb, synth

    if args.workload == "uneven64":
        return run_uneven(args, torch, sb, synth, world, rank, local, dist)
    if args.workload == "volume":
        return run_volume(args, torch, sb, synth, world, rank, local, dist)
    default_b = WORKLOADS[args.workload][1]
    wl = workload_of(synth, args.workload)
    B = args.batch or default_b
    pcg_kw = ({"fixed_iters": wl.pcg_fixed_iters} if wl.pcg_fixed_iters > 0
              else {"tol": wl.pcg_tol, "maxit": wl.pcg_maxit})
    t0 = time.perf_counter()
    slices, sens_h, mask_h, y_h = make_inputs(wl, B, rank_seed(wl.seed, rank))
    log(f"[bench] rank {rank}: generated {B} slices in {time.perf_counter() - t0:.1f}s")
    dev = torch.device("cuda", local)
    d_sens = torch.from_numpy(sens_h).to(dev)
    d_mask = torch.from_numpy(mask_h).to(dev)
    d_y = torch.from_numpy(y_h).to(dev)
    x = torch.zeros((B, wl.ny, wl.nx), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)
    wav = sb.SB_WAVELET_DAUB4 if args.wavelet == "daub4" else sb.SB_WAVELET_HAAR
    ncv = args.compress if 0 < args.compress < wl.ncoils else wl.ncoils
    prec, dtype_label = PRECS[args.prec]
    tuned = None
    groups = args.groups
    if args.autotune and ncv == wl.ncoils:
        from paper_1710_01758_gb300 import autotune

        def make(g):
            p = sb.Plan(wl.nx, wl.ny, ncv, B, wl.mu, wl.lam, wl.gam, wl.wavelet_levels, stream=stream, groups=g,
                        wavelet=wav, prec=prec)
            p.set_coils(d_sens)
            p.set_mask(d_mask)
            return p

        t0 = time.perf_counter()
        tuned = autotune.tune(make, wl.nx, wl.ny, ncv, B, prec)
        tuned["tuning_s"] = round(time.perf_counter() - t0, 2)
        log(f"[bench] autotune: {tuned}")
        groups = tuned["groups"]
    plan = sb.Plan(wl.nx, wl.ny, ncv, B, wl.mu, wl.lam, wl.gam, wl.wavelet_levels, stream=stream,
                   groups=groups, wavelet=wav, prec=prec)
    if args.no_graphs:
        plan.set_graphs(False)
    if args.general_passes:
        plan.set_tuning(general_passes=args.general_passes)
    if tuned:
        plan.set_tuning(col_tile=tuned["col_tile"], poll_every=tuned["poll_every"],
                        apply_tile=tuned.get("apply_tile", 0))

    def step(ys=d_y, ss=d_sens, ms=d_mask, xx=x):
        if ncv < wl.ncoils:  # coil compression (Methods, "Coil Compression") is part of the step
            ys, ss, _, _ = sb.coil_compress(ys, ss, ncv, stream)
        plan.set_coils(ss)
        plan.set_mask(ms)
        st, iters, _ = plan.split_bregman(ys, xx, wl.n_outer, wl.n_inner, tau_tv=wl.tau, tau_w=wl.tau, **pcg_kw)
        if st != sb.SB_OK:
            raise RuntimeError(f"split_bregman: {sb.status_string(st)}")
        return int(sum(sum(i) for i in iters)), iters

    for _ in range(args.warmup):
        step()
    # the timed steps run without the per-kernel-class event timer (two event records around
    # every launch cost throughput); the split of a step comes from one extra step afterwards
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = sb.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    total_iters = 0
    iters_last = None
    for _ in range(args.steps):
        it, iters_last = step()
        total_iters += it
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = sb.kernel_launches() - launches0
    clocks = sampler.stop()
    if dist:
        dist.barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    # where one step's time goes: one extra untimed step of the same batch as ONE slice group
    # (one stream, so the per-launch event times do not overlap and add up to the step), the
    # event timer on every kernel class (direct launches: the timer turns graph replay off)
    split = None
    if ncv == wl.ncoils:
        one = sb.Plan(wl.nx, wl.ny, ncv, B, wl.mu, wl.lam, wl.gam, wl.wavelet_levels, stream=stream, groups=1,
                      wavelet=wav, prec=prec)
        if tuned:
            one.set_tuning(col_tile=tuned["col_tile"], poll_every=tuned["poll_every"],
                           apply_tile=tuned.get("apply_tile", 0))
        one.set_timing((1 << sb.SB_KCLASS_COUNT) - 1)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        one.set_coils(d_sens)
        one.set_mask(d_mask)
        xs1 = torch.zeros_like(x)
        st1, it1, _ = one.split_bregman(d_y, xs1, wl.n_outer, wl.n_inner, tau_tv=wl.tau, tau_w=wl.tau, **pcg_kw)
        s1.record(stream)
        torch.cuda.synchronize()
        step_ms = s0.elapsed_time(s1)
        timing1 = {sb.KCLASS_NAMES[c]: one.timing(c) for c in range(sb.SB_KCLASS_COUNT)}
        one.close()
        kern_ms = sum(v[1] for v in timing1.values())
        split = {"step_ms": round(step_ms, 3), "pcg_iterations": int(sum(sum(i) for i in it1)),
                 "classes": {k: {"launches": v[0], "ms": round(v[1], 3), "share_of_step": round(v[1] / step_ms, 4)}
                             for k, v in timing1.items() if v[0]},
                 "host_polls_and_gaps_ms": round(step_ms - kern_ms, 3),
                 "host_polls_and_gaps_share": round((step_ms - kern_ms) / step_ms, 4),
                 "how": "one extra untimed step of the same batch as one slice group on one stream, CUDA events "
                        "around every launch (no graph replay); the shares add up to that step"}
    total_all = total_iters
    elapsed_max = elapsed
    if dist:
        elapsed_max, total_all = reduce_over_ranks(dist, dev, elapsed, total_iters)
    value = total_all / elapsed_max
    recon_per_s = args.steps * B * world / elapsed_max

    # dominant kernel: q = A p.  Algorithmic bytes per slice and application (the same for every
    # mask): p and S read, q written, (2 + Nc) 8 N.  The general path (arbitrary masks: three
    # passes through a coil scratch) moves more, (48 Nc + 24) N: S twice, the scratch written and
    # read three times, p twice, q once; that is reported beside, as its own figure
    n = wl.nx * wl.ny
    general = wl.density == "random"
    cluster = general and plan.tuning()["general_passes"] == 1 and wl.nx in (64, 128, 256) and wl.ny in (64, 128, 256)
    bytes_per_slice_iter = (2 + ncv) * 8 * n
    impl_bytes_per_slice_iter = ((48 * ncv + 24) if general and not cluster else (2 + ncv) * 8) * n
    a_label = ("q = A p: k_apply_A_cl (one cluster launch)" if cluster else
               "q = A p: k_g3_fwd_y + k_g2_x + k_g3_inv_y" if general else
               "k_apply_A8 (q = A p)" if (wl.ny == 256 and plan.tuning()["apply_tile"] == 8 and prec == 0)
               else "k_apply_A (q = A p)")
    peak, peak_kind = peaks()
    # the dominant kernel timed alone over the whole batch (every slice active), same kernel and
    # launch configuration as in the step, right after the timed region
    plan.set_timing(1 << sb.SB_KCLASS_APPLY_A)
    qbuf = torch.empty_like(x)
    n_apply = 20
    for _ in range(n_apply):
        plan.apply_A(x, qbuf)
    k1_alone_n, k1_alone_ms = plan.timing(sb.SB_KCLASS_APPLY_A)
    plan.set_timing(0)
    k1_alone_us = 1e3 * k1_alone_ms / n_apply  # per application of A (one or three launches)
    achieved = B * bytes_per_slice_iter / (k1_alone_us / 1e6) / 1e9
    # the whole PCG iteration (q = A p and the preconditioner step with the CG updates) timed alone
    # over the batch, as the step runs it (slice groups, graphs): fixed-iteration solves of 24 and
    # 8 iterations, the difference over 16 iterations (no solve start-up in it).  Algorithmic bytes
    # per slice and iteration with a fused schedule: q = A p reads p and S and writes q,
    # (16 + 8 Nc) N; M^{-1} reads r, q, 1/k and writes r, z, 36 N; the update reads x, p, z and
    # writes x, p, 40 N: (92 + 8 Nc) N.  The three-pass M^{-1} built here adds the round trip of its
    # intermediate t: (108 + 8 Nc) N, reported as implementation bytes
    bytes_pcg_iter = (92 + 8 * ncv) * n
    impl_bytes_pcg_iter = (108 + 8 * ncv) * n
    pcg_iter = None
    if not general and not args.no_pcg_iter:
        gen = torch.Generator(device=dev).manual_seed(11)
        bvec = torch.complex(torch.randn(x.shape, device=dev, generator=gen),
                             torch.randn(x.shape, device=dev, generator=gen)).to(torch.complex64)

        short = []  # slices whose fixed-length solve stopped early (CG breakdown once converged)

        def pcg_time(n_it):
            xs = torch.zeros_like(x)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            # returns when the solve has finished; a well-conditioned system can reach rounding
            # level within n_it iterations and then break down (p^H A p <= 0): such a slice stops
            # early, which the timing below must not count as iterations
            _, res = sb.sb_pcg_solve(plan.handle, bvec.data_ptr(), xs.data_ptr(), sb.pcg_opts(fixed_iters=n_it), B,
                                     allow=(sb.SB_ERR_NOT_CONVERGED, sb.SB_ERR_BREAKDOWN, sb.SB_ERR_NONFINITE))
            short.extend(i for i, r in enumerate(res) if r[0] < n_it)
            return time.perf_counter() - t0

        pcg_time(24), pcg_time(8)
        t24 = min(pcg_time(24) for _ in range(3))
        t8 = min(pcg_time(8) for _ in range(3))
        it_us = 1e6 * (t24 - t8) / 16
        gbs = B * bytes_pcg_iter / (it_us / 1e6) / 1e9
        if short:  # fewer than 24 iterations ran in some slice: no valid per-iteration time
            pcg_iter = {"us": None, "frac": None, "note": f"{len(set(short))} slices stopped before the fixed "
                                                            "iteration count (converged to rounding level, CG breakdown)"}
        else:
            pcg_iter = {"us": it_us, "achieved_gbs": gbs, "peak": peak, "frac": gbs / peak,
                        "algorithmic_bytes_per_iteration": B * bytes_pcg_iter,
                        "bytes_rule": "(92 + 8 Nc) N per slice (fused schedule: q = A p, M^{-1}, updates)",
                        "implementation_bytes_per_iteration": B * impl_bytes_pcg_iter,
                        "how": f"fixed 24- and 8-iteration PCG solves over the {B}-slice batch (slice groups, "
                               "graphs), best of 3 each, difference / 16"}

    # untimed diagnostics (rank 0): preconditioned vs plain CG iteration counts on a sub-batch,
    # image error vs the FP64 oracle, the oracle's own throughput
    extra = {}
    if rank == 0 and ncv == wl.ncoils:
        nsub = min(8, B)
        sub = sb.Plan(wl.nx, wl.ny, wl.ncoils, nsub, wl.mu, wl.lam, wl.gam, wl.wavelet_levels, stream=stream,
                      wavelet=wav, prec=prec)
        sub.set_coils(d_sens[:nsub].contiguous())
        sub.set_mask(d_mask[:nsub].contiguous())
        xs = torch.zeros((nsub, wl.ny, wl.nx), dtype=torch.complex64, device=dev)
        _, it_plain, _ = sub.split_bregman(d_y[:nsub].contiguous(), xs, wl.n_outer, wl.n_inner,
                                           tau_tv=wl.tau, tau_w=wl.tau, precond=sb.SB_PRECOND_NONE, **pcg_kw)
        sub.close()
        it_pre = iters_last[:nsub]
        extra["pcg_iters_per_solve"] = {
            "circulant": round(float(np.mean(it_pre)), 3), "plain_cg": round(float(np.mean(it_plain)), 3),
            "reduction": round(float(np.sum(it_plain)) / max(1, float(np.sum(it_pre))), 3),
            "first_solve": [round(float(np.mean([i[0] for i in it_plain])), 2),
                            round(float(np.mean([i[0] for i in it_pre])), 2)],
            "last_solve": [round(float(np.mean([i[-1] for i in it_plain])), 2),
                           round(float(np.mean([i[-1] for i in it_pre])), 2)],
            "first_last_order": "[plain CG, circulant]",
            "paper_context": "paper (MATLAB, in-vivo spine, parameter set 1): 6x fewer iterations in the first "
                             "and 3.5x in the last Split Bregman iteration, 4.65x overall (Results, Fig. 5a "
                             "paragraph); context, not a target",
            "slices": nsub}
    if rank == 0:
        if not args.no_cpu_baseline:
            ncpu = max(1, min(host_cores(), B))
            with oracle_pool(ncpu) as pool:
                x_or, it_or, wall, busy, nproc, act = oracle_parallel(pool, wl, slices[:ncpu],
                                                                      wavelet=args.wavelet, nv=ncv)
            xg = x[0].cpu().numpy()
            extra["err_vs_fp64"] = float(np.linalg.norm(xg - x_or) / np.linalg.norm(x_or))
            extra["shrink_active_frac"] = {"value": act, "how": "FP64 oracle on the sampled slices: mean over the "
                                           "solves of the fraction of non-zero shrink outputs (steps 6-8)"}
            extra["cpu_baseline"] = {"value": it_or / wall, "unit": UNIT, "cores": nproc, "kind": "oracle",
                                     "sample": f"slices 0..{nproc - 1} of the batch, one per process on {nproc} "
                                               f"host cores, full {wl.n_outer}-iteration Split Bregman, FP64 numpy",
                                     "per_core": it_or / busy}

    # end to end through the public API with host buffers (pinned), copies inside the timed region:
    # the inputs of step i + 1 are copied on a second stream into the other of two device buffer
    # sets while step i computes (step i - 1, the last user of that set, has returned: the call
    # synchronises); the result of every step is read back on the compute stream
    e2e = None
    if not args.no_e2e:
        hs = torch.from_numpy(sens_h).pin_memory()
        hm = torch.from_numpy(mask_h).pin_memory()
        hy = torch.from_numpy(y_h).pin_memory()
        hx = torch.empty((B, wl.ny, wl.nx), dtype=torch.complex64).pin_memory()
        h2d = hs.numel() * 8 + hm.numel() + hy.numel() * 8
        d2h = hx.numel() * 8
        bufs = [(d_sens, d_mask, d_y), (torch.empty_like(d_sens), torch.empty_like(d_mask), torch.empty_like(d_y))]
        copy_stream = torch.cuda.Stream(dev)
        copied = [torch.cuda.Event(), torch.cuda.Event()]

        def upload(k):
            with torch.cuda.stream(copy_stream):
                for dst, src in zip(bufs[k], (hs, hm, hy)):
                    dst.copy_(src, non_blocking=True)
                copied[k].record(copy_stream)

        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        copy_stream.wait_event(e0)
        e2e_iters = 0
        upload(0)
        for i in range(args.steps):
            k = i % 2
            stream.wait_event(copied[k])
            if i + 1 < args.steps:
                upload(1 - k)
            ss, ms, ys = bufs[k]
            it, _ = step(ys, ss, ms, x)
            e2e_iters += it
            hx.copy_(x, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e_el = e0.elapsed_time(e1) / 1e3
        if dist:
            e_el, e2e_iters = reduce_over_ranks(dist, dev, e_el, e2e_iters)
        e2e = {"value": e2e_iters / e_el, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    plan.close()
    alu = alu_side(wl, B, ncv, k1_alone_us, clocks, general, sm_count(dev))
    hbm_floor_us = B * bytes_per_slice_iter / (peak * 1e9) * 1e6
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": dtype_label, "scalars": "fp64", "data": "synthetic",
                "config": workload_config(wl, B, {"parallelism": f"{world} ranks x independent batches",
                                                  "wavelet": args.wavelet, "virtual_coils": ncv,
                                                  "precision": args.prec, "autotune": tuned,
                                                  "graphs": not args.no_graphs}),
                "recon_per_s": recon_per_s,
                "pcg_iters_per_step": total_all / args.steps,
                "roofline": roofline_line(a_label, achieved, peak, alu, hbm_floor_us, {
                             "frac": (achieved / peak) if achieved else None,
                             "traffic": TRAFFIC_K1 if (args.workload == "256" and B == 64) else None,
                             "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                             else "fallback",
                             "timing": f"timed alone: {n_apply} applications ({k1_alone_n} launches) over the "
                                       f"{B}-slice batch, CUDA events on the plan stream, after the timed region",
                             "algorithmic_bytes_per_launch": B * bytes_per_slice_iter,
                             "bytes_rule": "(2 + Nc) 8 N per slice: p and S read, q written",
                             "implementation_bytes_per_launch": B * impl_bytes_per_slice_iter,
                             "implementation_over_algorithmic": impl_bytes_per_slice_iter / bytes_per_slice_iter,
                             "mean_launch_us": k1_alone_us}),
                "pcg_iteration": pcg_iter,
                "tensor_core": tensor_core_rate(args, wl, B, ncv, k1_alone_us),
                "step_split": split,
                "gpu_launches": int(launches),
                "clocks": clocks, "e2e": e2e}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def roofline_line(kernel, achieved_gbs, peak_gbs, alu, hbm_floor_us, rest):
    """The dominant kernel's roofline object: bound by the larger of its two floors, HBM bytes at
    the measured copy peak or FP32 flops at the derived CUDA-core peak.  Both sides are kept; the
    top-level achieved / peak / frac are the binding side's."""
    hbm = dict(rest, achieved=achieved_gbs, peak=peak_gbs, unit="GB/s", floor_us=hbm_floor_us)
    out = {"kernel": kernel, "hbm": hbm, "alu": alu}
    if alu and alu["floor_us"] > hbm_floor_us:
        out.update(bound="alu", achieved=alu["achieved_tflops"], peak=alu["peak_tflops"], unit="TFLOP/s",
                   frac=alu["frac"], traffic=rest.get("traffic"), peak_kind=alu["peak_kind"])
    else:
        out.update(bound="hbm", achieved=achieved_gbs, peak=peak_gbs, unit="GB/s", frac=rest.get("frac"),
                   traffic=rest.get("traffic"), peak_kind=rest.get("peak_kind"))
    return out


def alu_side(wl, B, ncv, k1_us, clocks, general, sms):
    """The FP32 side of the dominant kernel's roofline (the bound is the larger of the two floors):
    algorithmic flops per pixel and coil = the data term's transforms at 5 log2(n) per point each
    (line masks: two length-ny transforms; other masks: two 2D transforms of nx ny points), the
    sensitivity product (6), the mask (2) and the conjugate product accumulated (8); peak =
    SMs (queried) x 128 lanes x 2 flops x the median SM clock sampled during the timed region."""
    if not k1_us:
        return None
    tlen = wl.nx * wl.ny if general else wl.ny
    flops = B * wl.nx * wl.ny * ncv * (2 * 5 * math.log2(tlen) + 6 + 2 + 8)
    ghz = ((clocks or {}).get("sm_mhz") or 2070.0) / 1e3
    peak = sms * FP32_LANES_PER_SM * 2 * ghz / 1e3  # TFLOP/s
    achieved = flops / (k1_us / 1e6) / 1e12
    return {"flops_per_launch": flops, "achieved_tflops": achieved, "peak_tflops": peak, "frac": achieved / peak,
            "floor_us": flops / (peak * 1e12) * 1e6,
            "peak_kind": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x median sampled SM clock"}


def tensor_core_rate(args, wl, B, ncv, k1_us):
    """Split-precision modes: the MMA work of one q = A p over the batch per launch time.  Per coil
    and 8-column tile: ny = 256, four radix-16 stages of 2 K-steps x 3 split products of
    128 x 32 x 16; ny = 512, two radix-16 stages of two 128-row groups x 2 K-steps x 3 products of
    128 x 32 x 16 and two radix-32 stages of 4 K-steps x 3 products of 128 x 64 x 16."""
    if args.prec == "fp32" or not k1_us:
        return None
    mma = lambda m, n: 2 * m * n * 16  # noqa: E731
    if wl.ny == 512:
        per_tile = 2 * (2 * 2 * 3 * mma(128, 32)) + 2 * (4 * 3 * mma(128, 64))
    else:
        per_tile = 4 * (2 * 3 * mma(128, 32))
    flops = B * ncv * (wl.nx // 8) * per_tile
    return {"mma_tflops_per_launch": flops / 1e12, "achieved_tflops": flops / (k1_us / 1e6) / 1e12,
            "note": "kind::f16 tcgen05.mma; the kernel is bound by the stage round trips "
                    "(TMEM -> registers -> shared memory), not by the tensor pipe"}


def per_slice_loop(torch, sb, dev, groups, members, sens, masks, ys, wls, batched_recon_per_s):
    """The uneven batch reconstructed one slice at a time with the same library (one 1-slice plan
    per geometry, coils and mask set per slice as in the batched step), timed once after a warm-up
    slice per geometry: the per-slice loop that batching is compared against."""
    stream = torch.cuda.current_stream(dev)
    loop = []
    for (nx, ny, nc), ids in sorted(groups.items()):
        w = wls[ids[0]]
        loop.append(sb.Plan(nx, ny, nc, 1, w.mu, w.lam, w.gam, w.wavelet_levels, stream=stream))
    w0 = wls[0]
    xs1 = [torch.zeros((1, p.shape[1], p.shape[2]), dtype=torch.complex64, device=dev) for p in loop]

    def one(k, i):
        p = loop[k]
        p.set_coils(sens[k][i:i + 1])
        p.set_mask(masks[k][i:i + 1])
        xs1[k].zero_()
        st, iters, _ = p.split_bregman(ys[k][i:i + 1], xs1[k], w0.n_outer, w0.n_inner, tol=w0.pcg_tol,
                                       maxit=w0.pcg_maxit)
        if st != sb.SB_OK:
            raise RuntimeError(f"split_bregman: {sb.status_string(st)}")
        return int(sum(sum(r) for r in iters))

    for k in range(len(loop)):
        one(k, 0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n = iters = 0
    for k, (ids, _) in enumerate(members):
        for i in range(len(ids)):
            iters += one(k, i)
            n += 1
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    for p in loop:
        p.close()
    return {"recon_per_s": n / t, "pcg_iters_per_s": iters / t, "slices": n,
            "batched_over_loop": batched_recon_per_s / (n / t),
            "how": "one slice at a time through sb_split_bregman (1-slice plan per geometry), CUDA events"}


def run_uneven(args, torch, sb, synth, world, rank, local, dist):
    """64 slices of mixed size, coil count and R: one plan per geometry, each on its own stream,
    reconstructed concurrently by sb_split_bregman_many.  A step = k construction of every plan
    (sb_set_mask) + the concurrent reconstructions."""
    import collections
    import numpy as np
    wls = synth.uneven_workloads(seed=rank_seed(synth.UNEVEN_SEED, rank))
    groups = collections.defaultdict(list)
    for i, w in enumerate(wls):
        groups[(w.nx, w.ny, w.ncoils)].append(i)
    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    plans, ys, xs, sens, masks, members = [], [], [], [], [], []
    tuned_all = {}
    for (nx, ny, nc), ids in sorted(groups.items()):
        sl = [synth.uneven_slice(wls, i) for i in ids]
        w = wls[ids[0]]
        sens.append(torch.from_numpy(np.stack([s.sens for s in sl]).astype(np.complex64)).to(dev))
        masks.append(torch.from_numpy(np.stack([s.mask for s in sl])).to(dev))
        ys.append(torch.from_numpy(np.stack([s.y for s in sl]).astype(np.complex64)).to(dev))
        xs.append(torch.zeros((len(ids), ny, nx), dtype=torch.complex64, device=dev))
        pstream = torch.cuda.Stream(dev)
        g, tuning = 0, None
        if args.autotune:
            from paper_1710_01758_gb300 import autotune

            def make(gg, nx=nx, ny=ny, nc=nc, ids=ids, w=w, k=len(sens) - 1):
                p = sb.Plan(nx, ny, nc, len(ids), w.mu, w.lam, w.gam, w.wavelet_levels, stream=pstream, groups=gg)
                p.set_coils(sens[k])
                p.set_mask(masks[k])
                return p

            torch.cuda.synchronize()
            tuning = autotune.tune(make, nx, ny, nc, len(ids))
            g = tuning["groups"]
            tuned_all[f"{nx}x{ny}x{nc}"] = {k: tuning[k] for k in ("groups", "col_tile", "poll_every")}
        plan = sb.Plan(nx, ny, nc, len(ids), w.mu, w.lam, w.gam, w.wavelet_levels, stream=pstream, groups=g)
        if tuning:
            plan.set_tuning(col_tile=tuning["col_tile"], poll_every=tuning["poll_every"])
        plans.append(plan)
        members.append((ids, sl))
    torch.cuda.synchronize()
    log(f"[bench] rank {rank}: generated {len(wls)} uneven slices ({len(plans)} geometries) in "
        f"{time.perf_counter() - t0:.1f}s")
    w0 = wls[0]

    def step():
        for p, s_, m_ in zip(plans, sens, masks):
            p.set_coils(s_)
            p.set_mask(m_)
        st, iters, _ = sb.split_bregman_many(plans, ys, xs, w0.n_outer, w0.n_inner, tol=w0.pcg_tol,
                                             maxit=w0.pcg_maxit)
        if st != sb.SB_OK:
            raise RuntimeError(f"split_bregman_many: {sb.status_string(st)}")
        return int(sum(sum(sum(r) for r in it) for it in iters))

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = sb.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev0.record(torch.cuda.current_stream(dev))
    torch.cuda.synchronize()
    total = 0
    for _ in range(args.steps):
        total += step()
    ends = []
    for p in plans:
        e = torch.cuda.Event(enable_timing=True)
        e.record(p.stream)
        ends.append(e)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = sb.kernel_launches() - launches0
    elapsed = max(ev0.elapsed_time(e) for e in ends) / 1e3
    total_all, elapsed_max = total, elapsed
    if dist:
        elapsed_max, total_all = reduce_over_ranks(dist, dev, elapsed, total)
    extra = {}
    if rank == 0 and not args.no_loop:
        extra["per_slice_loop"] = per_slice_loop(torch, sb, dev, groups, members, sens, masks, ys, wls,
                                                 batched_recon_per_s=args.steps * len(wls) / elapsed)
    if rank == 0 and not args.no_cpu_baseline:
        ids, sl = members[0]
        x_or, it_or, t_or = oracle_recon(wls[ids[0]], sl[0])
        extra["err_vs_fp64"] = float(np.linalg.norm(xs[0][0].cpu().numpy() - x_or) / np.linalg.norm(x_or))
        extra["err_slice"] = wls[ids[0]].name
        extra["cpu_baseline"] = {"value": it_or / t_or, "unit": UNIT, "cores": host_threads(), "kind": "oracle",
                                 "sample": f"one {wls[ids[0]].name} slice, full Split Bregman, FP64 numpy"}
    for p in plans:
        p.close()
    if rank == 0:
        sizes = collections.Counter(f"{w.nx}x{w.ny}" for w in wls)
        line = {"metric": METRIC, "value": total_all / elapsed_max, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp32",
                "scalars": "fp64", "data": "synthetic",
                "config": {"workload": f"{len(wls)} uneven slices ({len(plans)} geometries)",
                           "sizes": dict(sizes), "coils": sorted({w.ncoils for w in wls}),
                           "accel": sorted({w.accel for w in wls}), "haar_levels": w0.wavelet_levels,
                           "n_outer": w0.n_outer, "pcg_tol": w0.pcg_tol, "precond": "circulant",
                           "l2": "inputs larger than L2", "parallelism": f"{world} ranks x independent batches",
                           "autotune": tuned_all or None},
                "recon_per_s": args.steps * len(wls) * world / elapsed_max,
                "pcg_iters_per_step": total_all / args.steps, "roofline": None,
                "gpu_launches": int(launches), "clocks": clocks, "e2e": None}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_volume(args, torch, sb, synth, world, rank, local, dist):
    """One 256x256x128 volume, 16 coils, (ky, kz) lines at R = 8 with a 24 x 24 centre, 3D TV +
    3-level 3D Haar, 15 Split Bregman iterations with PCG to 1e-3.  A step = k construction +
    reconstruction."""
    import numpy as np
    v = synth.VOLUME_256
    t0 = time.perf_counter()
    s = synth.make_volume(v, rank_seed(v.seed, rank))
    log(f"[bench] rank {rank}: generated the volume in {time.perf_counter() - t0:.1f}s")
    dev = torch.device("cuda", local)
    sens_h = np.ascontiguousarray(s.sens[None].astype(np.complex64))
    mask_h = np.ascontiguousarray(s.mask[None])
    y_h = np.ascontiguousarray(s.y[None].astype(np.complex64))
    d_sens = torch.from_numpy(sens_h).to(dev)
    d_mask = torch.from_numpy(mask_h).to(dev)
    d_y = torch.from_numpy(y_h).to(dev)
    x = torch.zeros((1, v.nz, v.ny, v.nx), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)
    plan = sb.Plan(v.nx, v.ny, v.ncoils, 1, v.mu, v.lam, v.gam, v.wavelet_levels, stream=stream, nz=v.nz)

    def step(ss=d_sens, ms=d_mask, ys=d_y):
        plan.set_coils(ss)
        plan.set_mask(ms)
        st, iters, _ = plan.split_bregman(ys, x, v.n_outer, v.n_inner, tol=v.pcg_tol, maxit=v.pcg_maxit)
        if st != sb.SB_OK:
            raise RuntimeError(f"split_bregman: {sb.status_string(st)}")
        return int(sum(sum(i) for i in iters))

    for _ in range(args.warmup):
        step()
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = sb.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    total = 0
    for _ in range(args.steps):
        total += step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = sb.kernel_launches() - launches0
    elapsed = ev0.elapsed_time(ev1) / 1e3
    total_all, elapsed_max = total, elapsed
    if dist:
        elapsed_max, total_all = reduce_over_ranks(dist, dev, elapsed, total)

    # where a step's time goes: one extra untimed step with the event timer on every class (the
    # volume is one slice group on one stream, so the class times add up to the step)
    plan.set_timing((1 << sb.SB_KCLASS_COUNT) - 1)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    it_split = step()
    s1.record(stream)
    torch.cuda.synchronize()
    step_ms = s0.elapsed_time(s1)
    timing = {sb.KCLASS_NAMES[c]: plan.timing(c) for c in range(sb.SB_KCLASS_COUNT)}
    plan.set_timing(0)
    kern_ms = sum(t[1] for t in timing.values())
    split = {"step_ms": round(step_ms, 3), "pcg_iterations": it_split,
             "classes": {k: {"launches": t[0], "ms": round(t[1], 3), "share_of_step": round(t[1] / step_ms, 4)}
                         for k, t in timing.items() if t[0]},
             "host_polls_and_gaps_ms": round(step_ms - kern_ms, 3),
             "how": "one extra untimed step, CUDA events around every launch; the shares add up to that step"}

    # q = A p timed alone (three launches: y DFT per coil into the coil scratch, z DFT + mask +
    # inverse, inverse y DFT + coil combine + TV).  Algorithmic bytes per application: p and S
    # read, q written, (16 + 8 Nc) N; the three passes move (48 Nc + 24) N
    n = v.nx * v.ny * v.nz
    peak, peak_kind = peaks()
    plan.set_timing(1 << sb.SB_KCLASS_APPLY_A)
    qbuf = torch.empty_like(x)
    n_apply = 5
    for _ in range(n_apply):
        plan.apply_A(x, qbuf)
    a_n, a_ms = plan.timing(sb.SB_KCLASS_APPLY_A)
    plan.set_timing(0)
    a_us = 1e3 * a_ms / n_apply
    alg = (16 + 8 * v.ncoils) * n
    impl = (48 * v.ncoils + 24) * n
    achieved = alg / (a_us / 1e6) / 1e9
    roofline = {"bound": "hbm", "kernel": "q = A p: k_g3_fwd_y + k_g3_z + k_g3_inv_y", "achieved": achieved,
                "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
                "algorithmic_bytes_per_launch": alg, "bytes_rule": "(16 + 8 Nc) N: p and S read, q written",
                "implementation_bytes_per_launch": impl, "implementation_over_algorithmic": impl / alg,
                "mean_launch_us": a_us,
                "timing": f"timed alone: {n_apply} applications ({a_n} launches), CUDA events on the plan stream"}

    extra = {}
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle as it stands on the same volume, bounded sample: the operator work of one PCG
        # iteration (one application of A and one of M^{-1}, FP64 numpy on one host core)
        from oracle import operators, precond
        k = precond.clamp_k(precond.k_diag(s.sens, s.mask, v.mu, v.lam, v.gam, 3))
        p0 = x[0].cpu().numpy().astype(np.complex128)
        t0 = time.perf_counter()
        operators.apply_A(p0, s.sens, s.mask, v.mu, v.lam, v.gam, 3)
        precond.apply_precond(p0, k, 3)
        t_it = time.perf_counter() - t0
        extra["cpu_baseline"] = {"value": 1.0 / t_it, "unit": UNIT, "cores": host_threads(), "kind": "oracle",
                                 "sample": "the operator work of one PCG iteration on the full volume (one "
                                           "application of A and one of M^{-1}), FP64 numpy"}

    e2e = None
    if not args.no_e2e:
        # end to end with host buffers: every step uploads the coil maps, the mask and the k-space
        # data from pinned memory and reads the image back, all inside the timed region
        hs = torch.from_numpy(sens_h).pin_memory()
        hm = torch.from_numpy(mask_h).pin_memory()
        hy = torch.from_numpy(y_h).pin_memory()
        hx = torch.empty(tuple(x.shape), dtype=torch.complex64).pin_memory()
        es, em, ey = torch.empty_like(d_sens), torch.empty_like(d_mask), torch.empty_like(d_y)
        h2d = hs.numel() * 8 + hm.numel() + hy.numel() * 8
        d2h = hx.numel() * 8
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e_it = 0
        for _ in range(args.steps):
            es.copy_(hs, non_blocking=True)
            em.copy_(hm, non_blocking=True)
            ey.copy_(hy, non_blocking=True)
            e_it += step(es, em, ey)
            hx.copy_(x, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e_el = e0.elapsed_time(e1) / 1e3
        if dist:
            e_el, e_it = reduce_over_ranks(dist, dev, e_el, e_it)
        e2e = {"value": e_it / e_el, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    plan.close()
    if rank == 0:
        line = {"metric": METRIC, "value": total_all / elapsed_max, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp32",
                "scalars": "fp64", "data": "synthetic",
                "config": {"workload": f"1 x [{v.name}]", "nx": v.nx, "ny": v.ny, "nz": v.nz, "ncoils": v.ncoils,
                           "accel": v.accel, "centre": v.centre, "haar_levels": v.wavelet_levels,
                           "n_outer": v.n_outer, "pcg_tol": v.pcg_tol, "precond": "circulant",
                           "l2": "inputs larger than L2 (1.1 GB of coil maps)",
                           "parallelism": f"{world} ranks x independent volumes"},
                "recon_per_s": args.steps * world / elapsed_max,
                "pcg_iters_per_step": total_all / args.steps, "roofline": roofline,
                "step_split": split, "gpu_launches": int(launches), "clocks": clocks, "e2e": e2e}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
