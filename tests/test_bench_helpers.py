"""Host-side helpers of bench.py on CPU: the tensor-core work per launch for both stage shapes
(counted by hand from the stage structure), the precision labels, and the workload config that
the reference arm and our arm share."""
import os
import types

import bench
from paper_1710_01758_gb300 import synth


def _args(prec):
    return types.SimpleNamespace(prec=prec)


def test_tensor_core_work_per_launch():
    mma = lambda m, n: 2 * m * n * 16  # flops of one M x N x 16 product  # noqa: E731
    wl = synth.METRIC_256  # 256 rows: four radix-16 stages x 2 K-steps x 3 split products
    r = bench.tensor_core_rate(_args("split-fp16"), wl, 64, 12, 100.0)
    per_tile = 4 * 2 * 3 * mma(128, 32)
    assert r["mma_tflops_per_launch"] == 64 * 12 * (256 // 8) * per_tile / 1e12
    assert abs(r["achieved_tflops"] - r["mma_tflops_per_launch"] / 100e-6) < 1e-9
    wl5 = synth.LARGE_512  # 512 rows: two radix-16 stages of two M groups, two radix-32 of 4 K-steps
    r5 = bench.tensor_core_rate(_args("split-bf16"), wl5, 8, 32, 50.0)
    per_tile5 = 2 * (2 * 2 * 3 * mma(128, 32)) + 2 * (4 * 3 * mma(128, 64))
    assert r5["mma_tflops_per_launch"] == 8 * 32 * (512 // 8) * per_tile5 / 1e12
    assert bench.tensor_core_rate(_args("fp32"), wl, 64, 12, 100.0) is None


def test_precision_labels_and_workload_config():
    assert bench.PRECS["fp32"][0] == 0 and bench.PRECS["split-bf16"][0] == 1 and bench.PRECS["split-fp16"][0] == 2
    wl = synth.METRIC_256
    cfg = bench.workload_config(wl, 64, {"sample": "s"})
    assert cfg["workload"] == f"64 x [{wl.name}]" and cfg["batch_slices"] == 64 and cfg["sample"] == "s"
    assert (cfg["nx"], cfg["ny"], cfg["ncoils"]) == (256, 256, 12)
    # the reference arm reports the same workload string as our arm's default
    assert bench.WORKLOADS["256"] == ("METRIC_256", 64)


def test_alu_side_of_the_roofline():
    """Two length-256 transforms at 5 log2(256) flops per point, plus 16 flops of products and
    mask: 96 per pixel and coil; the peak is 152 x 128 x 2 flops per clock."""
    wl = synth.METRIC_256
    r = bench.alu_side(wl, 64, 12, 168.0, {"sm_mhz": 2070.0}, general=False, sms=152)
    assert r["flops_per_launch"] == 64 * 256 * 256 * 12 * 96
    assert abs(r["peak_tflops"] - 152 * 128 * 2 * 2.07 / 1e3) < 1e-9
    assert abs(r["achieved_tflops"] - r["flops_per_launch"] / 168e-6 / 1e12) < 1e-9
    assert r["floor_us"] < 168.0
    g = bench.alu_side(wl, 64, 12, 168.0, None, general=True, sms=152)
    assert g["flops_per_launch"] == 64 * 256 * 256 * 12 * (2 * 5 * 16 + 16)


def test_roofline_takes_the_binding_floor():
    alu = {"floor_us": 110.0, "achieved_tflops": 20.0, "peak_tflops": 80.0, "frac": 0.25, "peak_kind": "derived"}
    r = bench.roofline_line("k", 700.0, 6700.0, alu, 70.0, {"frac": 700 / 6700, "traffic": None, "peak_kind": "m"})
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["frac"] == 0.25 and r["hbm"]["floor_us"] == 70.0
    r = bench.roofline_line("k", 3000.0, 6700.0, dict(alu, floor_us=60.0), 70.0, {"frac": 3000 / 6700})
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and abs(r["frac"] - 3000 / 6700) < 1e-12


def test_workload_names_resolve():
    """Every --workload name maps to a synth workload; the active-shrink and parameter-set lines
    keep the headline geometry and set explicit thresholds."""
    for name in bench.WORKLOADS:
        assert bench.workload_of(synth, name).nx > 0
    for name in ("shrink256", "set1", "set2", "set3"):
        wl = bench.workload_of(synth, name)
        assert (wl.nx, wl.ny, wl.ncoils, wl.tau) == (256, 256, 12, 0.02)
    assert (bench.workload_of(synth, "set2").mu, bench.workload_of(synth, "set2").lam) == (1e-2, 4e-3)
    assert synth.VOLUME_256.wavelet_levels == 3 and synth.VOLUME_256.n_outer == 15


def test_clock_sampler_keeps_only_rows_of_the_timed_region(tmp_path, monkeypatch):
    """bench.ClockSampler waits for nvidia-smi's first row before the timed region and keeps only
    the rows written after that: a fake nvidia-smi writes five idle rows at once, then, while the
    region runs, three rows at full clock with the power-cap reason active."""
    import time
    fake = tmp_path / "nvidia-smi"
    idle = "0, 1000, 2070, 100.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    busy = "0, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active"
    fake.write_text("#!/bin/bash\n" + "".join(f"echo '{idle}'\n" for _ in range(5)) + "sleep 0.5\n" +
                    "".join(f"echo '{busy}'\nsleep 0.05\n" for _ in range(3)) + "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    s = bench.ClockSampler(0)
    s.start()
    assert s.proc is not None and s.skip == 5
    time.sleep(1.2)
    c = s.stop()
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
