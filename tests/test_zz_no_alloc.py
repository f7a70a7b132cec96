"""The allocation-free preconditioner entry point (sb_apply_precond_noalloc) against the FP64
oracle's M^{-1} r = F^H diag(k)^{-1} F r (Eq. precon), called through the C ABI.

sb_apply_precond_noalloc serves callers that cannot allocate device memory when they apply the
preconditioner (a reconstruction pipeline with a memory budget frozen after start-up, a plugin
that is handed only pre-allocated buffers); its intermediate lives in one fixed device array
that every call shares.  The checks:
  * every supported (nx, ny) pair, two calls in a row per pair, so the array's leftover contents
    from one call cannot leak into the next one;
  * one call at the largest batch the array holds (2^20 complex elements), and one in place
    (d_r == d_z);
  * the very first call of a fresh process made on a non-blocking stream (the set-up's twiddle
    copy must be complete before that stream's kernels read it);
  * sizes beyond the array refused, not truncated.
k is a seeded positive field given to both sides as the same float32 values.  This file is named
to be collected last.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import precond
from paper_1710_01758_gb300 import synth

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5          # one operator application, relative L2 (as for sb_apply_precond)
SIZES = (32, 64, 128, 256)
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _inputs(nb, ny, nx, rng):
    r = synth.random_complex((nb, ny, nx), rng).astype(np.complex64)
    k = rng.uniform(0.05, 1.5, (nb, ny, nx)).astype(np.float32)
    return r, k


def _oracle(r, k):
    return precond.apply_precond(r.astype(np.complex128), k.astype(np.float64), 2)


def _run(torch, sb, r, k, in_place=False, stream=None):
    nb, ny, nx = r.shape
    d_r = torch.from_numpy(r).cuda()
    d_k = torch.from_numpy(k).cuda()
    d_z = d_r if in_place else torch.empty_like(d_r)
    s = stream if stream is not None else torch.cuda.current_stream()
    with torch.cuda.stream(s):
        sb.sb_apply_precond_noalloc(d_r.data_ptr(), d_k.data_ptr(), d_z.data_ptr(), nx, ny, nb, s.cuda_stream)
    s.synchronize()
    return d_z.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("ny", SIZES)
@pytest.mark.parametrize("nx", SIZES)
def test_noalloc_matches_oracle_every_size_two_calls(nx, ny):
    torch = _torch()
    from paper_1710_01758_gb300 import sb

    rng = np.random.default_rng(1000 + 7 * nx + ny)
    for call, nb in enumerate((3, 2)):
        r, k = _inputs(nb, ny, nx, rng)
        err = _rel(_run(torch, sb, r, k), _oracle(r, k))
        assert err <= OP_TOL, (nx, ny, call, err)


def test_noalloc_maximum_batch_and_in_place():
    torch = _torch()
    from paper_1710_01758_gb300 import sb

    rng = np.random.default_rng(77)
    r, k = _inputs(16, 256, 256, rng)                # 16 * 256 * 256 = 2^20 elements: the limit
    assert r.size == 1 << 20
    want = _oracle(r, k)
    err = _rel(_run(torch, sb, r, k), want)
    assert err <= OP_TOL, err
    err_ip = _rel(_run(torch, sb, r, k, in_place=True), want)
    assert err_ip <= OP_TOL, err_ip
    # one element more than the scratch holds is refused
    d = torch.zeros(8, dtype=torch.complex64, device="cuda")
    with pytest.raises(sb.SbError) as ei:
        sb.sb_apply_precond_noalloc(d.data_ptr(), d.data_ptr(), d.data_ptr(), 256, 256, 17, 0)
    assert ei.value.status == sb.SB_ERR_INVALID_ARG


_FRESH = r"""
import numpy as np, torch
from oracle import precond
from paper_1710_01758_gb300 import sb, synth
rng = np.random.default_rng(5)
r = synth.random_complex((4, 128, 256), rng).astype(np.complex64)
k = rng.uniform(0.05, 1.5, r.shape).astype(np.float32)
s = torch.cuda.Stream()          # non-blocking with respect to the legacy stream
with torch.cuda.stream(s):
    d_r = torch.from_numpy(r).to('cuda', non_blocking=False)
    d_k = torch.from_numpy(k).to('cuda', non_blocking=False)
    d_z = torch.empty_like(d_r)
s.synchronize()
sb.sb_apply_precond_noalloc(d_r.data_ptr(), d_k.data_ptr(), d_z.data_ptr(), 256, 128, 4, s.cuda_stream)
s.synchronize()
want = precond.apply_precond(r.astype(np.complex128), k.astype(np.float64), 2)
err = float(np.linalg.norm(d_z.cpu().numpy() - want) / np.linalg.norm(want))
print("ERR", err)
"""


def test_noalloc_first_call_in_fresh_process_on_side_stream():
    _torch()
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    res = subprocess.run([sys.executable, "-c", _FRESH], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    err = float([ln for ln in res.stdout.splitlines() if ln.startswith("ERR")][-1].split()[1])
    assert err <= OP_TOL, err
