"""The allocation-free preconditioner entry point (sb_apply_precond_noalloc) against the plan
path (sb_apply_precond), called through the C ABI twice in a row.

sb_apply_precond_noalloc serves callers that cannot allocate device memory when they apply the
preconditioner; its intermediate lives in a fixed device array shared by all calls.  Two
consecutive calls check that the array's leftover contents from the first call do not leak
into the second.  This file is named to be collected last.
"""
import numpy as np
import pytest

from paper_1710_01758_gb300 import synth

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5


def test_noalloc_matches_plan_path_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_01758_gb300 import sb

    nx, ny, nc, nb = 128, 256, 6, 3
    rng = np.random.default_rng(2024)
    sens = np.stack([synth.coil_maps(ny, nx, nc, rng) for _ in range(nb)])
    mask = np.stack([synth.line_mask(ny, nx, 4.0, 8, rng) for _ in range(nb)])
    plan = sb.Plan(nx, ny, nc, nb, 1.0, 0.05, 0.05, 0)
    d_sens = torch.from_numpy(sens).to(torch.complex64).cuda()
    plan.set_coils(d_sens)
    plan.set_mask(torch.from_numpy(mask).cuda())
    k = plan.k()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        r = torch.from_numpy(synth.random_complex((nb, ny, nx), rng)).to(torch.complex64).cuda()
        ref = plan.apply_precond(r)
        z = torch.empty_like(r)
        sb.sb_apply_precond_noalloc(r.data_ptr(), k.data_ptr(), z.data_ptr(), nx, ny, nb, stream)
        torch.cuda.synchronize()
        err = (torch.linalg.vector_norm(z - ref) / torch.linalg.vector_norm(ref)).item()
        assert err <= OP_TOL, (call, err)
    # sizes beyond the fixed scratch are refused, not truncated
    big = 17 * 256 * 256
    with pytest.raises(sb.SbError) as ei:
        sb.sb_apply_precond_noalloc(r.data_ptr(), k.data_ptr(), z.data_ptr(), 256, 256, 17, stream)
    assert ei.value.status == sb.SB_ERR_INVALID_ARG and big > (1 << 20)
    plan.close()
