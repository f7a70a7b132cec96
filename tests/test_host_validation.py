"""Host-side argument checking of the C ABI, on the CPU: descriptors and arguments that the
library must refuse before any device work, with the status code the header documents."""
import ctypes

import pytest

from paper_1710_01758_gb300 import sb


def create(**kw):
    base = dict(nx=64, ny=64, ncoils=2, nbatch=1, mu=1.0, lam=0.1, gam=0.1, wavelet_levels=2)
    extra = {k: kw.pop(k) for k in list(kw) if k in ("groups", "precond_passes", "nz", "wavelet", "prec")}
    base.update(kw)
    d = sb.plan_desc(base["nx"], base["ny"], base["ncoils"], base["nbatch"], base["mu"], base["lam"], base["gam"],
                     base["wavelet_levels"], **extra)
    for k in ("ndim",):
        if k in kw:
            setattr(d, k, kw[k])
    out = ctypes.c_void_p()
    return sb._lib.sb_plan_create(ctypes.byref(d), None, ctypes.byref(out)), out


@pytest.mark.parametrize("kw,status", [
    (dict(ncoils=0), sb.SB_ERR_INVALID_ARG),
    (dict(nbatch=0), sb.SB_ERR_INVALID_ARG),
    (dict(mu=0.0), sb.SB_ERR_INVALID_ARG),
    (dict(lam=-1.0), sb.SB_ERR_INVALID_ARG),
    (dict(gam=float("nan")), sb.SB_ERR_INVALID_ARG),
    (dict(wavelet_levels=-1), sb.SB_ERR_INVALID_ARG),
    (dict(groups=-2), sb.SB_ERR_INVALID_ARG),
    (dict(precond_passes=2), sb.SB_ERR_INVALID_ARG),
    (dict(wavelet=3), sb.SB_ERR_INVALID_ARG),
    (dict(ndim=4), sb.SB_ERR_INVALID_ARG),
    (dict(nx=48), sb.SB_ERR_UNSUPPORTED),            # not a supported transform length
    (dict(ny=1024), sb.SB_ERR_UNSUPPORTED),
    (dict(wavelet_levels=6), sb.SB_ERR_UNSUPPORTED),  # Haar blocks larger than the 32 x 32 tiles
    (dict(prec=sb.SB_PREC_SPLIT_BF16), sb.SB_ERR_UNSUPPORTED),  # tensor-core stages: ny 256 or 512 only
    (dict(ny=128, prec=sb.SB_PREC_SPLIT_FP16), sb.SB_ERR_UNSUPPORTED),
    (dict(nx=36, ny=256, prec=sb.SB_PREC_SPLIT_FP16), sb.SB_ERR_UNSUPPORTED),  # nx not a transform length
    (dict(ny=256, nz=32, prec=sb.SB_PREC_SPLIT_FP16), sb.SB_ERR_UNSUPPORTED),  # volumes stay FP32
    (dict(prec=7), sb.SB_ERR_INVALID_ARG),
    (dict(nz=16), sb.SB_ERR_UNSUPPORTED),            # volume depth below the shortest transform
    (dict(nz=32, wavelet_levels=5), sb.SB_ERR_UNSUPPORTED),
    (dict(nz=32, wavelet=1), sb.SB_ERR_UNSUPPORTED),  # Daubechies-4 is 2D only
    (dict(nx=32, ny=32, wavelet_levels=5, wavelet=1), sb.SB_ERR_UNSUPPORTED),  # coarsest band < 4
])
def test_plan_descriptor_refused(kw, status):
    st, out = create(**kw)
    assert st == status, (kw, sb.status_string(st))
    assert not out.value


def test_status_strings():
    for code, name in [(sb.SB_OK, "SB_OK"), (sb.SB_ERR_UNSUPPORTED, "SB_ERR_UNSUPPORTED"),
                       (sb.SB_ERR_TIMEOUT, "SB_ERR_TIMEOUT"), (99, "SB_ERR_UNKNOWN")]:
        assert sb.status_string(code) == name


def test_null_arguments_refused():
    assert sb._lib.sb_plan_create(None, None, None) == sb.SB_ERR_INVALID_ARG
    assert sb._lib.sb_plan_destroy(None) == sb.SB_OK
    for fn in ("sb_set_coils", "sb_set_mask", "sb_get_k"):
        assert getattr(sb._lib, fn)(None, None) == sb.SB_ERR_INVALID_ARG
    assert sb._lib.sb_apply_A(None, None, None) != sb.SB_OK
    t = sb.sb_tuning(16, 4)
    assert sb._lib.sb_set_tuning(None, ctypes.byref(t)) == sb.SB_ERR_INVALID_ARG
    assert sb._lib.sb_get_tuning(None, ctypes.byref(t)) == sb.SB_ERR_INVALID_ARG
    assert sb._lib.sb_set_graphs(None, 1) == sb.SB_ERR_INVALID_ARG
    assert sb._lib.sb_split_bregman_many(None, 0, None, None, None, None) == sb.SB_ERR_INVALID_ARG
    # coil compression: nv > nc and more than 32 coils are refused before any device work
    p = ctypes.c_void_p(16)
    assert sb._lib.sb_coil_compress(p, p, 64, 4, 1, 5, ctypes.c_void_p(32), ctypes.c_void_p(48), None, None,
                                    None) == sb.SB_ERR_INVALID_ARG
    assert sb._lib.sb_coil_compress(p, p, 64, 33, 1, 4, ctypes.c_void_p(32), ctypes.c_void_p(48), None, None,
                                    None) == sb.SB_ERR_INVALID_ARG
    assert sb._lib.sb_apply_precond_noalloc(None, None, None, 64, 64, 1, None) == sb.SB_ERR_INVALID_ARG
    # the allocation-free preconditioner: lengths outside {32, 64, 128, 256} are unsupported,
    # sizes beyond its fixed scratch and empty batches are invalid; all refused before device work
    q = ctypes.c_void_p(64)
    assert sb._lib.sb_apply_precond_noalloc(p, q, p, 48, 64, 1, None) == sb.SB_ERR_UNSUPPORTED
    assert sb._lib.sb_apply_precond_noalloc(p, q, p, 64, 512, 1, None) == sb.SB_ERR_UNSUPPORTED
    assert sb._lib.sb_apply_precond_noalloc(p, q, p, 256, 256, 17, None) == sb.SB_ERR_INVALID_ARG
    assert sb._lib.sb_apply_precond_noalloc(p, q, p, 256, 256, 0, None) == sb.SB_ERR_INVALID_ARG
    # the wait check needs a plan
    assert sb._lib.sb_set_wait_check(None, 1024, 1) == sb.SB_ERR_INVALID_ARG
