"""Python binding of the C ABI in ``include/sb.h`` (ctypes; argument marshalling only).

Every function here forwards to ``lib/libsbpcg.so`` with the same name.  Device arrays are
passed as raw device pointers (``torch.Tensor.data_ptr()`` of contiguous complex64 / uint8 /
float32 CUDA tensors); nothing is computed in Python.  If the library has not been built the
import of this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libsbpcg.so")

# sb_status
SB_OK = 0
SB_ERR_INVALID_ARG = 1
SB_ERR_UNSUPPORTED = 2
SB_ERR_CUDA = 3
SB_ERR_NOT_READY = 4
SB_ERR_NONFINITE = 5
SB_ERR_BREAKDOWN = 6
SB_ERR_NOT_CONVERGED = 7
SB_ERR_TIMEOUT = 8
# sb_precision
SB_PREC_FP32 = 0
SB_PREC_SPLIT_BF16 = 1
SB_PREC_SPLIT_FP16 = 2
# sb_precond
SB_PRECOND_NONE = 0
SB_PRECOND_CIRCULANT = 1
SB_PRECOND_JACOBI = 2
# wavelet kinds (sb_plan_desc.wavelet)
SB_WAVELET_HAAR = 0
SB_WAVELET_DAUB4 = 1


class sb_plan_desc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("ncoils", ctypes.c_int), ("nbatch", ctypes.c_int), ("mu", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("gamma", ctypes.c_double), ("wavelet_levels", ctypes.c_int),
                ("prec", ctypes.c_int), ("groups", ctypes.c_int), ("precond_passes", ctypes.c_int),
                ("wavelet", ctypes.c_int)]


class sb_tuning(ctypes.Structure):
    _fields_ = [("col_tile", ctypes.c_int), ("poll_every", ctypes.c_int), ("apply_tile", ctypes.c_int),
                ("general_passes", ctypes.c_int)]


class sb_pcg_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("fixed_iters", ctypes.c_int),
                ("precond", ctypes.c_int)]


class sb_pcg_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_resid", ctypes.c_double), ("converged", ctypes.c_int)]


class sb_sb_opts(ctypes.Structure):
    _fields_ = [("n_outer", ctypes.c_int), ("n_inner", ctypes.c_int), ("pcg", sb_pcg_opts),
                ("tau_tv", ctypes.c_double), ("tau_w", ctypes.c_double), ("init_rss", ctypes.c_int),
                ("h_iters", ctypes.POINTER(ctypes.c_int))]


# (name, restype, argtypes) of every exported entry point
_P = ctypes.c_void_p
SIGNATURES = [
    ("sb_plan_create", ctypes.c_int, [ctypes.POINTER(sb_plan_desc), _P, ctypes.POINTER(_P)]),
    ("sb_plan_destroy", ctypes.c_int, [_P]),
    ("sb_set_coils", ctypes.c_int, [_P, _P]),
    ("sb_set_mask", ctypes.c_int, [_P, _P]),
    ("sb_get_k", ctypes.c_int, [_P, _P]),
    ("sb_apply_A", ctypes.c_int, [_P, _P, _P]),
    ("sb_apply_precond", ctypes.c_int, [_P, _P, _P]),
    ("sb_pcg_solve", ctypes.c_int, [_P, _P, _P, ctypes.POINTER(sb_pcg_opts), ctypes.POINTER(sb_pcg_result)]),
    ("sb_split_bregman", ctypes.c_int, [_P, _P, _P, ctypes.POINTER(sb_sb_opts), ctypes.POINTER(sb_pcg_result)]),
    ("sb_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("sb_plan_last_error", ctypes.c_char_p, [_P]),
    ("sb_kernel_launches", ctypes.c_uint64, []),
    ("sb_apply_precond_noalloc", ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    ("sb_set_wait_check", ctypes.c_int, [_P, ctypes.c_uint, ctypes.c_int]),
    ("sb_split_bregman_many", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P),
                                             ctypes.POINTER(_P), ctypes.POINTER(sb_sb_opts),
                                             ctypes.POINTER(ctypes.POINTER(sb_pcg_result))]),
    ("sb_coil_compress", ctypes.c_int, [_P, _P, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P,
                                        _P, ctypes.POINTER(ctypes.c_double), _P]),
    ("sb_coil_compression_matrix", ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    ("sb_plan_set_timing", ctypes.c_int, [_P, ctypes.c_uint]),
    ("sb_set_graphs", ctypes.c_int, [_P, ctypes.c_int]),
    ("sb_set_tuning", ctypes.c_int, [_P, _P]),
    ("sb_get_tuning", ctypes.c_int, [_P, _P]),
    ("sb_plan_get_timing", ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                          ctypes.POINTER(ctypes.c_double)]),
]

# sb_kernel_class
SB_KCLASS_APPLY_A = 0
SB_KCLASS_PRECOND_ROW_FWD = 1
SB_KCLASS_PRECOND_COL = 2
SB_KCLASS_PRECOND_ROW_INV = 3
SB_KCLASS_RHS = 4
SB_KCLASS_SB_UPDATE = 5
SB_KCLASS_VEC = 6
SB_KCLASS_OTHER = 7
SB_KCLASS_PRECOND_FUSED = 8
SB_KCLASS_COUNT = 9
KCLASS_NAMES = ["apply_A", "precond_row_fwd", "precond_col", "precond_row_inv", "rhs", "sb_update", "vec",
                "other", "precond_fused"]


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no fallback)")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load()


class SbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


def status_string(status: int) -> str:
    return _lib.sb_status_string(status).decode()


def kernel_launches() -> int:
    return int(_lib.sb_kernel_launches())


def _check(status: int, plan=None, allow=()):
    if status != SB_OK and status not in allow:
        msg = _lib.sb_plan_last_error(plan).decode() if plan else ""
        raise SbError(status, msg)
    return status


def plan_desc(nx, ny, ncoils, nbatch, mu, lam, gam, wavelet_levels, prec=SB_PREC_FP32, groups=0,
              precond_passes=0, nz=1, wavelet=0) -> sb_plan_desc:
    """nz > 1 describes volumes (ndim = 3) of nz planes; wavelet: SB_WAVELET_HAAR or
    SB_WAVELET_DAUB4."""
    return sb_plan_desc(3 if nz > 1 else 2, nx, ny, nz, ncoils, nbatch, mu, lam, gam, wavelet_levels, prec, groups,
                        precond_passes, wavelet)


def sb_plan_create(desc: sb_plan_desc, stream: int = 0) -> int:
    out = _P()
    _check(_lib.sb_plan_create(ctypes.byref(desc), _P(stream), ctypes.byref(out)))
    return out.value


def sb_plan_destroy(plan: int) -> None:
    _check(_lib.sb_plan_destroy(_P(plan)))


def sb_set_coils(plan: int, d_sens: int) -> None:
    _check(_lib.sb_set_coils(_P(plan), _P(d_sens)), plan)


def sb_set_mask(plan: int, d_mask: int) -> None:
    _check(_lib.sb_set_mask(_P(plan), _P(d_mask)), plan)


def sb_get_k(plan: int, d_k: int) -> None:
    _check(_lib.sb_get_k(_P(plan), _P(d_k)), plan)


def sb_apply_A(plan: int, d_x: int, d_y: int) -> None:
    _check(_lib.sb_apply_A(_P(plan), _P(d_x), _P(d_y)), plan)


def sb_apply_precond(plan: int, d_r: int, d_z: int) -> None:
    _check(_lib.sb_apply_precond(_P(plan), _P(d_r), _P(d_z)), plan)


def pcg_opts(tol=1e-3, maxit=200, fixed_iters=0, precond=SB_PRECOND_CIRCULANT) -> sb_pcg_opts:
    return sb_pcg_opts(tol, maxit, fixed_iters, precond)


def sb_pcg_solve(plan: int, d_b: int, d_x: int, opts: sb_pcg_opts, nbatch: int, allow=(SB_ERR_NOT_CONVERGED,)):
    """Returns (status, [(iters, rel_resid, converged)] per slice)."""
    res = (sb_pcg_result * nbatch)()
    st = _check(_lib.sb_pcg_solve(_P(plan), _P(d_b), _P(d_x), ctypes.byref(opts), res), plan, allow)
    return st, [(r.iters, r.rel_resid, bool(r.converged)) for r in res]


def sb_split_bregman(plan: int, d_y: int, d_x: int, n_outer: int, n_inner: int, pcg: sb_pcg_opts, nbatch: int,
                     tau_tv: float = 0.0, tau_w: float = 0.0, init_rss: bool = True,
                     allow=(SB_ERR_NOT_CONVERGED,)):
    """Returns (status, iters[nbatch][n_outer * n_inner], last results per slice)."""
    nsolve = n_outer * n_inner
    iters = (ctypes.c_int * (nbatch * nsolve))()
    opts = sb_sb_opts(n_outer, n_inner, pcg, tau_tv, tau_w, 1 if init_rss else 0,
                      ctypes.cast(iters, ctypes.POINTER(ctypes.c_int)))
    last = (sb_pcg_result * nbatch)()
    st = _check(_lib.sb_split_bregman(_P(plan), _P(d_y), _P(d_x), ctypes.byref(opts), last), plan, allow)
    it = [[iters[b * nsolve + i] for i in range(nsolve)] for b in range(nbatch)]
    return st, it, [(r.iters, r.rel_resid, bool(r.converged)) for r in last]


def sb_split_bregman_many(plans, d_ys, d_xs, nbatches, n_outer: int, n_inner: int, pcg: sb_pcg_opts,
                          tau_tv: float = 0.0, tau_w: float = 0.0, init_rss: bool = True,
                          allow=(SB_ERR_NOT_CONVERGED,)):
    """Concurrent sb_split_bregman over several plans.  Returns (status, [iters per plan],
    [last results per plan]) with the per-plan layouts of sb_split_bregman."""
    n = len(plans)
    nsolve = n_outer * n_inner
    iters = [(ctypes.c_int * (nb * nsolve))() for nb in nbatches]
    opts = (sb_sb_opts * n)(*[sb_sb_opts(n_outer, n_inner, pcg, tau_tv, tau_w, 1 if init_rss else 0,
                                         ctypes.cast(it, ctypes.POINTER(ctypes.c_int))) for it in iters])
    lasts = [(sb_pcg_result * nb)() for nb in nbatches]
    last_p = (ctypes.POINTER(sb_pcg_result) * n)(*[ctypes.cast(l, ctypes.POINTER(sb_pcg_result)) for l in lasts])
    st = _lib.sb_split_bregman_many((_P * n)(*plans), n, (_P * n)(*d_ys), (_P * n)(*d_xs), opts, last_p)
    if st != SB_OK and st not in allow:
        msgs = "; ".join(_lib.sb_plan_last_error(_P(p)).decode() for p in plans)
        raise SbError(st, msgs)
    its = [[[it[b * nsolve + i] for i in range(nsolve)] for b in range(nb)] for it, nb in zip(iters, nbatches)]
    return st, its, [[(r.iters, r.rel_resid, bool(r.converged)) for r in l] for l in lasts]


def coil_compression_matrix(cov, nv):
    """Host-only: (matrix [nv][nc] complex128, eigenvalues [nc] descending) of a Hermitian
    covariance ``cov`` (numpy complex128 [nc][nc])."""
    import numpy as np
    nc = cov.shape[0]
    c = np.ascontiguousarray(cov, np.complex128)
    mat = np.zeros((nv, nc), np.complex128)
    eig = np.zeros(nc, np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(_lib.sb_coil_compression_matrix(c.ctypes.data_as(dp), nc, nv, mat.ctypes.data_as(dp),
                                           eig.ctypes.data_as(dp)))
    return mat, eig


def coil_compress(y, sens, nv, stream=None):
    """sb_coil_compress on torch CUDA tensors y, sens [nb][nc][...]; returns (y_v, sens_v, matrices
    [nb][nv][nc] complex64 numpy, eigenvalues [nb][nc])."""
    import numpy as np
    import torch
    nb, nc = y.shape[0], y.shape[1]
    npix = y[0, 0].numel()
    yo = torch.empty((nb, nv) + tuple(y.shape[2:]), dtype=y.dtype, device=y.device)
    so = torch.empty((nb, nv) + tuple(sens.shape[2:]), dtype=sens.dtype, device=sens.device)
    mat = np.zeros((nb, nv, nc), np.complex64)
    eig = np.zeros((nb, nc), np.float64)
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(_lib.sb_coil_compress(_P(y.data_ptr()), _P(sens.data_ptr()), npix, nc, nb, nv, _P(yo.data_ptr()),
                                 _P(so.data_ptr()), _P(mat.ctypes.data), eig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 _P(s.cuda_stream)))
    return yo, so, mat, eig


def sb_apply_precond_noalloc(d_r: int, d_k: int, d_z: int, nx: int, ny: int, nbatch: int, stream: int = 0) -> None:
    """Plan-free, allocation-free M^{-1} r (see include/sb.h)."""
    _check(_lib.sb_apply_precond_noalloc(_P(d_r), _P(d_k), _P(d_z), nx, ny, nbatch, _P(stream)))


def sb_plan_set_timing(plan: int, class_mask: int) -> None:
    _check(_lib.sb_plan_set_timing(_P(plan), class_mask), plan)


def sb_plan_get_timing(plan: int, kernel_class: int):
    """(launches, total_ms) of the kernel class since sb_plan_set_timing."""
    n = ctypes.c_uint64()
    ms = ctypes.c_double()
    _check(_lib.sb_plan_get_timing(_P(plan), kernel_class, ctypes.byref(n), ctypes.byref(ms)), plan)
    return int(n.value), float(ms.value)


class Plan:
    """Owns an sb_plan and the device tensors it borrows (torch CUDA tensors)."""

    def __init__(self, nx, ny, ncoils, nbatch, mu, lam, gam, wavelet_levels, stream=None, groups=0,
                 precond_passes=0, nz=1, wavelet=0, prec=SB_PREC_FP32):
        import torch
        self.torch = torch
        self.nbatch = nbatch
        self.shape = (nbatch, nz, ny, nx) if nz > 1 else (nbatch, ny, nx)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        self.handle = sb_plan_create(plan_desc(nx, ny, ncoils, nbatch, mu, lam, gam, wavelet_levels, prec=prec,
                                               groups=groups, precond_passes=precond_passes, nz=nz, wavelet=wavelet),
                                     s.cuda_stream)
        self._sens = None

    def close(self):
        if self.handle:
            sb_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c64(self, t):
        assert t.is_cuda and t.dtype == self.torch.complex64 and t.is_contiguous()
        return t.data_ptr()

    def set_coils(self, sens):
        self._sens = sens  # borrowed by the plan: keep it alive
        sb_set_coils(self.handle, self._c64(sens))

    def set_mask(self, mask):
        assert mask.is_cuda and mask.dtype == self.torch.uint8 and mask.is_contiguous()
        sb_set_mask(self.handle, mask.data_ptr())

    def k(self):
        out = self.torch.empty(self.shape, dtype=self.torch.float32, device="cuda")
        sb_get_k(self.handle, out.data_ptr())
        return out

    def apply_A(self, x, y=None):
        y = self.torch.empty_like(x) if y is None else y
        sb_apply_A(self.handle, self._c64(x), self._c64(y))
        return y

    def apply_precond(self, r, z=None):
        z = self.torch.empty_like(r) if z is None else z
        sb_apply_precond(self.handle, self._c64(r), self._c64(z))
        return z

    def pcg_solve(self, b, x, **kw):
        return sb_pcg_solve(self.handle, self._c64(b), self._c64(x), pcg_opts(**kw), self.nbatch)

    def set_tuning(self, col_tile: int = 0, poll_every: int = 0, apply_tile: int = 0, general_passes: int = 0):
        """Columns per CTA of the preconditioner's column pass (8, 16, 32), PCG iterations per
        convergence poll, columns per CTA of q = A p at 256 and 512 rows (8, 16) and the general
        path's schedule of q = A p and of the right-hand side (1 = one cluster launch each, 3 =
        three passes); 0 keeps the current value."""
        t = sb_tuning(col_tile, poll_every, apply_tile, general_passes)
        _check(_lib.sb_set_tuning(_P(self.handle), ctypes.byref(t)), self.handle)

    def tuning(self) -> dict:
        t = sb_tuning(0, 0, 0, 0)
        _check(_lib.sb_get_tuning(_P(self.handle), ctypes.byref(t)), self.handle)
        return {"col_tile": t.col_tile, "poll_every": t.poll_every, "apply_tile": t.apply_tile,
                "general_passes": t.general_passes}

    def set_graphs(self, enable: bool):
        """Replay the PCG iteration blocks from CUDA graphs (default) or launch directly."""
        _check(_lib.sb_set_graphs(_P(self.handle), 1 if enable else 0), self.handle)

    def set_timing(self, class_mask: int):
        sb_plan_set_timing(self.handle, class_mask)

    def set_wait_check(self, wait_polls: int = 0, withhold_coil_tiles: bool = False):
        """Poll limit of the bounded device waits (0 = default) and, for checking them, whether
        the line-path coil-tile kernels withhold their TMA requests (see include/sb.h)."""
        _check(_lib.sb_set_wait_check(_P(self.handle), wait_polls, 1 if withhold_coil_tiles else 0), self.handle)

    def timing(self, kernel_class: int):
        return sb_plan_get_timing(self.handle, kernel_class)

    def split_bregman(self, y, x, n_outer, n_inner=1, tau_tv=0.0, tau_w=0.0, init_rss=True, **pcg_kw):
        return sb_split_bregman(self.handle, self._c64(y), self._c64(x), n_outer, n_inner, pcg_opts(**pcg_kw),
                                self.nbatch, tau_tv, tau_w, init_rss)


def split_bregman_many(plans, ys, xs, n_outer, n_inner=1, tau_tv=0.0, tau_w=0.0, init_rss=True, **pcg_kw):
    """sb_split_bregman_many over Plan objects (one per geometry) and their y / x tensors.  Give
    each plan its own CUDA stream so that the reconstructions overlap on the GPU."""
    return sb_split_bregman_many([p.handle for p in plans], [p._c64(y) for p, y in zip(plans, ys)],
                                 [p._c64(x) for p, x in zip(plans, xs)], [p.nbatch for p in plans], n_outer,
                                 n_inner, pcg_opts(**pcg_kw), tau_tv, tau_w, init_rss)
