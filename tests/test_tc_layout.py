"""CPU model of the tensor-core q = A p kernels' shared-memory operand layouts.

The layout constants are read from the kernel source (k_applyA_tc.cu), so this model follows any
change to them.  A 16-bit element at byte offset o of an operand buffer is mem[o // 2]; the
kernels' stores (own rows and the transposes of the factorisation) and the descriptor reads of
tcgen05.mma (K-major core matrices: row rr of a core matrix at +16 rr, element kk at +2 kk,
K-adjacent core matrices `lbo` apart, 8-row groups `sbo` apart) are modelled on those arrays.
Checked: the four-stage transform (256 = 16 x 16 and 512 = 16 x 32) with the bf16 and fp16 splits
against numpy's orthonormal FFT round trip through a line mask; every stored element inside the
buffer at a distinct address; the transposed stores of a warp on 32 distinct banks and the
16-byte row stores at the minimum four wavefronts.  This checks the layout and stage algebra on
the host; the kernels themselves are checked against the FP64 oracle by the GPU tests.
"""
import pathlib
import re

import numpy as np
import pytest

SRC = pathlib.Path(__file__).resolve().parents[1] / "paper_1710_01758_gb300" / "csrc" / "k_applyA_tc.cu"


def constants():
    text = SRC.read_text()

    def get(name):
        return int(re.search(rf"\b{name}\s*=\s*(\d+)", text).group(1))

    c = {k: get(k) for k in ("kLboA", "kSboA", "kLboB", "kSboB", "kBmat", "kSbo1", "kSbo2", "kSboB32", "kBmat32",
                             "kA5bytes")}
    c["kAbytes"] = 16 * c["kSboA"]
    return c


C = constants()


def rnd(x, dt):
    """Round-to-nearest-even to bf16 or fp16, returned as float64."""
    x = np.asarray(x, np.float32)
    if dt == "fp16":
        return x.astype(np.float16).astype(np.float64)
    b = x.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


def split(v, dt):
    """hi = round(v), lo = round((v - hi) 2^L) in FP32 arithmetic, as the kernels do."""
    ls = np.float32(1.0 if dt == "bf16" else 1024.0)
    v = np.asarray(v, np.float32)
    hi = rnd(v, dt)
    lo = rnd((v - hi.astype(np.float32)) * ls, dt)
    return hi, lo


def dft_block(n, scale, dt, sbo):
    """The six B operands (forward / inverse x hi, hi 2^-L, lo) of the real-form scaled n-point DFT."""
    L = 1.0 if dt == "bf16" else 1.0 / 1024.0
    N = 2 * n
    nn, k = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    ko, e = nn >> 1, k >> 1
    off = ((nn >> 3) * sbo + (k >> 3) * 128 + (nn & 7) * 16 + (k & 7) * 2) // 2
    mats = []
    for sgn in (-2.0, 2.0):
        th = sgn * np.pi * ((ko * e) % n) / n
        wr, wi = np.cos(th) * scale, np.sin(th) * scale
        v = np.where(nn % 2 == 0, np.where(k % 2 == 0, wr, -wi), np.where(k % 2 == 0, wi, wr))
        h = rnd(v, dt)
        lo = rnd(v - h, dt)
        h2 = rnd(h * L, dt)
        for part in (h, h2, lo):
            img = np.zeros(N * N)
            img[off] = part
            mats.append(img)
    return mats


def gather(mem, start, rows, lbo, sbo, ksteps):
    """The [rows x 16 ksteps] matrix an MMA sequence reads from a K-major operand at `start`."""
    r = np.arange(rows)[:, None]
    k = np.arange(16 * ksteps)[None, :]
    off = start + (r >> 3) * sbo + (k >> 3) * lbo + (r & 7) * 16 + (k & 7) * 2
    return mem[off // 2]


def mma_stage(A, Bs, a_start, rows, lbo, sbo, b_sbo, n_out, ksteps):
    """sum over the split products A_hi B_hi + A_lo B_hi' + A_hi B_lo (hi at a_start, lo one part later)."""
    a_hi = gather(A, a_start, rows, lbo, sbo, ksteps)
    a_lo = gather(A, a_start + ksteps * 2 * lbo, rows, lbo, sbo, ksteps)
    b = [gather(m, 0, n_out, 128, b_sbo, ksteps) for m in Bs]
    return a_hi @ b[0].T + a_lo @ b[1].T + a_hi @ b[2].T


def store(A, off_fn, rows, kcs, vals, dt, used=None):
    """Store complex vals at (row, complex element kc) of both parts; optionally record addresses."""
    hr, lr = split(vals.real, dt)
    hi_, li = split(vals.imag, dt)
    for part, (re_, im_) in ((0, (hr, hi_)), (1, (lr, li))):
        o = off_fn(rows, kcs, part)
        A[o // 2] = re_
        A[o // 2 + 1] = im_
        if used is not None:
            used.append(o)


def a_off(sbo, kpart):
    lbo = C["kLboA"]

    def f(row, kc, part):
        k = 2 * kc
        return (row >> 3) * sbo + (part * kpart + (k >> 3)) * lbo + (row & 7) * 16 + (k & 7) * 2
    return f


def reference(u, mask):
    return np.fft.ifft(mask[:, None] * np.fft.fft(u, axis=0, norm="ortho"), axis=0, norm="ortho")


@pytest.mark.parametrize("dt,tol", [("fp16", 1e-6), ("bf16", 3e-5)])
def test_256_row_transform(dt, tol):
    rng = np.random.default_rng(0)
    u = (rng.standard_normal((256, 8)) + 1j * rng.standard_normal((256, 8))) * 0.4
    mask = (rng.random(256) < 0.3).astype(float)
    Bs = dft_block(16, 0.25, dt, C["kSboB"])
    fwd, inv = Bs[:3], Bs[3:]
    tw = np.exp(-2j * np.pi * np.arange(256) / 256)
    off = a_off(C["kSboA"], 4)
    A = np.zeros(C["kAbytes"] // 2)
    used = []
    j, s, e = np.meshgrid(np.arange(8), np.arange(16), np.arange(16), indexing="ij")
    rows = 16 * j + s
    store(A, off, rows, e, u[s + 16 * e, j], dt, used)
    D = mma_stage(A, fwd, 0, 128, C["kLboA"], C["kSboA"], C["kSboB"], 32, 2)
    T = (D[:, 0::2] + 1j * D[:, 1::2]).reshape(8, 16, 16)  # [j, s, k1]
    k1 = e  # the third grid axis serves as k1 here
    store(A, off, 16 * j + k1, s, T * tw[s * k1], dt, used)
    D = mma_stage(A, fwd, 0, 128, C["kLboA"], C["kSboA"], C["kSboB"], 32, 2)
    X = (D[:, 0::2] + 1j * D[:, 1::2]).reshape(8, 16, 16)  # [j, k1, k2]
    Xf = np.zeros((256, 8), complex)
    Xf[s + 16 * e, j] = X  # k = k1 + 16 k2 with k1 = s axis, k2 = e axis
    assert np.linalg.norm(Xf - np.fft.fft(u, axis=0, norm="ortho")) <= tol * np.linalg.norm(Xf)
    store(A, off, 16 * j + s, e, X * mask[s + 16 * e], dt)
    D = mma_stage(A, inv, 0, 128, C["kLboA"], C["kSboA"], C["kSboB"], 32, 2)
    T2 = (D[:, 0::2] + 1j * D[:, 1::2]).reshape(8, 16, 16)  # [j, k1, s']
    store(A, off, 16 * j + e, s, np.conj(tw[e * s]) * T2, dt)  # row (j, s'), element k1
    D = mma_stage(A, inv, 0, 128, C["kLboA"], C["kSboA"], C["kSboB"], 32, 2)
    V = (D[:, 0::2] + 1j * D[:, 1::2]).reshape(8, 16, 16)  # [j, s, e]
    v = np.zeros((256, 8), complex)
    v[s + 16 * e, j] = V
    ref = reference(u, mask)
    assert np.linalg.norm(v - ref) <= tol * np.linalg.norm(ref)
    # every element inside the buffer, each 4-byte pair at its own address
    allo = np.concatenate([o.ravel() for o in used])
    assert allo.max() + 4 <= C["kAbytes"] and allo.min() >= 0
    assert len(np.unique(used[0])) == used[0].size and len(np.unique(used[2])) == used[2].size


@pytest.mark.parametrize("dt,tol", [("fp16", 1e-6), ("bf16", 3e-5)])
def test_512_row_transform(dt, tol):
    rng = np.random.default_rng(1)
    u = (rng.standard_normal((512, 8)) + 1j * rng.standard_normal((512, 8))) * 0.4
    mask = (rng.random(512) < 0.3).astype(float)
    B16 = dft_block(16, 0.25, dt, C["kSboB"])
    B32 = dft_block(32, 1 / np.sqrt(32), dt, C["kSboB32"])
    tw = np.exp(-2j * np.pi * np.arange(512) / 512)
    off1, off2 = a_off(C["kSbo1"], 4), a_off(C["kSbo2"], 8)
    A = np.zeros(C["kA5bytes"] // 2)

    def stage16(Bs):
        return np.concatenate([mma_stage(A, Bs, g * 16 * C["kSbo1"], 128, C["kLboA"], C["kSbo1"], C["kSboB"], 32, 2)
                               for g in (0, 1)])

    def stage32(Bs):
        return mma_stage(A, Bs, 0, 128, C["kLboA"], C["kSbo2"], C["kSboB32"], 64, 4)

    j, s, e = np.meshgrid(np.arange(8), np.arange(32), np.arange(16), indexing="ij")  # y = s + 32 e
    store(A, off1, 32 * j + s, e, u[s + 32 * e, j], dt)
    D = stage16(B16[:3])
    T = (D[:, 0::2] + 1j * D[:, 1::2]).reshape(8, 32, 16)  # [j, s, k1]
    store(A, off2, 16 * j + e, s, T * tw[s * e], dt)  # row (j, k1), element s
    D = stage32(B32[:3])
    X = (D[:, 0::2] + 1j * D[:, 1::2]).reshape(8, 16, 32)  # [j, k1, k2]
    jj, k1, k2 = np.meshgrid(np.arange(8), np.arange(16), np.arange(32), indexing="ij")
    Xf = np.zeros((512, 8), complex)
    Xf[k1 + 16 * k2, jj] = X
    assert np.linalg.norm(Xf - np.fft.fft(u, axis=0, norm="ortho")) <= tol * np.linalg.norm(Xf)
    store(A, off2, 16 * jj + k1, k2, X * mask[k1 + 16 * k2], dt)
    D = stage32(B32[3:])
    T2 = (D[:, 0::2] + 1j * D[:, 1::2]).reshape(8, 16, 32)  # [j, k1, s']
    store(A, off1, 32 * jj + k2, k1, np.conj(tw[k2 * k1]) * T2, dt)  # row (j, s'), element k1
    D = stage16(B16[3:])
    V = (D[:, 0::2] + 1j * D[:, 1::2]).reshape(8, 32, 16)  # [j, s, e]
    v = np.zeros((512, 8), complex)
    v[s + 32 * e, j] = V
    ref = reference(u, mask)
    assert np.linalg.norm(v - ref) <= tol * np.linalg.norm(ref)
    assert max(off1(255, 15, 1), off2(127, 31, 1)) + 4 <= C["kA5bytes"]


def banks(offs):
    """Multiplicity of the most-used 4-byte bank over a warp's accesses."""
    return np.bincount((np.asarray(offs) // 4) % 32, minlength=32).max()


def test_store_bank_patterns():
    off = a_off(C["kSboA"], 4)
    for w in range(8):  # 256 rows: two threads per TMEM lane; warp w reads lanes 32 (w mod 4) ..
        r = 32 * (w & 3) + np.arange(32)
        h = w >> 2
        j, s = r >> 4, r & 15
        for i in range(8):  # transposed stores: element s of row (j, k1 = 8 h + i)
            assert banks(off(16 * j + 8 * h + i, s, 0)) == 1
        for q2 in range(2):  # own-row 16-byte stores: four words per thread, four wavefronts
            o = off(r, 8 * h + 4 * q2, 0)
            assert banks(np.concatenate([o + 4 * t for t in range(4)])) == 4
    off1, off2 = a_off(C["kSbo1"], 4), a_off(C["kSbo2"], 8)
    for w in range(8):  # 512 rows: stage-1 row R1 = 128 h + r, stage-2 row r with half h
        r = 32 * (w & 3) + np.arange(32)
        h = w >> 2
        R1 = 128 * h + r
        j1, s = R1 >> 5, R1 & 31
        for kk in range(16):  # stage 2 input: element s of row (j1, k1)
            assert banks(off2(16 * j1 + kk, s, 0)) == 1
        j2, k1 = r >> 4, r & 15
        for i in range(16):  # stage 4 input: element k1 of row (j2, s' = 16 h + i)
            assert banks(off1(32 * j2 + 16 * h + i, k1, 0)) == 1
