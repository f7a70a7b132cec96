// q = A p with the DFT stages of the data term on the tensor cores (the split-precision modes).
//
// A = mu sum_c S_c^H F^H R F S_c + lambda D^H D + gamma I (Eq. system; PI+CS paragraph), with a
// mask constant along the readout axis x, so the data term is a length-256 DFT along y per
// column, the mask, and the inverse DFT.  Each 256-point transform is factored 16 x 16:
// y = s + 16 e and k = k1 + 16 k2,
//   X[k1 + 16 k2] = 1/4 sum_s W_256^{s k1} W_16^{s k2} (1/4 sum_e W_16^{e k1} u[s + 16 e])
// (unitary overall, 1/4 per stage), and the inverse runs the conjugate steps in reverse order.
// Each of the four radix-16 stages is one tensor-core product D[128 x 32] = A[128 x 32] B^T with
// A = 128 sub-vectors of 16 complex values (8 columns x 16 per column) as 32 reals, interleaved
// (re, im), and B = the real form of the 16-point DFT matrix (32 x 32).  The operands are split
// in two 16-bit terms, v = v_hi + v_lo (bf16 or fp16), and a stage accumulates
//   A_hi B_hi + (A_lo 2^L)(B_hi 2^-L) + A_hi B_lo
// in FP32 in tensor memory (L = 10 for fp16, which keeps the low parts in its normal range;
// L = 0 for bf16).  For fp16 the p tile of a CTA is first scaled by an exact power of two so
// that its largest component lies in [1/2, 1).  Between stages the 32 accumulator columns of
// each lane come back to registers (tcgen05.ld), take the twiddles W_256^{+-s k1} or the mask,
// and are split and stored as the next stage's A operand; the transposes of the factorisation
// happen in that store.  Coil tiles arrive by TMA as 8-column boxes with the 64-byte swizzle.
// The epilogue (periodic 5-point stencil, gamma p, Re(p^H q) and alpha) is that of the FP32
// kernel.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"
#include "umma.cuh"

namespace sb {
namespace {

constexpr int kTcNY = 256, kTcTX = 8, kTcNT = 256;
// A operand: 128 rows x (32 hi + 32 lo) 16-bit elements.  K-adjacent core matrices 144 B apart
// and 8-row groups 1184 B apart: the transposed stores of a warp (16 rows' worth of one element
// each from 32 threads) then fall on 32 distinct banks.
constexpr uint32_t kLboA = 144, kSboA = 1184;
constexpr int kAbytes = 16 * kSboA;
// B operands: 32 rows x 32 elements, 2048 B each, in the order forward (hi, hi 2^-L, lo),
// inverse (hi, hi 2^-L, lo).
constexpr uint32_t kLboB = 128, kSboB = 512, kBmat = 2048;
constexpr int kBbytes = 6 * kBmat;

__device__ __forceinline__ uint32_t pad1024(const void* p) {
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    return ((a + 1023u) & ~1023u) - a;
}

// 8-column tile (64-byte rows) with the 64-byte TMA swizzle: 16-byte chunk index ^= (row >> 1) & 3
__device__ __forceinline__ int swz64(int row, int col) {
    return row * kTcTX + ((((col >> 1) ^ ((row >> 1) & 3)) << 1) | (col & 1));
}

// byte offset of complex element kc (elements 2 kc, 2 kc + 1) of A-operand row `row`, part 0 (hi)
// or 1 (lo)
__device__ __forceinline__ uint32_t a_off(int row, int kc, int part) {
    const int k = 2 * kc;
    return (uint32_t)(row >> 3) * kSboA + (uint32_t)(part * 4 + (k >> 3)) * kLboA + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

template <bool BF16>
__device__ __forceinline__ void split_pack(float2 v, float ls, uint32_t& hi, uint32_t& lo) {
    if constexpr (BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn((v.x - hf.x) * ls, (v.y - hf.y) * ls);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __half2 h = __floats2half2_rn(v.x, v.y);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn((v.x - hf.x) * ls, (v.y - hf.y) * ls);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

// half h of the thread's own A row: complex elements 8 h .. 8 h + 7, two 16-byte stores per part
template <bool BF16>
__device__ __forceinline__ void write_half_row(unsigned char* A, int row, int h, const float2 (&v)[8], float ls) {
#pragma unroll
    for (int q2 = 0; q2 < 2; ++q2) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) split_pack<BF16>(v[4 * q2 + i], ls, hi[i], lo[i]);
        *reinterpret_cast<uint4*>(A + a_off(row, 8 * h + 4 * q2, 0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(A + a_off(row, 8 * h + 4 * q2, 1)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

template <bool BF16>
__device__ __forceinline__ void write_elem(unsigned char* A, int row, int kc, float2 v, float ls) {
    uint32_t h, l;
    split_pack<BF16>(v, ls, h, l);
    *reinterpret_cast<uint32_t*>(A + a_off(row, kc, 0)) = h;
    *reinterpret_cast<uint32_t*>(A + a_off(row, kc, 1)) = l;
}

// one radix-16 stage on 128 sub-vectors: 2 K-steps x 3 split products, D overwritten
__device__ __forceinline__ void issue_stage(uint32_t d_tmem, uint32_t a_s, uint32_t b_s, uint32_t idesc) {
#pragma unroll
    for (int st = 0; st < 2; ++st) {
        const uint64_t ah = umma_desc(a_s + (uint32_t)(2 * st) * kLboA, kLboA, kSboA);
        const uint64_t al = umma_desc(a_s + (uint32_t)(4 + 2 * st) * kLboA, kLboA, kSboA);
        const uint64_t bh = umma_desc(b_s + (uint32_t)(2 * st) * kLboB, kLboB, kSboB);
        const uint64_t bh2 = umma_desc(b_s + kBmat + (uint32_t)(2 * st) * kLboB, kLboB, kSboB);
        const uint64_t bl = umma_desc(b_s + 2 * kBmat + (uint32_t)(2 * st) * kLboB, kLboB, kSboB);
        umma_f16(d_tmem, ah, bh, idesc, st > 0 ? 1u : 0u);
        umma_f16(d_tmem, al, bh2, idesc, 1u);
        umma_f16(d_tmem, ah, bl, idesc, 1u);
    }
}

template <bool BF16, bool PCG>
__global__ void __launch_bounds__(kTcNT, 3)
k_apply_A_tc(const __grid_constant__ CUtensorMap smap8, const float2* __restrict__ p, float2* __restrict__ q,
             const float* __restrict__ maskw, const float2* __restrict__ tw_g, const uint4* __restrict__ bmat,
             int nx, int nc, float mu, float lam, float gam, SliceState* st, Red red) {
    constexpr int NY = kTcNY, NT = kTcNT, TX = kTcTX, NW = NT / 32;
    const int b = blockIdx.y;
    if (PCG && st[b].state != ST_ACTIVE) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + pad1024(smem_raw);
    float2* sbuf = reinterpret_cast<float2*>(smem);                // [2][NY * TX] swizzled coil tiles
    unsigned char* Aop = smem + 2 * NY * TX * sizeof(float2);      // A operand
    unsigned char* Bop = Aop + kAbytes;                            // six B operands
    float2* tw = reinterpret_cast<float2*>(Bop + kBbytes);          // tw[16 a + b] = W_256^{a b}
    float2* halo = tw + NY;                                         // [2][NY]: columns x0-1, x0+TX
    float* mk = reinterpret_cast<float*>(halo + 2 * NY);
    double* red_s = reinterpret_cast<double*>(mk + NY);
    __shared__ __align__(8) uint64_t full[2], mma_bar;
    __shared__ uint32_t tmem_s;
    __shared__ float wmax[NW];
    __shared__ int flag;

    // TMEM lane (= A row) r = (j, s) is shared by the threads tid = r (half 0) and r + 128
    // (half 1; warps w and w + 4 read the same lanes): each owns 8 of the row's 16 complex values
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int r = tid & 127, h = tid >> 7;
    const int j = r >> 4, s = r & 15;  // column of the tile, sub-vector index within it
    const int x0 = blockIdx.x * TX, x = x0 + j;
    const int rbase = swz64(s, j);     // rows s + 16 e share the swizzle term of s
    auto S_at = [rbase](const float2* S, int e) { return S[rbase + e * 16 * TX]; };
    auto load_tile = [&](int c) {
        uint64_t* bar = &full[c & 1];
        mbar_arrive_expect_tx(bar, NY * TX * sizeof(float2));
        tma_load_2d(sbuf + (c & 1) * NY * TX, &smap8, 2 * x0, (b * nc + c) * NY, bar);
    };

    if (w == 0) tmem_alloc(&tmem_s, 32);
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&mma_bar, 1);
        mbar_init_fence();
    }
    for (int i = tid; i < kBbytes / 16; i += NT) reinterpret_cast<uint4*>(Bop)[i] = bmat[i];
    for (int i = tid; i < NY; i += NT) {
        tw[i] = tw_g[(i >> 4) * (i & 15)];
        mk[i] = maskw[(size_t)b * NY + i] * (float)NY;  // the line weights carry 1/ny; the stages are unitary
    }
    const size_t img = (size_t)b * NY * nx;
    float2 pv[8], acc[8];
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        pv[i] = p[img + (size_t)(s + 16 * (8 * h + i)) * nx + x];
        acc[i] = make_float2(0.f, 0.f);
        m = fmaxf(m, fmaxf(fabsf(pv[i].x), fabsf(pv[i].y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) wmax[w] = m;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0)
        for (int c = 0; c < 2 && c < nc; ++c) load_tile(c);
    m = wmax[0];
#pragma unroll
    for (int i = 1; i < NW; ++i) m = fmaxf(m, wmax[i]);
    float scale = 1.f, unscale = 1.f;
    if (!BF16 && m > 0.f && isfinite(m)) {
        int ex;
        frexpf(m, &ex);
        scale = ldexpf(1.f, -ex);
        unscale = ldexpf(1.f, ex);
    }
    const float ls = BF16 ? 1.f : 1024.f;
    const uint32_t tmem = tmem_s;
    const uint32_t t_lane = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(16 * h);
    const uint32_t a_s = smem_addr(Aop), b_s = smem_addr(Bop);
    constexpr uint32_t idesc = umma_idesc_f16(128, 32, BF16);
    uint32_t mph = 0;
    // operands stored -> one thread issues the stage -> everyone waits for its completion
    auto stage = [&](int dir, int prefetch) {
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            issue_stage(tmem, a_s, b_s + (uint32_t)dir * 3u * kBmat, idesc);
            umma_commit(&mma_bar);
            if (prefetch >= 0) load_tile(prefetch);  // the other stage's tile is no longer read
        }
        mbar_wait(&mma_bar, mph, red.err, red.wait_limit);
        mph ^= 1u;
        tc_fence_after();
    };

    float d[16];
    for (int c = 0; c < nc; ++c) {
        const float2* S = sbuf + (c & 1) * NY * TX;
        mbar_wait(&full[c & 1], (c >> 1) & 1, red.err, red.wait_limit);
        float2 u[8];
        // stage 1: row (j, s) holds u[s + 16 e], e < 16 (this thread: e = 8 h + i)
#pragma unroll
        for (int i = 0; i < 8; ++i) u[i] = cscale(cmul(S_at(S, 8 * h + i), pv[i]), scale);
        write_half_row<BF16>(Aop, r, h, u, ls);
        stage(0, (c >= 1 && c + 1 < nc) ? c + 1 : -1);
        tmem_ld16(t_lane, d);  // T[s][k1], k1 = 8 h + i
        // twiddle W_256^{s k1}; row (j, k1) of stage 2 takes element s
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k1 = 8 * h + i;
            write_elem<BF16>(Aop, 16 * j + k1, s, cmul(make_float2(d[2 * i], d[2 * i + 1]), tw[16 * k1 + s]), ls);
        }
        stage(0, -1);
        tmem_ld16(t_lane, d);  // row (j, k1 = s): X[k1 + 16 k2], k2 = 8 h + i
#pragma unroll
        for (int i = 0; i < 8; ++i) u[i] = cscale(make_float2(d[2 * i], d[2 * i + 1]), mk[s + 16 * (8 * h + i)]);
        write_half_row<BF16>(Aop, r, h, u, ls);
        stage(1, -1);
        tmem_ld16(t_lane, d);  // row (j, k1 = s): T'[s'][k1], s' = 8 h + i
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int s2 = 8 * h + i;
            write_elem<BF16>(Aop, 16 * j + s2, s, cmulc(tw[16 * s2 + s], make_float2(d[2 * i], d[2 * i + 1])), ls);
        }
        stage(1, -1);
        tmem_ld16(t_lane, d);  // row (j, s): (F^H R F u)[s + 16 e], e = 8 h + i, scaled
#pragma unroll
        for (int i = 0; i < 8; ++i)
            acc[i] = cfmac(acc[i], S_at(S, 8 * h + i), make_float2(d[2 * i], d[2 * i + 1]));
    }
    // periodic 5-point stencil for lambda (D_x^H D_x + D_y^H D_y) p; p tile in stage 0
    tc_fence_before();
    __syncthreads();
    if (w == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 32);
    }
    float2* pt = sbuf;
#pragma unroll
    for (int i = 0; i < 8; ++i) pt[rbase + (8 * h + i) * 16 * TX] = pv[i];
    for (int i = tid; i < NY; i += NT) {
        halo[i] = p[img + (size_t)i * nx + (x0 == 0 ? nx - 1 : x0 - 1)];
        halo[NY + i] = p[img + (size_t)i * nx + (x0 + TX == nx ? 0 : x0 + TX)];
    }
    __syncthreads();
    float dot = 0.f;
    const float mus = mu * unscale;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int y = s + 16 * (8 * h + i);
        const float2 up = pt[swz64(y == 0 ? NY - 1 : y - 1, j)];
        const float2 dn = pt[swz64(y == NY - 1 ? 0 : y + 1, j)];
        const float2 lf = j > 0 ? pt[swz64(y, j - 1)] : halo[y];
        const float2 rt = j < TX - 1 ? pt[swz64(y, j + 1)] : halo[NY + y];
        const float tvx = 4.f * pv[i].x - up.x - dn.x - lf.x - rt.x;
        const float tvy = 4.f * pv[i].y - up.y - dn.y - lf.y - rt.y;
        float2 o;
        o.x = fmaf(mus, acc[i].x, fmaf(lam, tvx, gam * pv[i].x));
        o.y = fmaf(mus, acc[i].y, fmaf(lam, tvy, gam * pv[i].y));
        q[img + (size_t)y * nx + x] = o;
        dot = fmaf(pv[i].x, o.x, fmaf(pv[i].y, o.y, dot));
    }
    if constexpr (PCG) {
        double v[1] = {(double)dot}, tot[1];
        const int np = gridDim.x;
        if (last_block_total<1>(v, red.part, np, b * np + blockIdx.x, red.counter + b, tot, red_s, &flag) &&
            threadIdx.x == 0) {
            SliceState& S = st[b];
            const double pq = tot[0];
            S.pq = pq;
            if (!isfinite(pq) || !isfinite(S.rho)) {
                S.state = ST_NONFINITE;
            } else if (!(pq > 0.0)) {
                S.state = ST_BREAKDOWN;
            } else {
                S.alpha = S.rho / pq;
                S.iters += 1;
            }
        }
    }
}

// ---- 512-row columns: 512 = 16 x 32, y = s + 32 e, k = k1 + 16 k2 (s, k2 < 32; e, k1 < 16).
// Stages 1 and 4 are radix 16 over e (k1) on the 256 sub-vectors (j, s) of 8 columns: two M = 128
// MMA groups, TMEM columns 0-31 and 32-63; stages 2 and 3 are radix 32 over s (k2) on the 128
// sub-vectors (j, k1): one M = 128, N = 64 product with four K-steps.  One thread per stage-1 row
// (16 values), two per stage-2 row (16 of its 32 values).  The 1/4 and 1/sqrt 32 scales make the
// transform unitary.
constexpr int kT5NY = 512;
constexpr uint32_t kSbo1 = 1168;  // stage-1/4 A rows (16 complex per part): 4 row-groups apart = 64 mod 128 B
constexpr uint32_t kSbo2 = 2320;  // stage-2/3 A rows (32 complex per part)
constexpr int kA5bytes = 37888;   // max(32 x 1168, 16 x 2320), rounded up to 1 KB
constexpr uint32_t kSboB32 = 1024, kBmat32 = 8192;
constexpr int kB5bytes = kBbytes + 6 * (int)kBmat32;

__device__ __forceinline__ uint32_t a1_off(int row, int kc, int part) {
    const int k = 2 * kc;
    return (uint32_t)(row >> 3) * kSbo1 + (uint32_t)(part * 4 + (k >> 3)) * kLboA + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}
__device__ __forceinline__ uint32_t a2_off(int row, int kc, int part) {
    const int k = 2 * kc;
    return (uint32_t)(row >> 3) * kSbo2 + (uint32_t)(part * 8 + (k >> 3)) * kLboA + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

template <bool BF16>
__device__ __forceinline__ void write_elem_at(unsigned char* A, uint32_t off_hi, uint32_t off_lo, float2 v, float ls) {
    uint32_t h, l;
    split_pack<BF16>(v, ls, h, l);
    *reinterpret_cast<uint32_t*>(A + off_hi) = h;
    *reinterpret_cast<uint32_t*>(A + off_lo) = l;
}

// 16 consecutive complex values (elements kc0 .. kc0 + 15) of one A row, four 16-byte stores per part
template <bool BF16, class Off>
__device__ __forceinline__ void write16(unsigned char* A, Off off, int row, int kc0, const float2 (&v)[16], float ls) {
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) split_pack<BF16>(v[4 * q4 + i], ls, hi[i], lo[i]);
        *reinterpret_cast<uint4*>(A + off(row, kc0 + 4 * q4, 0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(A + off(row, kc0 + 4 * q4, 1)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

// radix-16 stage on the 256 rows of the stage-1 layout: two M groups into TMEM columns 0 and 32
__device__ __forceinline__ void issue_stage16x2(uint32_t d_tmem, uint32_t a_s, uint32_t b_s, uint32_t idesc) {
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        const uint32_t ag = a_s + (uint32_t)g * 16u * kSbo1;
#pragma unroll
        for (int st = 0; st < 2; ++st) {
            const uint64_t ah = umma_desc(ag + (uint32_t)(2 * st) * kLboA, kLboA, kSbo1);
            const uint64_t al = umma_desc(ag + (uint32_t)(4 + 2 * st) * kLboA, kLboA, kSbo1);
            const uint64_t bh = umma_desc(b_s + (uint32_t)(2 * st) * kLboB, kLboB, kSboB);
            const uint64_t bh2 = umma_desc(b_s + kBmat + (uint32_t)(2 * st) * kLboB, kLboB, kSboB);
            const uint64_t bl = umma_desc(b_s + 2 * kBmat + (uint32_t)(2 * st) * kLboB, kLboB, kSboB);
            umma_f16(d_tmem + 32u * g, ah, bh, idesc, st > 0 ? 1u : 0u);
            umma_f16(d_tmem + 32u * g, al, bh2, idesc, 1u);
            umma_f16(d_tmem + 32u * g, ah, bl, idesc, 1u);
        }
    }
}

// radix-32 stage on the 128 rows of the stage-2 layout: N = 64, four K-steps
__device__ __forceinline__ void issue_stage32(uint32_t d_tmem, uint32_t a_s, uint32_t b_s, uint32_t idesc) {
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        const uint64_t ah = umma_desc(a_s + (uint32_t)(2 * st) * kLboA, kLboA, kSbo2);
        const uint64_t al = umma_desc(a_s + (uint32_t)(8 + 2 * st) * kLboA, kLboA, kSbo2);
        const uint64_t bh = umma_desc(b_s + (uint32_t)(2 * st) * kLboB, kLboB, kSboB32);
        const uint64_t bh2 = umma_desc(b_s + kBmat32 + (uint32_t)(2 * st) * kLboB, kLboB, kSboB32);
        const uint64_t bl = umma_desc(b_s + 2 * kBmat32 + (uint32_t)(2 * st) * kLboB, kLboB, kSboB32);
        umma_f16(d_tmem, ah, bh, idesc, st > 0 ? 1u : 0u);
        umma_f16(d_tmem, al, bh2, idesc, 1u);
        umma_f16(d_tmem, ah, bl, idesc, 1u);
    }
}

template <bool BF16, bool PCG>
__global__ void __launch_bounds__(kTcNT, 1)
k_apply_A_tc512(const __grid_constant__ CUtensorMap smap8, const float2* __restrict__ p, float2* __restrict__ q,
                const float* __restrict__ maskw, const float2* __restrict__ tw_g, const uint4* __restrict__ bmat,
                int nx, int nc, float mu, float lam, float gam, SliceState* st, Red red) {
    constexpr int NY = kT5NY, NT = kTcNT, TX = kTcTX, NW = NT / 32;
    const int b = blockIdx.y;
    if (PCG && st[b].state != ST_ACTIVE) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + pad1024(smem_raw);
    float2* sbuf = reinterpret_cast<float2*>(smem);                // [2][NY * TX] swizzled coil tiles
    unsigned char* Aop = smem + 2 * NY * TX * sizeof(float2);      // A operand (both layouts)
    unsigned char* Bop = Aop + kA5bytes;                           // DFT16 x 6, then DFT32 x 6
    float2* tw = reinterpret_cast<float2*>(Bop + kB5bytes);         // tw[32 k1 + s] = W_512^{s k1}
    float2* halo = tw + NY;                                         // [2][NY]
    float* mk = reinterpret_cast<float*>(halo + 2 * NY);
    double* red_s = reinterpret_cast<double*>(mk + NY);
    __shared__ __align__(8) uint64_t full[2], mma_bar;
    __shared__ uint32_t tmem_s;
    __shared__ float wmax[NW];
    __shared__ int flag;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int r = tid & 127, h = tid >> 7;
    const int R1 = 128 * h + r;            // stage-1 row: column j1, sub-vector s
    const int j1 = R1 >> 5, s = R1 & 31;
    const int j2 = r >> 4, k1 = r & 15;    // stage-2 row r: column j2, frequency k1; half h
    const int x0 = blockIdx.x * TX, x = x0 + j1;
    const int rbase = swz64(s, j1);        // rows s + 32 e share the swizzle term of s
    auto S_at = [rbase](const float2* S, int e) { return S[rbase + e * 32 * TX]; };
    auto load_tile = [&](int c) {
        uint64_t* bar = &full[c & 1];
        mbar_arrive_expect_tx(bar, NY * TX * sizeof(float2));
        float2* dst = sbuf + (c & 1) * NY * TX;
        tma_load_2d(dst, &smap8, 2 * x0, (b * nc + c) * NY, bar);
        tma_load_2d(dst + 256 * TX, &smap8, 2 * x0, (b * nc + c) * NY + 256, bar);
    };

    if (w == 0) tmem_alloc(&tmem_s, 64);
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&mma_bar, 1);
        mbar_init_fence();
    }
    for (int i = tid; i < kB5bytes / 16; i += NT) reinterpret_cast<uint4*>(Bop)[i] = bmat[i];
    for (int i = tid; i < NY; i += NT) {
        tw[i] = tw_g[(i >> 5) * (i & 31)];
        mk[i] = maskw[(size_t)b * NY + i] * (float)NY;  // the line weights carry 1/ny; the stages are unitary
    }
    const size_t img = (size_t)b * NY * nx;
    float2 pv[16], acc[16];
    float m = 0.f;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        pv[e] = p[img + (size_t)(s + 32 * e) * nx + x];
        acc[e] = make_float2(0.f, 0.f);
        m = fmaxf(m, fmaxf(fabsf(pv[e].x), fabsf(pv[e].y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) wmax[w] = m;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0)
        for (int c = 0; c < 2 && c < nc; ++c) load_tile(c);
    m = wmax[0];
#pragma unroll
    for (int i = 1; i < NW; ++i) m = fmaxf(m, wmax[i]);
    float scale = 1.f, unscale = 1.f;
    if (!BF16 && m > 0.f && isfinite(m)) {
        int ex;
        frexpf(m, &ex);
        scale = ldexpf(1.f, -ex);
        unscale = ldexpf(1.f, ex);
    }
    const float ls = BF16 ? 1.f : 1024.f;
    const uint32_t tmem = tmem_s;
    const uint32_t t_lane = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(32 * h);
    const uint32_t a_s = smem_addr(Aop), b16 = smem_addr(Bop), b32 = b16 + (uint32_t)kBbytes;
    constexpr uint32_t idesc16 = umma_idesc_f16(128, 32, BF16), idesc32 = umma_idesc_f16(128, 64, BF16);
    uint32_t mph = 0;
    auto stage = [&](int kind, int dir, int prefetch) {  // kind 0: radix 16 (two groups), 1: radix 32
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            if (kind == 0) issue_stage16x2(tmem, a_s, b16 + (uint32_t)dir * 3u * kBmat, idesc16);
            else issue_stage32(tmem, a_s, b32 + (uint32_t)dir * 3u * kBmat32, idesc32);
            umma_commit(&mma_bar);
            if (prefetch >= 0) load_tile(prefetch);
        }
        mbar_wait(&mma_bar, mph, red.err, red.wait_limit);
        mph ^= 1u;
        tc_fence_after();
    };

    float d[32];
    for (int c = 0; c < nc; ++c) {
        const float2* S = sbuf + (c & 1) * NY * TX;
        mbar_wait(&full[c & 1], (c >> 1) & 1, red.err, red.wait_limit);
        float2 u[16];
        // stage 1: row (j1, s) holds u[s + 32 e], e < 16
#pragma unroll
        for (int e = 0; e < 16; ++e) u[e] = cscale(cmul(S_at(S, e), pv[e]), scale);
        write16<BF16>(Aop, a1_off, R1, 0, u, ls);
        stage(0, 0, (c >= 1 && c + 1 < nc) ? c + 1 : -1);
        tmem_ld32(t_lane, d);  // T[s][k1], k1 < 16
        // twiddle W_512^{s k1}; row (j1, k1) of stage 2 takes element s
#pragma unroll
        for (int kk = 0; kk < 16; ++kk)
            write_elem_at<BF16>(Aop, a2_off(16 * j1 + kk, s, 0), a2_off(16 * j1 + kk, s, 1),
                                cmul(make_float2(d[2 * kk], d[2 * kk + 1]), tw[32 * kk + s]), ls);
        stage(1, 0, -1);
        tmem_ld32(t_lane, d);  // row (j2, k1): X[k1 + 16 k2], k2 = 16 h + i
#pragma unroll
        for (int i = 0; i < 16; ++i) u[i] = cscale(make_float2(d[2 * i], d[2 * i + 1]), mk[k1 + 16 * (16 * h + i)]);
        write16<BF16>(Aop, a2_off, r, 16 * h, u, ls);
        stage(1, 1, -1);
        tmem_ld32(t_lane, d);  // row (j2, k1): T'[s'][k1], s' = 16 h + i
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int s2 = 16 * h + i;
            write_elem_at<BF16>(Aop, a1_off(32 * j2 + s2, k1, 0), a1_off(32 * j2 + s2, k1, 1),
                                cmulc(tw[32 * k1 + s2], make_float2(d[2 * i], d[2 * i + 1])), ls);
        }
        stage(0, 1, -1);
        tmem_ld32(t_lane, d);  // row (j1, s): (F^H R F u)[s + 32 e], scaled
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] = cfmac(acc[e], S_at(S, e), make_float2(d[2 * e], d[2 * e + 1]));
    }
    tc_fence_before();
    __syncthreads();
    if (w == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 64);
    }
    float2* pt = sbuf;
#pragma unroll
    for (int e = 0; e < 16; ++e) pt[rbase + e * 32 * TX] = pv[e];
    for (int i = tid; i < NY; i += NT) {
        halo[i] = p[img + (size_t)i * nx + (x0 == 0 ? nx - 1 : x0 - 1)];
        halo[NY + i] = p[img + (size_t)i * nx + (x0 + TX == nx ? 0 : x0 + TX)];
    }
    __syncthreads();
    float dot = 0.f;
    const float mus = mu * unscale;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int y = s + 32 * e;
        const float2 up = pt[swz64(y == 0 ? NY - 1 : y - 1, j1)];
        const float2 dn = pt[swz64(y == NY - 1 ? 0 : y + 1, j1)];
        const float2 lf = j1 > 0 ? pt[swz64(y, j1 - 1)] : halo[y];
        const float2 rt = j1 < TX - 1 ? pt[swz64(y, j1 + 1)] : halo[NY + y];
        const float tvx = 4.f * pv[e].x - up.x - dn.x - lf.x - rt.x;
        const float tvy = 4.f * pv[e].y - up.y - dn.y - lf.y - rt.y;
        float2 o;
        o.x = fmaf(mus, acc[e].x, fmaf(lam, tvx, gam * pv[e].x));
        o.y = fmaf(mus, acc[e].y, fmaf(lam, tvy, gam * pv[e].y));
        q[img + (size_t)y * nx + x] = o;
        dot = fmaf(pv[e].x, o.x, fmaf(pv[e].y, o.y, dot));
    }
    if constexpr (PCG) {
        double v[1] = {(double)dot}, tot[1];
        const int np = gridDim.x;
        if (last_block_total<1>(v, red.part, np, b * np + blockIdx.x, red.counter + b, tot, red_s, &flag) &&
            threadIdx.x == 0) {
            SliceState& S = st[b];
            const double pq = tot[0];
            S.pq = pq;
            if (!isfinite(pq) || !isfinite(S.rho)) {
                S.state = ST_NONFINITE;
            } else if (!(pq > 0.0)) {
                S.state = ST_BREAKDOWN;
            } else {
                S.alpha = S.rho / pq;
                S.iters += 1;
            }
        }
    }
}

constexpr size_t kSmemApplyATc512 = 1024 + 2 * kT5NY * kTcTX * sizeof(float2) + kA5bytes + kB5bytes +
                                    3 * kT5NY * sizeof(float2) + kT5NY * sizeof(float) + 64 * sizeof(double);

constexpr size_t kSmemApplyATc = 1024 + 2 * kTcNY * kTcTX * sizeof(float2) + kAbytes + kBbytes +
                                 3 * kTcNY * sizeof(float2) + kTcNY * sizeof(float) + 64 * sizeof(double);

template <bool BF16>
cudaError_t launch_tc512(const Dims& d, const TcOperands& tc, const float2* p, float2* q, const float* maskw,
                         float mu, float lam, float gam, SliceState* st, Red red, cudaStream_t s) {
    const dim3 grid(d.nx / kTcTX, d.nb);
    cudaError_t e;
    if (st) {
        if ((e = set_smem_limit(k_apply_A_tc512<BF16, true>, (int)kSmemApplyATc512)) != cudaSuccess) return e;
        k_apply_A_tc512<BF16, true><<<grid, kTcNT, kSmemApplyATc512, s>>>(
            *tc.smap8, p, q, maskw, tc.tw, static_cast<const uint4*>(tc.bmat), d.nx, d.nc, mu, lam, gam, st, red);
    } else {
        if ((e = set_smem_limit(k_apply_A_tc512<BF16, false>, (int)kSmemApplyATc512)) != cudaSuccess) return e;
        k_apply_A_tc512<BF16, false><<<grid, kTcNT, kSmemApplyATc512, s>>>(
            *tc.smap8, p, q, maskw, tc.tw, static_cast<const uint4*>(tc.bmat), d.nx, d.nc, mu, lam, gam, st, red);
    }
    return cudaGetLastError();
}

template <bool BF16>
cudaError_t launch_tc(const Dims& d, const TcOperands& tc, const float2* p, float2* q, const float* maskw,
                      float mu, float lam, float gam, SliceState* st, Red red, cudaStream_t s) {
    if (d.ny == kT5NY) return launch_tc512<BF16>(d, tc, p, q, maskw, mu, lam, gam, st, red, s);
    const dim3 grid(d.nx / kTcTX, d.nb);
    cudaError_t e;
    if (st) {
        if ((e = set_smem_limit(k_apply_A_tc<BF16, true>, (int)kSmemApplyATc)) != cudaSuccess) return e;
        k_apply_A_tc<BF16, true><<<grid, kTcNT, kSmemApplyATc, s>>>(*tc.smap8, p, q, maskw, tc.tw,
                                                                    static_cast<const uint4*>(tc.bmat), d.nx, d.nc,
                                                                    mu, lam, gam, st, red);
    } else {
        if ((e = set_smem_limit(k_apply_A_tc<BF16, false>, (int)kSmemApplyATc)) != cudaSuccess) return e;
        k_apply_A_tc<BF16, false><<<grid, kTcNT, kSmemApplyATc, s>>>(*tc.smap8, p, q, maskw, tc.tw,
                                                                     static_cast<const uint4*>(tc.bmat), d.nx,
                                                                     d.nc, mu, lam, gam, st, red);
    }
    return cudaGetLastError();
}

}  // namespace

bool apply_A_tc_supported(const Dims& d) {
    return (d.ny == kTcNY || d.ny == kT5NY) && d.nx % kTcTX == 0 && d.nx >= kTcTX;
}

cudaError_t launch_apply_A_tc(const Dims& d, const TcOperands& tc, const float2* p, float2* q, const float* maskw,
                              float mu, float lam, float gam, SliceState* st, Red red, cudaStream_t s) {
    if (!apply_A_tc_supported(d) || !tc.smap8 || !tc.tw || !tc.bmat) return cudaErrorInvalidValue;
    return tc.bf16 ? launch_tc<true>(d, tc, p, q, maskw, mu, lam, gam, st, red, s)
                   : launch_tc<false>(d, tc, p, q, maskw, mu, lam, gam, st, red, s);
}

// B operands of the split stages: the real form of the scaled n-point DFT matrix (n = 16: 1/4;
// n = 32: 1/sqrt 32), forward then inverse, each as hi, hi * 2^-L and lo, in the core-matrix
// layout (N = K = 2n, K-adjacent core matrices 128 B apart, 8-row groups 32 n B apart).
namespace {
void build_dft_block(bool bf16, int n, double scale, uint16_t* img) {
    const double L = bf16 ? 1.0 : 1.0 / 1024.0;
    const size_t per = (size_t)(2 * n) * (2 * n);  // elements per matrix
    const size_t sbo = 32 * (size_t)n;            // bytes between 8-row groups: 2n / 8 core matrices of 128 B
    for (int dir = 0; dir < 2; ++dir) {
        for (int nn = 0; nn < 2 * n; ++nn) {
            for (int k = 0; k < 2 * n; ++k) {
                const int ko = nn >> 1, e = k >> 1;
                const double th = (dir == 0 ? -2.0 : 2.0) * M_PI * (double)((ko * e) % n) / (double)n;
                const double wr = std::cos(th) * scale, wi = std::sin(th) * scale;
                // out_re = a_re wr - a_im wi, out_im = a_re wi + a_im wr
                double v;
                if ((nn & 1) == 0) v = (k & 1) == 0 ? wr : -wi;
                else v = (k & 1) == 0 ? wi : wr;
                uint16_t bh, bh2, bl;
                if (bf16) {
                    const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
                    const float hi = __bfloat162float(h);
                    const __nv_bfloat16 l = __float2bfloat16_rn((float)(v - (double)hi));
                    const __nv_bfloat16 h2 = __float2bfloat16_rn((float)((double)hi * L));
                    bh = *reinterpret_cast<const uint16_t*>(&h);
                    bh2 = *reinterpret_cast<const uint16_t*>(&h2);
                    bl = *reinterpret_cast<const uint16_t*>(&l);
                } else {
                    const __half h = __float2half_rn((float)v);
                    const float hi = __half2float(h);
                    const __half l = __float2half_rn((float)(v - (double)hi));
                    const __half h2 = __float2half_rn((float)((double)hi * L));
                    bh = *reinterpret_cast<const uint16_t*>(&h);
                    bh2 = *reinterpret_cast<const uint16_t*>(&h2);
                    bl = *reinterpret_cast<const uint16_t*>(&l);
                }
                const size_t off = ((size_t)(nn >> 3) * sbo + (size_t)(k >> 3) * kLboB + (nn & 7) * 16 + (k & 7) * 2) / 2;
                img[(dir * 3 + 0) * per + off] = bh;
                img[(dir * 3 + 1) * per + off] = bh2;
                img[(dir * 3 + 2) * per + off] = bl;
            }
        }
    }
}
}  // namespace

void build_tc_bmat(bool bf16, uint16_t* img) {
    for (int i = 0; i < kB5bytes / 2; ++i) img[i] = 0;
    build_dft_block(bf16, 16, 0.25, img);
    build_dft_block(bf16, 32, 1.0 / std::sqrt(32.0), img + kBbytes / 2);
}

size_t tc_bmat_bytes() { return kB5bytes; }

}  // namespace sb
