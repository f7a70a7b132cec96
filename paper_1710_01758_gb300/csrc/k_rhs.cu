// Right-hand side of Eq. system (step 4 of Algorithm 1) fused with the outer data update
// (steps 12-14) and the initial PCG residual.
//
// Per column tile of one slice and per coil c (yt = F_x^H y on the sampled lines, see k_sb.cu):
//   u   = R_y F_y (S_c x)                      forward DFT along y, kept on sampled lines
//   yt  = yt + yt1 - u                         outer update (ADDBACK), written back
//   e  += S_c^H F_y^H (yt - u)                 inverse DFT: data term of b - A x
// With B(y) = sum_c S_c^H F^H R y_c (linear) the data term of b is bd = B(y^[j]); the outer
// update y^[j+1] = y^[j] + y^[1] - R F S x gives bd' = bd + bd1 - B(R F S x), and the pass
// computes e = bd' - B(R F S x), so bd' = (e + bd + bd1) / 2 exactly, without a second
// inverse transform per coil.  Then b = mu bd' + g, r = mu e + g - lambda D^H D x - gamma x,
// with ||b||^2, ||r||^2 and the initial convergence test in the last CTA of the slice.  The
// coil tile S_c and the compact rows of yt and yt1 arrive by TMA into a shared-memory stage
// (the load of coil c + 1 is issued as soon as coil c has left the stage; the second CTA on
// the SM computes meanwhile).
#include "common.cuh"
#include "kernels.h"
#include "tiles.cuh"
#include "tma.cuh"
#include "umma.cuh"

namespace sb {
namespace {

constexpr int TX = kColTile;

struct ColIdx {
    int col;
    __device__ __forceinline__ int operator()(int pos) const { return pos * TX + col; }
};

// one pipeline stage: ~95 KB of shared memory at ny = 256 lets two CTAs share an SM, which
// hides the coil-tile loads better than a second stage at one CTA per SM (measured: 125 us
// against 173 us per 16-slice launch inside the benchmark)
template <int NY>
constexpr int kRhsStages = 1;

template <int NY, bool ADDBACK>
__global__ void __launch_bounds__(TX * NY / 16, is_pow2(NY) && NY <= 256 ? 2 : 1)
k_rhs(const __grid_constant__ CUtensorMap smap, const __grid_constant__ CUtensorMap ymap,
      const __grid_constant__ CUtensorMap y1map, SbFields f, int nx, int nc, const float2* __restrict__ xin,
      float2* __restrict__ r, const float2* __restrict__ tw_g, float mu, float lam, float gam, SliceState* st,
      double tol2, Red red) {
    constexpr int T = NY / 16;
    constexpr int NT = TX * T;
    constexpr int NST = kRhsStages<NY>;
    constexpr int SBOX = coil_box_rows(NY);  // rows per TMA box of a coil tile
    const int b = blockIdx.y;
    const int ms = f.ms;  // <= 256: one box of compact rows
    const uint32_t sbytes = NY * TX * sizeof(float2);
    const uint32_t ybytes = ms * TX * sizeof(float2);
    const uint32_t stage_bytes = sbytes + (ADDBACK ? 2u : 1u) * ybytes;
    const int stage_elems = (NY + 2 * ms) * TX;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* stages = reinterpret_cast<float2*>(smem);  // [NST][S tile | yt rows | yt1 rows]
    float2* xbuf = stages + NST * stage_elems;          // FFT exchange, then the x tile
    float2* xbuf2 = xbuf + NY * TX;                     // mixed-radix sizes: out-of-place stages
    float2* tw = xbuf2 + (is_pow2(NY) ? 0 : NY * TX);
    float2* halo = tw + NY;
    int* sl = reinterpret_cast<int*>(halo + 2 * NY);
    double* red_s = reinterpret_cast<double*>(sl + NY);
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int flag;

    const int tid = threadIdx.x, col = tid % TX, t = tid / TX;
    const int x0 = blockIdx.x * TX, xg = x0 + col;
    auto issue = [&](int c, int stage) {
        float2* dst = stages + stage * stage_elems;
        mbar_arrive_expect_tx(&bars[stage], stage_bytes);
#pragma unroll
        for (int r0 = 0; r0 < NY; r0 += SBOX) tma_load_2d(dst + r0 * TX, &smap, 2 * x0, (b * nc + c) * NY + r0, &bars[stage]);
        tma_load_2d(dst + NY * TX, &ymap, 2 * x0, (b * nc + c) * ms, &bars[stage]);
        if (ADDBACK) tma_load_2d(dst + (NY + ms) * TX, &y1map, 2 * x0, (b * nc + c) * ms, &bars[stage]);
    };
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init_fence();
    }
    __syncthreads();
    // kRedWithholdCoilTiles: no tile is requested, so the waits below run out (nothing in flight)
    const bool loads = !(red.flags & kRedWithholdCoilTiles);
    if (tid == 0 && loads)
        for (int c = 0; c < NST && c < nc; ++c) issue(c, c);
    for (int i = tid; i < NY; i += NT) {
        tw[i] = tw_g[i];
        sl[i] = f.slot[(size_t)b * NY + i];
    }
    const size_t img = (size_t)b * NY * nx;
    float2 xv[16], racc[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        xv[e] = xin[img + (size_t)(t + T * e) * nx + xg];
        racc[e] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    const ColIdx idx{col};
    const float sc = rsqrtf((float)NY);
    for (int c = 0; c < nc; ++c) {
        const int stage = c % NST;
        mbar_wait(&bars[stage], (c / NST) & 1, red.err, red.wait_limit);
        const float2* S = stages + stage * stage_elems;
        const float2* Yt = S + NY * TX;
        const float2* Y1 = Yt + ms * TX;
        const size_t ybase = ((size_t)b * nc + c) * ms * nx;
        float2 u[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) u[e] = cmul(S[idx(t + T * e)], xv[e]);
        fft_bar2<NY, false>(u, t, xbuf, xbuf2, idx, tw, CtaBar{});
        // on sampled lines: tt = R F S x (unitary scale), yv = y^[j] after the outer update,
        // u <- yv - tt; zero elsewhere
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int s = sl[t + T * e];
            if (s >= 0) {
                const float2 tt = cscale(u[e], sc);
                float2 yv = Yt[s * TX + col];
                if (ADDBACK) {
                    yv = csub(cadd(yv, Y1[s * TX + col]), tt);
                    f.yt[ybase + (size_t)s * nx + xg] = yv;
                }
                u[e] = csub(yv, tt);
            } else {
                u[e] = make_float2(0.f, 0.f);
            }
        }
        __syncthreads();
        fft_bar2<NY, true>(u, t, xbuf, xbuf2, idx, tw, CtaBar{});
#pragma unroll
        for (int e = 0; e < 16; ++e) racc[e] = cfmac(racc[e], S[idx(t + T * e)], cscale(u[e], sc));
        __syncthreads();  // this stage's tiles and xbuf are free
        if (tid == 0 && loads && c + NST < nc) issue(c + NST, stage);
    }
    // bd' = (racc + bd + bd1) / 2 after an outer update (else bd' = bd);
    // b = mu bd' + g ;  r = mu racc + g - lam D^H D x - gam x
#pragma unroll
    for (int e = 0; e < 16; ++e) xbuf[idx(t + T * e)] = xv[e];
    for (int i = tid; i < NY; i += NT) {
        halo[i] = xin[img + (size_t)i * nx + (x0 == 0 ? nx - 1 : x0 - 1)];
        halo[NY + i] = xin[img + (size_t)i * nx + (x0 + TX == nx ? 0 : x0 + TX)];
    }
    __syncthreads();
    float bb = 0.f, rr = 0.f;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int yy = t + T * e;
        const size_t gi = img + (size_t)yy * nx + xg;
        const float2 gv = f.g[gi];
        const float2 up = xbuf[idx(yy == 0 ? NY - 1 : yy - 1)];
        const float2 dn = xbuf[idx(yy == NY - 1 ? 0 : yy + 1)];
        const float2 lf = col > 0 ? xbuf[idx(yy) - 1] : halo[yy];
        const float2 rt = col < TX - 1 ? xbuf[idx(yy) + 1] : halo[NY + yy];
        const float tvx = 4.f * xv[e].x - up.x - dn.x - lf.x - rt.x;
        const float tvy = 4.f * xv[e].y - up.y - dn.y - lf.y - rt.y;
        float2 bdv = f.bd[gi];
        if (ADDBACK) {
            const float2 b1 = f.bd1[gi];
            bdv = make_float2(0.5f * (racc[e].x + bdv.x + b1.x), 0.5f * (racc[e].y + bdv.y + b1.y));
            f.bd[gi] = bdv;
        }
        const float2 bvec = make_float2(fmaf(mu, bdv.x, gv.x), fmaf(mu, bdv.y, gv.y));
        float2 rv;
        rv.x = fmaf(mu, racc[e].x, gv.x) - fmaf(lam, tvx, gam * xv[e].x);
        rv.y = fmaf(mu, racc[e].y, gv.y) - fmaf(lam, tvy, gam * xv[e].y);
        r[gi] = rv;
        bb += cabs2(bvec);
        rr += cabs2(rv);
    }
    double vv[2] = {(double)bb, (double)rr}, tot[2];
    const int np = gridDim.x;
    if (last_block_total<2>(vv, red.part, np, b * np + blockIdx.x, red.counter + b, tot, red_s, &flag) &&
        threadIdx.x == 0) {
        SliceState& S = st[b];
        S.bnorm2 = tot[0];
        S.rnorm2 = tot[1];
        S.iters = 0;
        S.rho = S.alpha = S.beta = S.pq = 0.0;
        if (!isfinite(tot[0]) || !isfinite(tot[1])) S.state = ST_NONFINITE;
        else if (tot[0] == 0.0) S.state = ST_ZERO;
        else if (tot[1] <= tol2 * tot[0]) S.state = ST_DONE;
        else S.state = ST_ACTIVE;
    }
}

// ---------------------------------------------------------------- 256 and 512 rows: k_rhs8
// The same pass for ny = 256 and 512 in the layout of k_apply_A8 (k_applyA.cu): 8 columns per
// CTA, ny / 16 threads per column (128 threads at 256 rows: a warp holds two whole columns, 16
// rows x 2 columns; 256 threads at 512 rows: a warp is one column), so the transforms' exchanges
// are warp-local; x, the data-term accumulator and the coil's sensitivities (between the forward
// product and the conjugate product) live in tensor memory (128 columns per CTA at 256 rows, 256
// at 512), and the thread's 15 stage-2 twiddles W_256^{r (t mod 16)} in the registers that this
// frees; the coil tile and the compact k-space rows (yt, yt1) arrive by TMA with the 64-byte
// swizzle into one stage each, released as soon as every warp has read them (the sensitivities
// into registers at the start of the coil, the k-space rows after the forward transform) and
// refilled at once by the last warp to release them.  Between the transforms a warp handles the
// sampled lines of its columns densely (its lanes over the compact slots, through the exchange
// region) instead of each thread testing its own 16 rows, which left most lanes idle on every
// row.  The epilogue's rows of g, bd and bd1 are prefetched into L2 during the last coil.
constexpr int TX8 = 8;
using tiles::ExIdx;

__device__ __forceinline__ int swz64(int row, int col) {
    return row * TX8 + ((((col >> 1) ^ ((row >> 1) & 3)) << 1) | (col & 1));
}
__device__ __forceinline__ uint32_t pad_to_512(const void* p) { return (512u - (smem_addr(p) & 511u)) & 511u; }
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// rows of the k-space stage reserved for yt (rounded up to 8 rows so that yt1 starts on a
// 512-byte boundary, as the 64-byte swizzle requires)
__host__ __device__ constexpr int ms_rows8(int ms) { return (ms + 7) & ~7; }

size_t rhs8_smem_bytes(int ny, int ms) {
    const size_t stride = ny == 512 ? ExIdx<512>::kStride : ExIdx<256>::kStride;
    return 512 + ((size_t)ny * TX8 + 2 * (size_t)ms_rows8(ms) * TX8 + stride * TX8 + ny) * sizeof(float2) +
           2 * (size_t)ny * sizeof(int) + 32 * sizeof(double);
}

template <int NY, bool ADDBACK>
__global__ void __launch_bounds__(TX8 * NY / 16, NY == 256 ? 4 : 2)
k_rhs8(const __grid_constant__ CUtensorMap smap8, const __grid_constant__ CUtensorMap ymap8,
       const __grid_constant__ CUtensorMap y1map8, SbFields f, int nx, int nc, const float2* __restrict__ xin,
       float2* __restrict__ r, const float2* __restrict__ tw_g, float mu, float lam, float gam, SliceState* st,
       double tol2, Red red) {
    static_assert(NY == 256 || NY == 512, "16 or 32 threads per column");
    // T = 16: a warp = 16 rows x 2 columns; T = 32: a warp = one column
    constexpr int T = NY / 16, NT = TX8 * T, NW = NT / 32, CPW = 32 / T;
    constexpr uint32_t kTmemCols = NY == 512 ? 256 : 128;
    const int b = blockIdx.y;
    const int ms = f.ms;
    const int msr = ms_rows8(ms);
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + pad_to_512(smem_raw);
    float2* sA = reinterpret_cast<float2*>(smem);  // [NY][8] coil tile; the x tile in the epilogue
    float2* sB = sA + NY * TX8;                      // [msr][8] yt rows, then [msr][8] yt1 rows
    float2* xbuf = sB + 2 * msr * TX8;               // [8][ExIdx::kStride] exchanges; halo in the epilogue
    float2* tw = xbuf + ExIdx<NY>::kStride * TX8;
    int* sl = reinterpret_cast<int*>(tw + NY);  // [NY] slot of each row (-1: not sampled)
    int* ln = sl + NY;                          // [ms] line of each slot
    double* red_s = reinterpret_cast<double*>(ln + NY);
    __shared__ __align__(8) uint64_t fullA, emptyA, fullB, emptyB;
    __shared__ uint32_t tmem_s;
    __shared__ unsigned ticketA, ticketB;
    __shared__ int flag;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int t = T == 16 ? (lane & 7) + 8 * (lane >> 4) : lane;
    const int col = T == 16 ? 2 * w + ((lane >> 3) & 1) : w;
    const int x0 = blockIdx.x * TX8, xg = x0 + col;
    const ExIdx<NY> idx{col * ExIdx<NY>::kStride};
    const int sb0 = swz64(t, col);
    auto gbar = []() { __syncwarp(); };
    const bool loads = !(red.flags & kRedWithholdCoilTiles);
    auto load_S = [&](int c) {
        mbar_arrive_expect_tx(&fullA, NY * TX8 * sizeof(float2));
#pragma unroll
        for (int r0 = 0; r0 < NY; r0 += 256)  // a TMA box spans at most 256 rows
            tma_load_2d(sA + r0 * TX8, &smap8, 2 * x0, (b * nc + c) * NY + r0, &fullA);
    };
    auto load_Y = [&](int c) {
        mbar_arrive_expect_tx(&fullB, (ADDBACK ? 2u : 1u) * (uint32_t)ms * TX8 * sizeof(float2));
        tma_load_2d(sB, &ymap8, 2 * x0, (b * nc + c) * ms, &fullB);
        if (ADDBACK) tma_load_2d(sB + msr * TX8, &y1map8, 2 * x0, (b * nc + c) * ms, &fullB);
    };

    if (w == 0) tmem_alloc(&tmem_s, kTmemCols);
    if (tid == 0) {
        mbar_init(&fullA, 1);
        mbar_init(&emptyA, NW);
        mbar_init(&fullB, 1);
        mbar_init(&emptyB, NW);
        ticketA = ticketB = 0;
        mbar_init_fence();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && loads) {
        load_S(0);
        load_Y(0);
    }
    // this warp's TMEM lanes 32 (w mod 4) .. +31; columns 96 (w / 4) + 0-31 hold x, + 32-63 the
    // data-term accumulator, + 64-95 S
    const uint32_t t_x = tmem_s + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(96 * (w >> 2));
    const uint32_t t_acc = t_x + 32, t_sv = t_x + 64;
    for (int i = tid; i < NY; i += NT) {
        tw[i] = tw_g[i];
        sl[i] = f.slot[(size_t)b * NY + i];
    }
    for (int i = tid; i < ms; i += NT) ln[i] = f.lines[(size_t)b * ms + i];
    const size_t img = (size_t)b * NY * nx;
    {
        float v[32];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const float2 xv = xin[img + (size_t)(t + T * e) * nx + xg];
            v[2 * e] = xv.x;
            v[2 * e + 1] = xv.y;
        }
        tmem_st32(t_x, v);
    }
    __syncthreads();
    uint32_t mb = 0;  // which of this thread's rows t + T e are sampled
#pragma unroll
    for (int e = 0; e < 16; ++e) mb |= (sl[t + T * e] >= 0 ? 1u : 0u) << e;
    const float sc = rsqrtf((float)NY);
    float2 twr[15];
#pragma unroll
    for (int r = 1; r < 16; ++r) twr[r - 1] = tw[r * 16 + (t & 15)];
    for (int c = 0; c < nc; ++c) {
        const uint32_t ph = c & 1;
        if (c == nc - 1) {  // the epilogue's rows of g, bd (and bd1) into L2
            for (int i = tid; i < NY * (ADDBACK ? 3 : 2); i += NT) {
                const int a = i / NY, y = i % NY;
                const float2* base = a == 0 ? f.g : (a == 1 ? f.bd : f.bd1);
                prefetch_l2(base + img + (size_t)y * nx + x0);
            }
        }
        mbar_wait(&fullA, ph, red.err, red.wait_limit);
        __syncwarp();
        uint32_t xr[32];
        if (c == 0) tmem_wait_st();
        tmem_ld32_issue(t_x, xr);
        float2 sv[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) sv[e] = sA[sb0 + e * T * TX8];
        __syncwarp();
        if (lane == 0) {  // this warp is done with the coil tile; the last warp refills it
            mbar_arrive(&emptyA);
            if (atomicAdd(&ticketA, 1u) % NW == NW - 1 && c + 1 < nc) {
                mbar_wait(&emptyA, ph, red.err, red.wait_limit);
                if (loads) load_S(c + 1);
            }
        }
        __syncwarp();
        tmem_ld_wait(xr);
        float2 u[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) u[e] = cmul(sv[e], make_float2(__uint_as_float(xr[2 * e]), __uint_as_float(xr[2 * e + 1])));
        {
            float v[32];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                v[2 * e] = sv[e].x;
                v[2 * e + 1] = sv[e].y;
            }
            tmem_st32(t_sv, v);
        }
        if constexpr (NY == 256) fft256_bar_rtw<false>(u, t, xbuf, idx, twr, gbar);
        else fft512_bar_rtw<false>(u, t, xbuf, idx, tw, twr, gbar);
        // on sampled lines: tt = R F S x (unitary scale), yv = y^[j] after the outer update,
        // u <- yv - tt; zero elsewhere.  The warp's columns go through the exchange region: every
        // thread stores its 16 values, the lanes then walk the compact slots of the warp's columns
        // (T = 16, two columns: lane l serves column 2 w + (l & 1), slots l / 2 + 16 i; T = 32:
        // slots l + 32 i of column w), and every thread reads its rows back.
        gbar();  // the forward transform's exchange reads are done
#pragma unroll
        for (int e = 0; e < 16; ++e) xbuf[idx(t + T * e)] = u[e];
        mbar_wait(&fullB, ph, red.err, red.wait_limit);
        __syncwarp();
        {
            const float2* Yt = sB;
            const float2* Y1 = sB + msr * TX8;
            const size_t ybase = ((size_t)b * nc + c) * ms * nx;
            const int cc = CPW == 2 ? 2 * w + (lane & 1) : w;  // the column this lane serves in the walk
            const ExIdx<NY> cidx{cc * ExIdx<NY>::kStride};
            for (int s = lane / CPW; s < ms; s += 32 / CPW) {
                const int yrow = ln[s];
                const float2 tt = cscale(xbuf[cidx(yrow)], sc);
                float2 yv = Yt[swz64(s, cc)];
                if (ADDBACK) {
                    yv = csub(cadd(yv, Y1[swz64(s, cc)]), tt);
                    f.yt[ybase + (size_t)s * nx + x0 + cc] = yv;
                }
                xbuf[cidx(yrow)] = csub(yv, tt);
            }
        }
        __syncwarp();
#pragma unroll
        for (int e = 0; e < 16; ++e)
            u[e] = ((mb >> e) & 1u) ? xbuf[idx(t + T * e)] : make_float2(0.f, 0.f);
        __syncwarp();
        if (lane == 0) {  // ... and with the k-space rows
            mbar_arrive(&emptyB);
            if (atomicAdd(&ticketB, 1u) % NW == NW - 1 && c + 1 < nc) {
                mbar_wait(&emptyB, ph, red.err, red.wait_limit);
                if (loads) load_Y(c + 1);
            }
        }
        gbar();
        if constexpr (NY == 256) fft256_bar_rtw<true>(u, t, xbuf, idx, twr, gbar);
        else fft512_bar_rtw<true>(u, t, xbuf, idx, tw, twr, gbar);
        // racc += conj(S) (sc u), in two halves of 8 values
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float a[16], s16[16];
            uint32_t ra[16], rs[16];
            tmem_wait_st();
            tmem_ld16_issue(t_sv + 16 * h, rs);
            if (c > 0) tmem_ld16_issue(t_acc + 16 * h, ra);
            else
#pragma unroll
                for (int i = 0; i < 16; ++i) ra[i] = 0u;
            tmem_ld_wait2(ra, rs);
#pragma unroll
            for (int i = 0; i < 16; ++i) s16[i] = __uint_as_float(rs[i]);
            if (c > 0) {
#pragma unroll
                for (int i = 0; i < 16; ++i) a[i] = __uint_as_float(ra[i]);
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) a[i] = 0.f;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float2 rr = cfmac(make_float2(a[2 * i], a[2 * i + 1]), make_float2(s16[2 * i], s16[2 * i + 1]), cscale(u[8 * h + i], sc));
                a[2 * i] = rr.x;
                a[2 * i + 1] = rr.y;
            }
            tmem_st16(t_acc + 16 * h, a);
        }
        gbar();
    }
    // bd' = (racc + bd + bd1) / 2 after an outer update (else bd' = bd);
    // b = mu bd' + g ;  r = mu racc + g - lam D^H D x - gam x
    __syncthreads();  // the stages and the exchange regions are free
    float2 xv[16], racc[16];
    {
        float v[32];
        tmem_wait_st();
        tmem_ld32(t_x, v);
#pragma unroll
        for (int e = 0; e < 16; ++e) xv[e] = make_float2(v[2 * e], v[2 * e + 1]);
        tmem_ld32(t_acc, v);
#pragma unroll
        for (int e = 0; e < 16; ++e) racc[e] = make_float2(v[2 * e], v[2 * e + 1]);
    }
    float2* xt = sA;
    float2* halo = xbuf;  // [2][NY]: columns x0-1 and x0+8
#pragma unroll
    for (int e = 0; e < 16; ++e) xt[sb0 + e * T * TX8] = xv[e];
    for (int i = tid; i < NY; i += NT) {
        halo[i] = xin[img + (size_t)i * nx + (x0 == 0 ? nx - 1 : x0 - 1)];
        halo[NY + i] = xin[img + (size_t)i * nx + (x0 + TX8 == nx ? 0 : x0 + TX8)];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (w == 0) tmem_dealloc(tmem_s, kTmemCols);
    float bb = 0.f, rr = 0.f;
    // the rows' g, bd (and bd1) loads are issued EC rows at a time: in one loop with the stores
    // of bd and r they could not be moved above the previous row's stores (the arrays may alias
    // as far as the compiler knows), and each row would wait for its loads in turn; 8 rows spill
    constexpr int EC = 4;
#pragma unroll
    for (int e0 = 0; e0 < 16; e0 += EC) {
        float2 gq[EC], bq[EC], b1q[EC];
#pragma unroll
        for (int k = 0; k < EC; ++k) {
            const size_t gi = img + (size_t)(t + T * (e0 + k)) * nx + xg;
            gq[k] = f.g[gi];
            bq[k] = f.bd[gi];
            if (ADDBACK) b1q[k] = f.bd1[gi];
        }
#pragma unroll
        for (int k = 0; k < EC; ++k) {
            const int e = e0 + k;
            const int yy = t + T * e;
            const size_t gi = img + (size_t)yy * nx + xg;
            const float2 gv = gq[k];
            const float2 up = xt[swz64(yy == 0 ? NY - 1 : yy - 1, col)];
            const float2 dn = xt[swz64(yy == NY - 1 ? 0 : yy + 1, col)];
            const float2 lf = col > 0 ? xt[swz64(yy, col - 1)] : halo[yy];
            const float2 rt = col < TX8 - 1 ? xt[swz64(yy, col + 1)] : halo[NY + yy];
            const float tvx = 4.f * xv[e].x - up.x - dn.x - lf.x - rt.x;
            const float tvy = 4.f * xv[e].y - up.y - dn.y - lf.y - rt.y;
            float2 bdv = bq[k];
            if (ADDBACK) {
                const float2 b1 = b1q[k];
                bdv = make_float2(0.5f * (racc[e].x + bdv.x + b1.x), 0.5f * (racc[e].y + bdv.y + b1.y));
                f.bd[gi] = bdv;
            }
            const float2 bvec = make_float2(fmaf(mu, bdv.x, gv.x), fmaf(mu, bdv.y, gv.y));
            float2 rv;
            rv.x = fmaf(mu, racc[e].x, gv.x) - fmaf(lam, tvx, gam * xv[e].x);
            rv.y = fmaf(mu, racc[e].y, gv.y) - fmaf(lam, tvy, gam * xv[e].y);
            r[gi] = rv;
            bb += cabs2(bvec);
            rr += cabs2(rv);
        }
    }
    double vv[2] = {(double)bb, (double)rr}, tot[2];
    const int np = gridDim.x;
    if (last_block_total<2>(vv, red.part, np, b * np + blockIdx.x, red.counter + b, tot, red_s, &flag) &&
        threadIdx.x == 0) {
        SliceState& S = st[b];
        S.bnorm2 = tot[0];
        S.rnorm2 = tot[1];
        S.iters = 0;
        S.rho = S.alpha = S.beta = S.pq = 0.0;
        if (!isfinite(tot[0]) || !isfinite(tot[1])) S.state = ST_NONFINITE;
        else if (tot[0] == 0.0) S.state = ST_ZERO;
        else if (tot[1] <= tol2 * tot[0]) S.state = ST_DONE;
        else S.state = ST_ACTIVE;
    }
}

template <int NY, bool AB>
cudaError_t rhs8(const Dims& d, const RhsMaps& m, const SbFields& f, const float2* x, float2* r, const float2* tw,
                 float mu, float lam, float gam, SliceState* st, double tol2, Red red, cudaStream_t s) {
    const size_t sm = rhs8_smem_bytes(NY, f.ms);
    // the fixed maximum (see rhs_n)
    cudaError_t e = set_smem_limit(k_rhs8<NY, AB>, (int)rhs8_smem_bytes(NY, 256));
    if (e != cudaSuccess) return e;
    k_rhs8<NY, AB><<<dim3(d.nx / TX8, d.nb), TX8 * NY / 16, sm, s>>>(*m.smap8, *m.ymap8, *m.y1map8, f, d.nx, d.nc, x,
                                                                    r, tw, mu, lam, gam, st, tol2, red);
    return cudaGetLastError();
}

template <int NY, bool AB>
cudaError_t rhs_n(const Dims& d, const CUtensorMap& smap, const CUtensorMap& ymap, const CUtensorMap& y1map,
                  const SbFields& f, const float2* x, float2* r, const float2* tw, float mu, float lam, float gam,
                  SliceState* st, double tol2, Red red, cudaStream_t s) {
    const size_t sm = rhs_smem_bytes(NY, f.ms);
    // the limit is shared by all host threads (concurrent plans differ in ms): set it to the size
    // of the largest ms the library accepts (256), never to this launch's own size
    cudaError_t e = set_smem_limit(k_rhs<NY, AB>, (int)rhs_smem_bytes(NY, 256));
    if (e != cudaSuccess) return e;
    k_rhs<NY, AB><<<dim3(d.nx / TX, d.nb), TX * NY / 16, sm, s>>>(smap, ymap, y1map, f, d.nx, d.nc, x, r, tw, mu,
                                                                   lam, gam, st, tol2, red);
    return cudaGetLastError();
}

}  // namespace

size_t rhs_smem_bytes(int ny, int ms) {
    if (ny == 256 || ny == 512) return rhs8_smem_bytes(ny, ms);
    const size_t nst = 1;
    const size_t xbufs = is_pow2(ny) ? 1 : 2;  // exchange regions (two for the out-of-place mixed-radix stages)
    return (nst * (size_t)(ny + 2 * ms) * TX + xbufs * (size_t)ny * TX + 3 * (size_t)ny) * sizeof(float2) +
           ny * sizeof(int) + 64 * sizeof(double);
}

cudaError_t launch_rhs(const Dims& d, const RhsMaps& m, const SbFields& f, int addback, const float2* x, float2* r,
                       const float2* tw_y, float mu, float lam, float gam, SliceState* st, double tol2, Red red,
                       cudaStream_t s) {
    const CUtensorMap &smap = *m.smap, &ymap = *m.ymap, &y1map = *m.y1map;
#define CALL(N)                                                                                        \
    return addback ? rhs_n<N, true>(d, smap, ymap, y1map, f, x, r, tw_y, mu, lam, gam, st, tol2, red, s) \
                   : rhs_n<N, false>(d, smap, ymap, y1map, f, x, r, tw_y, mu, lam, gam, st, tol2, red, s);
    switch (d.ny) {
        case 32: CALL(32)
        case 64: CALL(64)
        case 128: CALL(128)
        case 256:
            return addback ? rhs8<256, true>(d, m, f, x, r, tw_y, mu, lam, gam, st, tol2, red, s)
                           : rhs8<256, false>(d, m, f, x, r, tw_y, mu, lam, gam, st, tol2, red, s);
        case 512:
            return addback ? rhs8<512, true>(d, m, f, x, r, tw_y, mu, lam, gam, st, tol2, red, s)
                           : rhs8<512, false>(d, m, f, x, r, tw_y, mu, lam, gam, st, tol2, red, s);
        case 192: CALL(192)
        case 224: CALL(224)
        case 320: CALL(320)
        case 384: CALL(384)
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

}  // namespace sb
