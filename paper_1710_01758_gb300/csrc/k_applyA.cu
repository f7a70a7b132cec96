// q = A p (Eq. system) for a batch of slices, with the readout-axis shortcut of the data term:
// a mask constant along x gives F^H R F = (F_y^H R_y F_y) (x) I_x, so each coil needs one
// length-ny DFT along y, the mask, and one inverse DFT per column.
//
// One CTA owns TX = 16 full columns of one slice and loops over the coils:
//   u = S_c p  ->  DFT_y  ->  r_y / ny  ->  IDFT_y  ->  acc += conj(S_c) u,
// then adds the periodic TV stencil lambda (D_x^H D_x + D_y^H D_y) p and gamma p, stores q and
// (PCG mode) accumulates Re(p^H q) and sets alpha = rho / p^H q in the last CTA of the slice.
//
// Layout of the work:
//  * Coil tiles S_c[:, x0:x0+16] (ny x 128 B) arrive by TMA with the 128-byte swizzle into a
//    two-stage ring; a "full" mbarrier per stage completes on the bytes, an "empty" mbarrier
//    (one arrival per warp) tells the producing thread when the stage may be refilled.
//  * Each column transform belongs to ny / 16 threads of one exchange group (64 threads for
//    ny <= 256, 128 at ny = 512, whole warps of whole columns for ny = 16 x {12, 14, 20, 24});
//    a group owns CPG columns, exchanges data only through its private shared-memory region,
//    and synchronises with a named barrier of its own: no CTA-wide barrier inside the coil
//    loop (one group per CTA at ny = 224).  At ny = 256 a warp holds two whole columns (16 rows
//    x 2 columns; each half-warp 8 rows x 2 columns), and at ny = 128 four, so there the
//    exchanges are ordered by __syncwarp alone.
//  * 8-byte shared-memory accesses are served per half-warp, so each half-warp holds 8
//    consecutive rows of 2 adjacent columns: the TMA swizzle then spreads the tile reads over
//    16 distinct bank pairs, and so does the exchange region, stored column by column with one
//    pad slot per 16 positions and a column stride of 8 (mod 16) slots.
#include "common.cuh"
#include "kernels.h"
#include "tiles.cuh"
#include "tma.cuh"
#include "umma.cuh"

namespace sb {
namespace {

using tiles::ExIdx;
using tiles::pad_to_1024;
using tiles::swz;
using tiles::TileRows;
constexpr int TX = kColTile;

// rows of one TMA box (the box extent is limited to 256 per dimension)
template <int NY>
constexpr int kBoxRows = coil_box_rows(NY);

// issue the TMA loads of coil tile (slice b, coil c) into `dst`, completing on `bar`
template <int NY>
__device__ __forceinline__ void load_coil_tile(float2* dst, const CUtensorMap* map, int x0, int b, int nc, int c,
                                               uint64_t* bar) {
    mbar_arrive_expect_tx(bar, NY * TX * sizeof(float2));
#pragma unroll
    for (int r0 = 0; r0 < NY; r0 += kBoxRows<NY>)
        tma_load_2d(dst + r0 * TX, map, 2 * x0, (b * nc + c) * NY + r0, bar);
}

__host__ __device__ constexpr int lcm32(int t) {
    int m = 32;
    while (m % t != 0) m += 32;
    return m;
}

template <int NY, bool PCG>
__global__ void __launch_bounds__(TX * NY / 16, is_pow2(NY) && NY <= 256 ? 2 : 1)
k_apply_A(const __grid_constant__ CUtensorMap smap, const float2* __restrict__ p, float2* __restrict__ q,
          const float* __restrict__ maskw, const float2* __restrict__ tw_g, int nx, int nc, float mu, float lam,
          float gam, SliceState* st, Red red) {
    constexpr int T = NY / 16;            // threads per column transform
    constexpr int NT = TX * T;            // threads per CTA
    // threads per exchange group: 4 columns when T is a multiple of 8 (a warp = 8 rows x 4
    // columns needs T / 8 warps), else the smallest whole number of warps that holds whole
    // columns (lcm(T, 32): 96 threads for T = 12, 224 for 14, 160 for 20)
    constexpr int GT = NT < 64 ? NT : (T % 8 == 0 ? (4 * T > 64 ? 4 * T : 64) : lcm32(T));
    constexpr int CPG = GT / T;           // columns per group
    constexpr int NW = NT / 32;           // warps per CTA
    const int b = blockIdx.y;
    if (PCG && st[b].state != ST_ACTIVE) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + pad_to_1024(smem_raw);
    float2* sbuf = reinterpret_cast<float2*>(smem);  // [2][NY * TX] swizzled coil tiles
    float2* xbuf = sbuf + 2 * NY * TX;                // [TX][ExIdx::kStride] exchange regions
    // mixed-radix sizes: a second set of exchange regions for the out-of-place stages
    constexpr int kEx2 = is_pow2(NY) ? 0 : ExIdx<NY>::kStride * TX;
    float2* xbuf2 = xbuf + ExIdx<NY>::kStride * TX;
    float2* tw = xbuf2 + kEx2;
    float2* halo = tw + NY;                           // [2][NY]: columns x0-1 and x0+TX
    float2* mk = halo + 2 * NY;                       // [NY] mask weight w of each row as (w, w)
    double* red_s = reinterpret_cast<double*>(mk + NY);
    __shared__ __align__(8) uint64_t full[2], empty[2];
    __shared__ int flag;

    const int tid = threadIdx.x, lane = tid & 31;
    const int grp = tid / GT, gl = tid % GT;
    // T = 16 and T = 8: every column transform lies within one warp, so the exchanges need only
    // __syncwarp; otherwise a named barrier per exchange group
    constexpr bool kWarpLocal = (T == 16 || T == 8);
    int t, cl, col;
    if constexpr (T == 16) {  // a warp = 16 rows x 2 columns, a half-warp = 8 rows x 2 columns
        t = (lane & 7) + 8 * (lane >> 4);
        cl = (lane >> 3) & 1;
        col = 2 * (tid >> 5) + cl;
    } else if constexpr (T % 8 == 0) {  // a warp = 8 rows x 4 columns; a half-warp = 8 rows x 2 columns
        const int wg = gl >> 5;
        t = (lane & 7) + 8 * (wg % (T / 8));
        cl = (lane >> 3) + 4 * (wg / (T / 8));
        col = grp * CPG + cl;
    } else {
        t = gl / CPG;
        cl = gl % CPG;
        col = grp * CPG + cl;
    }
    const int x0 = blockIdx.x * TX, x = x0 + col;
    const ExIdx<NY> idx{col * ExIdx<NY>::kStride};
    float2* ex = xbuf;
    const TileRows<T> rows(t, col);
    const int bar_id = 1 + grp;
    auto gbar = [bar_id]() {
        if constexpr (kWarpLocal) __syncwarp();
        else named_bar(bar_id, GT);
    };

    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        mbar_init_fence();
    }
    __syncthreads();
    // kRedWithholdCoilTiles: no tile is requested, so the waits below run out (nothing in flight)
    const bool loads = !(red.flags & kRedWithholdCoilTiles);
    if (tid == 0 && loads)
        for (int c = 0; c < 2 && c < nc; ++c) load_coil_tile<NY>(sbuf + c * NY * TX, &smap, x0, b, nc, c, &full[c]);
    for (int i = tid; i < NY; i += NT) {
        tw[i] = tw_g[i];
        const float w = maskw[(size_t)b * NY + i];
        mk[i] = make_float2(w, w);
    }
    const size_t img = (size_t)b * NY * nx;
    float2 pv[16], acc[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        pv[e] = p[img + (size_t)(t + T * e) * nx + x];
        acc[e] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int c = 0; c < nc; ++c) {
        const int stage = c & 1;
        const uint32_t phase = (c >> 1) & 1;
        mbar_wait(&full[stage], phase, red.err, red.wait_limit);
        const float2* S = sbuf + stage * NY * TX;
        float2 u[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) u[e] = cmul(S[rows(e)], pv[e]);
        fft_bar2<NY, false>(u, t, ex, xbuf2, idx, tw, gbar);
#pragma unroll
        for (int e = 0; e < 16; ++e) u[e] = cscale2(u[e], mk[t + T * e]);
        gbar();  // the group's forward reads of ex are done
        fft_bar2<NY, true>(u, t, ex, xbuf2, idx, tw, gbar);
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] = cfmac(acc[e], S[rows(e)], u[e]);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[stage]);  // this warp is done with the stage
        gbar();                                     // ... and the group with ex
        if (tid == 0 && c + 2 < nc) {
            mbar_wait(&empty[stage], phase, red.err, red.wait_limit);
            if (loads) load_coil_tile<NY>(sbuf + stage * NY * TX, &smap, x0, b, nc, c + 2, &full[stage]);
        }
    }
    // periodic 5-point stencil for lambda (D_x^H D_x + D_y^H D_y) p; p tile in stage 0
    __syncthreads();  // every warp left the coil loop: the stage buffers are free
    float2* pt = sbuf;
#pragma unroll
    for (int e = 0; e < 16; ++e) pt[rows(e)] = pv[e];
    for (int i = tid; i < NY; i += NT) {
        halo[i] = p[img + (size_t)i * nx + (x0 == 0 ? nx - 1 : x0 - 1)];
        halo[NY + i] = p[img + (size_t)i * nx + (x0 + TX == nx ? 0 : x0 + TX)];
    }
    __syncthreads();
    float dot = 0.f;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int y = t + T * e;
        const float2 up = pt[swz(y == 0 ? NY - 1 : y - 1, col)];
        const float2 dn = pt[swz(y == NY - 1 ? 0 : y + 1, col)];
        const float2 lf = col > 0 ? pt[swz(y, col - 1)] : halo[y];
        const float2 rt = col < TX - 1 ? pt[swz(y, col + 1)] : halo[NY + y];
        const float tvx = 4.f * pv[e].x - up.x - dn.x - lf.x - rt.x;
        const float tvy = 4.f * pv[e].y - up.y - dn.y - lf.y - rt.y;
        float2 o;
        o.x = fmaf(mu, acc[e].x, fmaf(lam, tvx, gam * pv[e].x));
        o.y = fmaf(mu, acc[e].y, fmaf(lam, tvy, gam * pv[e].y));
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

// ---------------------------------------------------------------- 256 and 512 rows: k_apply_A8
// The same operator for ny = 256 and 512 with the per-thread state moved out of the register
// file, so that more warps fit on an SM (the kernel above holds p, the coil accumulator and the
// transform in 128 registers; at 256 rows two 110 KB CTAs fill an SM, 16 warps, and it is bound by
// issue latency; at 512 rows one CTA of 16 warps spills):
//  * a CTA owns 8 columns, ny / 16 threads per column (128 threads at 256 rows: a warp holds two
//    whole columns, 16 rows x 2 columns; 256 threads at 512 rows: a warp is one column), so the
//    transforms' exchanges are warp-local;
//  * its p values and the coil accumulator live in tensor memory (TMEM, 32-bit columns of the
//    thread's lane; warps w and w + 4 share lanes and take 96-column ranges 96 (w / 4) apart),
//    one tcgen05.ld / tcgen05.st per 16 values; the coil's 16 sensitivities are parked there too
//    between the forward product and the conjugate product (p, accumulator, S: 128 columns per
//    CTA at 256 rows, 256 at 512);
//  * the coil tile (ny rows x 8 columns, 64-byte TMA swizzle) has ONE stage: every thread copies
//    its 16 sensitivities to registers as soon as the tile lands and the stage is refilled with
//    the next coil at once (the last warp to release it issues the TMA), so the load of coil
//    c + 1 overlaps the transforms of coil c.
//  * a thread's 15 stage-2 twiddles W_256^{r (t mod 16)} stay in registers for the whole kernel
//    (30 shared-memory loads fewer per coil), in the registers that parking S frees.
// 256 rows: ~39 KB of shared memory and <= 128 registers, four CTAs (16 warps) per SM, 4 x 128
// TMEM columns; 512 rows: ~77 KB and <= 128 registers, two CTAs (16 warps) per SM, 2 x 256.
constexpr int TX8 = 8;

// float2 index of (row, col) in an 8-column tile written by TMA with the 64-byte swizzle
// (16-byte chunk index XOR (row >> 1) & 3)
__device__ __forceinline__ int swz64(int row, int col) {
    return row * TX8 + ((((col >> 1) ^ ((row >> 1) & 3)) << 1) | (col & 1));
}

// bytes from `p` to the next 512-byte boundary of the shared window (the 64-byte swizzle repeats
// every 512 bytes)
__device__ __forceinline__ uint32_t pad_to_512(const void* p) { return (512u - (smem_addr(p) & 511u)) & 511u; }

template <int NY, bool PCG>
__global__ void __launch_bounds__(TX8 * NY / 16, NY == 256 ? 4 : 2)
k_apply_A8(const __grid_constant__ CUtensorMap smap8, const float2* __restrict__ p, float2* __restrict__ q,
           const float* __restrict__ maskw, const float2* __restrict__ tw_g, int nx, int nc, float mu, float lam,
           float gam, SliceState* st, Red red) {
    static_assert(NY == 256 || NY == 512, "16 or 32 threads per column");
    constexpr int T = NY / 16, NT = TX8 * T, NW = NT / 32;
    constexpr uint32_t kTmemCols = NY == 512 ? 256 : 128;
    const int b = blockIdx.y;
    if (PCG && st[b].state != ST_ACTIVE) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + pad_to_512(smem_raw);
    float2* sbuf = reinterpret_cast<float2*>(smem);  // [NY][8] coil tile; the p tile in the epilogue
    float2* xbuf = sbuf + NY * TX8;                  // [8][ExIdx::kStride] exchanges; halo in the epilogue
    float2* tw = xbuf + ExIdx<NY>::kStride * TX8;
    float2* mk = tw + NY;                            // mask weight w of each row as (w, w)
    double* red_s = reinterpret_cast<double*>(mk + NY);
    __shared__ __align__(8) uint64_t full, empty;
    __shared__ uint32_t tmem_s;
    __shared__ unsigned ticket;
    __shared__ int flag;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    // T = 16: a warp = 16 rows x 2 columns, a half-warp 8 rows x 2 columns; T = 32: a warp = a column
    const int t = T == 16 ? (lane & 7) + 8 * (lane >> 4) : lane;
    const int col = T == 16 ? 2 * w + ((lane >> 3) & 1) : w;
    const int x0 = blockIdx.x * TX8, x = x0 + col;
    const ExIdx<NY> idx{col * ExIdx<NY>::kStride};
    const int sb0 = swz64(t, col);  // rows t + T e share the swizzle term of t
    auto gbar = []() { __syncwarp(); };
    const bool loads = !(red.flags & kRedWithholdCoilTiles);
    auto load_tile = [&](int c) {
        mbar_arrive_expect_tx(&full, NY * TX8 * sizeof(float2));
#pragma unroll
        for (int r0 = 0; r0 < NY; r0 += 256)  // a TMA box spans at most 256 rows
            tma_load_2d(sbuf + r0 * TX8, &smap8, 2 * x0, (b * nc + c) * NY + r0, &full);
    };

    if (w == 0) tmem_alloc(&tmem_s, kTmemCols);
    if (tid == 0) {
        mbar_init(&full, 1);
        mbar_init(&empty, NW);
        ticket = 0;
        mbar_init_fence();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && loads) load_tile(0);
    // this warp's TMEM lanes 32 (w mod 4) .. +31; columns 96 (w / 4) + 0-31 hold p, + 32-63 the
    // accumulator, + 64-95 the coil's sensitivities
    const uint32_t t_pv = tmem_s + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(96 * (w >> 2));
    const uint32_t t_acc = t_pv + 32, t_sv = t_pv + 64;
    for (int i = tid; i < NY; i += NT) {
        tw[i] = tw_g[i];
        const float wt = maskw[(size_t)b * NY + i];
        mk[i] = make_float2(wt, wt);
    }
    const size_t img = (size_t)b * NY * nx;
    {
        float v[32];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const float2 pv = p[img + (size_t)(t + T * e) * nx + x];
            v[2 * e] = pv.x;
            v[2 * e + 1] = pv.y;
        }
        tmem_st32(t_pv, v);
    }
    __syncthreads();
    float2 twr[15];
#pragma unroll
    for (int r = 1; r < 16; ++r) twr[r - 1] = tw[r * 16 + (t & 15)];
    for (int c = 0; c < nc; ++c) {
        const uint32_t ph = c & 1;
        mbar_wait(&full, ph, red.err, red.wait_limit);
        __syncwarp();  // the tcgen05 load below is warp-wide
        uint32_t pr[32];  // p, loaded from TMEM while the sensitivities come from shared memory
        if (c == 0) tmem_wait_st();
        tmem_ld32_issue(t_pv, pr);
        float2 sv[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) sv[e] = sbuf[sb0 + e * T * TX8];
        __syncwarp();
        if (lane == 0) {  // this warp is done with the tile; the last warp refills it
            mbar_arrive(&empty);
            if (atomicAdd(&ticket, 1u) % NW == NW - 1 && c + 1 < nc) {
                mbar_wait(&empty, ph, red.err, red.wait_limit);  // every warp arrived before its ticket
                if (loads) load_tile(c + 1);
            }
        }
        __syncwarp();  // the tcgen05 wait below is warp-wide
        tmem_ld_wait(pr);
        float2 u[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) u[e] = cmul(sv[e], make_float2(__uint_as_float(pr[2 * e]), __uint_as_float(pr[2 * e + 1])));
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
#pragma unroll
        for (int e = 0; e < 16; ++e) u[e] = cscale2(u[e], mk[t + T * e]);
        gbar();  // the warp's forward reads of its exchange region are done
        if constexpr (NY == 256) fft256_bar_rtw<true>(u, t, xbuf, idx, twr, gbar);
        else fft512_bar_rtw<true>(u, t, xbuf, idx, tw, twr, gbar);
        // acc += conj(S) u, in two halves of 8 values (16 TMEM columns each)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float a[16], s16[16];
            tmem_wait_st();
            tmem_ld16(t_sv + 16 * h, s16);
            if (c > 0) {
                tmem_ld16(t_acc + 16 * h, a);
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) a[i] = 0.f;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float2 r = cfmac(make_float2(a[2 * i], a[2 * i + 1]), make_float2(s16[2 * i], s16[2 * i + 1]), u[8 * h + i]);
                a[2 * i] = r.x;
                a[2 * i + 1] = r.y;
            }
            tmem_st16(t_acc + 16 * h, a);
        }
        gbar();  // ... and its inverse reads
    }
    // periodic 5-point stencil for lambda (D_x^H D_x + D_y^H D_y) p; p tile in the stage buffer
    __syncthreads();  // every warp left the coil loop: the stage and the exchange regions are free
    float2 pv[16], acc[16];
    {
        float v[32];
        tmem_wait_st();
        tmem_ld32(t_pv, v);
#pragma unroll
        for (int e = 0; e < 16; ++e) pv[e] = make_float2(v[2 * e], v[2 * e + 1]);
        tmem_ld32(t_acc, v);
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] = make_float2(v[2 * e], v[2 * e + 1]);
    }
    float2* pt = sbuf;
    float2* halo = xbuf;  // [2][NY]: columns x0-1 and x0+8
#pragma unroll
    for (int e = 0; e < 16; ++e) pt[sb0 + e * T * TX8] = pv[e];
    for (int i = tid; i < NY; i += NT) {
        halo[i] = p[img + (size_t)i * nx + (x0 == 0 ? nx - 1 : x0 - 1)];
        halo[NY + i] = p[img + (size_t)i * nx + (x0 + TX8 == nx ? 0 : x0 + TX8)];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (w == 0) tmem_dealloc(tmem_s, kTmemCols);  // every warp's TMEM reads are complete
    float dot = 0.f;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int y = t + T * e;
        const float2 up = pt[swz64(y == 0 ? NY - 1 : y - 1, col)];
        const float2 dn = pt[swz64(y == NY - 1 ? 0 : y + 1, col)];
        const float2 lf = col > 0 ? pt[swz64(y, col - 1)] : halo[y];
        const float2 rt = col < TX8 - 1 ? pt[swz64(y, col + 1)] : halo[NY + y];
        const float tvx = 4.f * pv[e].x - up.x - dn.x - lf.x - rt.x;
        const float tvy = 4.f * pv[e].y - up.y - dn.y - lf.y - rt.y;
        float2 o;
        o.x = fmaf(mu, acc[e].x, fmaf(lam, tvx, gam * pv[e].x));
        o.y = fmaf(mu, acc[e].y, fmaf(lam, tvy, gam * pv[e].y));
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

template <int NY>
constexpr size_t smem_apply_A8() {
    return 512 + ((size_t)NY * TX8 + (size_t)ExIdx<NY>::kStride * TX8 + 2 * NY) * sizeof(float2) +
           32 * sizeof(double);
}

template <int NY>
cudaError_t apply_A8(const Dims& d, const CUtensorMap& smap8, const float2* p, float2* q, const float* maskw,
                     const float2* tw, float mu, float lam, float gam, SliceState* st, Red red, cudaStream_t s) {
    const dim3 grid(d.nx / TX8, d.nb), block(TX8 * NY / 16);
    constexpr size_t sm = smem_apply_A8<NY>();
    static_assert(2 * NY * sizeof(float2) <= (size_t)ExIdx<NY>::kStride * TX8 * sizeof(float2),
                  "the halo fits in the exchange regions");
    cudaError_t e;
    if (st) {
        if ((e = set_smem_limit(k_apply_A8<NY, true>, (int)sm)) != cudaSuccess) return e;
        k_apply_A8<NY, true><<<grid, block, sm, s>>>(smap8, p, q, maskw, tw, d.nx, d.nc, mu, lam, gam, st, red);
    } else {
        if ((e = set_smem_limit(k_apply_A8<NY, false>, (int)sm)) != cudaSuccess) return e;
        k_apply_A8<NY, false><<<grid, block, sm, s>>>(smap8, p, q, maskw, tw, d.nx, d.nc, mu, lam, gam, st, red);
    }
    return cudaGetLastError();
}

template <int NY>
size_t smem_apply_A() {
    return 1024 + (2 * (size_t)NY * TX + (is_pow2(NY) ? 1 : 2) * (size_t)ExIdx<NY>::kStride * TX + 4 * NY) *
                      sizeof(float2) +
           64 * sizeof(double);
}

template <int NY>
cudaError_t apply_A_n(const Dims& d, const CUtensorMap& smap, const float2* p, float2* q, const float* maskw,
                      const float2* tw, float mu, float lam, float gam, SliceState* st, Red red, cudaStream_t s) {
    const dim3 grid(d.nx / TX, d.nb), block(TX * NY / 16);
    const size_t sm = smem_apply_A<NY>();
    cudaError_t e;
    if (st) {
        if ((e = set_smem_limit(k_apply_A<NY, true>, (int)sm)) !=
            cudaSuccess)
            return e;
        k_apply_A<NY, true><<<grid, block, sm, s>>>(smap, p, q, maskw, tw, d.nx, d.nc, mu, lam, gam, st, red);
    } else {
        if ((e = set_smem_limit(k_apply_A<NY, false>, (int)sm)) !=
            cudaSuccess)
            return e;
        k_apply_A<NY, false><<<grid, block, sm, s>>>(smap, p, q, maskw, tw, d.nx, d.nc, mu, lam, gam, st, red);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_apply_A(const Dims& d, const CUtensorMap& smap, const CUtensorMap& smap8, const float2* p,
                           float2* q, const float* maskw, const float2* tw_y, float mu, float lam, float gam,
                           SliceState* st, Red red, cudaStream_t s, int tile) {
    switch (d.ny) {
        case 32: return apply_A_n<32>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 64: return apply_A_n<64>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 128: return apply_A_n<128>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 256:
            return tile == 16 ? apply_A_n<256>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s)
                              : apply_A8<256>(d, smap8, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 512:
            return tile == 16 ? apply_A_n<512>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s)
                              : apply_A8<512>(d, smap8, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 192: return apply_A_n<192>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 224: return apply_A_n<224>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 320: return apply_A_n<320>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 384: return apply_A_n<384>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sb
