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
    float* mk = reinterpret_cast<float*>(halo + 2 * NY);
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
        mk[i] = maskw[(size_t)b * NY + i];
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
        for (int e = 0; e < 16; ++e) u[e] = cscale(u[e], mk[t + T * e]);
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

template <int NY>
size_t smem_apply_A() {
    return 1024 + (2 * (size_t)NY * TX + (is_pow2(NY) ? 1 : 2) * (size_t)ExIdx<NY>::kStride * TX + 3 * NY) *
                      sizeof(float2) +
           NY * sizeof(float) + 64 * sizeof(double);
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

cudaError_t launch_apply_A(const Dims& d, const CUtensorMap& smap, const float2* p, float2* q, const float* maskw,
                           const float2* tw_y, float mu, float lam, float gam, SliceState* st, Red red,
                           cudaStream_t s) {
    switch (d.ny) {
        case 32: return apply_A_n<32>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 64: return apply_A_n<64>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 128: return apply_A_n<128>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 256: return apply_A_n<256>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 512: return apply_A_n<512>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 192: return apply_A_n<192>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 224: return apply_A_n<224>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 320: return apply_A_n<320>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        case 384: return apply_A_n<384>(d, smap, p, q, maskw, tw_y, mu, lam, gam, st, red, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sb
