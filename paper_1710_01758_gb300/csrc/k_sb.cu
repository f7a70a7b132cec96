// Split Bregman kernels (Algorithm 1) around the PCG solve.
//
// The k-space data live in the hybrid space (k_y, x): yt = F_x^H y, stored only on the sampled
// phase-encode lines ("slots").  With a line mask F^H R F = (F_y^H R_y F_y) (x) I_x, so every
// data-term operation of Algorithm 1 (step 4's sum_i S_i^H F^H R^H y_i, steps 12-14's
// y_i += y_i^[1] - R F S_i x) becomes a length-ny transform along y, done per column tile
// exactly like the data term of A.
//
//  k_ytilde     yt1 = F_x^H y on the sampled lines (once per reconstruction).
//  k_rss        x = sqrt(sum_i |F^H y_i|^2) (step 1).
//  (the right-hand side and initial residual kernel is in k_rhs.cu)
//  k_sb_update  steps 6-11 on a 16x16 tile: TV shrink + Bregman updates, Haar analysis,
//               wavelet shrink + Bregman update, Haar synthesis, and the next
//               g = lam (D_x^H(d_x-b_x) + D_y^H(d_y-b_y)) + gam W^H(d_w-b_w).
#include "common.cuh"
#include "kernels.h"

namespace sb {
namespace {

constexpr int TX = 16;
constexpr int RY = 16;

struct ColIdx {
    int col;
    __device__ __forceinline__ int operator()(int pos) const { return pos * TX + col; }
};
template <int N>
struct RowIdx {
    int row;
    __device__ __forceinline__ int operator()(int pos) const {
        return row * (N + N / 16) + pos + (pos >> 4);
    }
};

// ------------------------------------------------------------------ yt1 = F_x^H y (sampled lines)
template <int NX>
__global__ void __launch_bounds__(RY * NX / 16)
k_ytilde(const float2* __restrict__ y, const int* __restrict__ lines, int ny, int nc, int ms, int nrows,
         float2* __restrict__ yt1, const float2* __restrict__ tw_g) {
    constexpr int T = NX / 16;
    constexpr int NT = RY * T;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* buf = reinterpret_cast<float2*>(smem);
    float2* tw = buf + RY * (NX + NX / 16);
    const int tid = threadIdx.x, t = tid % T, row = tid / T;
    const int grow = blockIdx.x * RY + row;  // over [nb][nc][ms]
    for (int i = tid; i < NX; i += NT) tw[i] = tw_g[i];
    const bool ok = grow < nrows;
    const int s = grow % ms, bc = grow / ms, b = bc / nc;
    const int ky = ok ? lines[(size_t)b * ms + s] : -1;
    float2 v[16];
    if (ky >= 0) {
        const size_t src = ((size_t)bc * ny + ky) * NX;
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = y[src + t + T * e];
    } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_2stage<NX, true>(v, t, buf, RowIdx<NX>{row}, tw);
    const float sc = rsqrtf((float)NX);
    if (ok)
#pragma unroll
        for (int e = 0; e < 16; ++e) yt1[(size_t)grow * NX + t + T * e] = cscale(v[e], sc);
}

// ------------------------------------------------------------------ root-sum-of-squares start
template <int NY>
__global__ void __launch_bounds__(TX * NY / 16)
k_rss(SbFields f, int nx, int nc, float2* __restrict__ x, const float2* __restrict__ tw_g) {
    constexpr int T = NY / 16;
    constexpr int NT = TX * T;
    const int b = blockIdx.y;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* buf0 = reinterpret_cast<float2*>(smem);
    float2* buf1 = buf0 + NY * TX;
    float2* tw = buf1 + NY * TX;
    int* sl = reinterpret_cast<int*>(tw + NY);
    const int tid = threadIdx.x, col = tid % TX, t = tid / TX;
    const int xg = blockIdx.x * TX + col;
    for (int i = tid; i < NY; i += NT) {
        tw[i] = tw_g[i];
        sl[i] = f.slot[(size_t)b * NY + i];
    }
    __syncthreads();
    float acc[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e] = 0.f;
    const ColIdx idx{col};
    const float sc = rsqrtf((float)NY);
    for (int c = 0; c < nc; ++c) {
        const float2* Y = f.yt1 + ((size_t)b * nc + c) * f.ms * nx;
        float2 v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int s = sl[t + T * e];
            v[e] = s >= 0 ? Y[(size_t)s * nx + xg] : make_float2(0.f, 0.f);
        }
        fft_2stage<NY, true>(v, t, (c & 1) ? buf1 : buf0, idx, tw);
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] += cabs2(v[e]) * (sc * sc);
    }
#pragma unroll
    for (int e = 0; e < 16; ++e)
        x[((size_t)b * NY + t + T * e) * nx + xg] = make_float2(sqrtf(acc[e]), 0.f);
}

// ------------------------------------------------------------------ steps 6-11 on a 16x16 tile
__device__ __forceinline__ float2 shrink(float2 z, float t) {
    const float m = sqrtf(cabs2(z));
    const float s = m > t ? (m - t) / m : 0.f;
    return cscale(z, s);
}

// One orthonormal Haar level on the leading `n` x `n` corner of a 16x16 tile (Mallat layout):
// along x, then along y.  inverse: along y, then along x.
__device__ void haar_level(float2 (*w)[16], int n, bool inverse) {
    const int tid = threadIdx.x;
    const int ry = tid / 16, cx = tid % 16;
    const float h = 0.70710678118654752f;
    const int half = n / 2;
    for (int pass = 0; pass < 2; ++pass) {
        const bool along_x = inverse ? (pass == 1) : (pass == 0);
        float2 o = make_float2(0.f, 0.f);
        const bool act = ry < n && cx < n;
        if (act) {
            const int i = along_x ? cx : ry;
            if (!inverse) {
                const int j = (i < half) ? i : i - half;
                const float2 a = along_x ? w[ry][2 * j] : w[2 * j][cx];
                const float2 c = along_x ? w[ry][2 * j + 1] : w[2 * j + 1][cx];
                o = (i < half) ? cscale(cadd(a, c), h) : cscale(csub(a, c), h);
            } else {
                const int j = i >> 1;
                const float2 lo = along_x ? w[ry][j] : w[j][cx];
                const float2 hi = along_x ? w[ry][j + half] : w[j + half][cx];
                o = (i & 1) ? cscale(csub(lo, hi), h) : cscale(cadd(lo, hi), h);
            }
        }
        __syncthreads();
        if (act) w[ry][cx] = o;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256)
k_sb_update(SbFields f, int nx, int ny, const float2* __restrict__ x, int levels, float lam, float gam,
            float tau_tv, float tau_w) {
    __shared__ float2 xs[18][18];   // x with a one-pixel periodic halo
    __shared__ float2 ux[17][17];   // d_x - b_x (new) on the tile and its +1 halo
    __shared__ float2 uy[17][17];
    __shared__ float2 w[16][16];
    const int b = blockIdx.z;
    const int y0 = blockIdx.y * 16, x0 = blockIdx.x * 16;
    const int tid = threadIdx.x;
    const size_t img = (size_t)b * ny * nx;
    for (int i = tid; i < 18 * 18; i += 256) {
        const int ly = i / 18, lx = i % 18;
        const int gy = (y0 - 1 + ly + ny) % ny, gx = (x0 - 1 + lx + nx) % nx;
        xs[ly][lx] = x[img + (size_t)gy * nx + gx];
    }
    __syncthreads();
    const int ty = tid / 16, tx = tid % 16;
    const size_t own = img + (size_t)(y0 + ty) * nx + x0 + tx;
    float2 gout = make_float2(0.f, 0.f);
    if (lam != 0.f) {
        // u = d - b (new) on the tile and its +1 halo; the halo cells belong to neighbouring
        // tiles, whose CTAs write their new b into the other buffer, so reading the old
        // buffer here is race-free
        for (int i = tid; i < 17 * 17; i += 256) {
            const int ly = i / 17, lx = i % 17;
            const int gy = (y0 + ly) % ny, gx = (x0 + lx) % nx;
            const size_t gi = img + (size_t)gy * nx + gx;
            const float2 xc = xs[ly + 1][lx + 1];
            const float2 dxv = csub(xc, xs[ly + 1][lx]);   // D_x x
            const float2 dyv = csub(xc, xs[ly][lx + 1]);   // D_y x
            const float2 bxv = f.bx[gi], byv = f.by[gi];
            const float2 dx = shrink(cadd(dxv, bxv), tau_tv);
            const float2 dy = shrink(cadd(dyv, byv), tau_tv);
            const float2 bxn = csub(cadd(bxv, dxv), dx);
            const float2 byn = csub(cadd(byv, dyv), dy);
            ux[ly][lx] = csub(dx, bxn);
            uy[ly][lx] = csub(dy, byn);
            if (ly < 16 && lx < 16) {
                f.bx_new[gi] = bxn;
                f.by_new[gi] = byn;
            }
        }
        __syncthreads();
        const float2 tvx = csub(ux[ty][tx], ux[ty][tx + 1]);
        const float2 tvy = csub(uy[ty][tx], uy[ty + 1][tx]);
        gout = cscale(cadd(tvx, tvy), lam);
    }
    if (gam != 0.f) {  // levels == 0: W is the identity
        w[ty][tx] = xs[ty + 1][tx + 1];
        __syncthreads();
        for (int l = 0, n = 16; l < levels; ++l, n >>= 1) haar_level(w, n, false);
        const float2 wc = w[ty][tx];
        const float2 bwv = f.bw[own];
        const float2 dw = shrink(cadd(wc, bwv), tau_w);
        const float2 bwn = csub(cadd(bwv, wc), dw);
        f.bw[own] = bwn;
        __syncthreads();
        w[ty][tx] = csub(dw, bwn);
        __syncthreads();
        for (int l = levels - 1; l >= 0; --l) haar_level(w, 16 >> l, true);
        gout = cadd(gout, cscale(w[ty][tx], gam));
    }
    f.g[own] = gout;
}

template <int NX>
size_t smem_row() { return (RY * (NX + NX / 16) + NX) * sizeof(float2); }

}  // namespace

cudaError_t launch_ytilde(const Dims& d, const float2* y, const int* lines, int ms, float2* yt1, const float2* tw_x,
                          cudaStream_t s) {
    const int nrows = d.nb * d.nc * ms;
    const dim3 grid((nrows + RY - 1) / RY);
    cudaError_t e;
#define CALL(N)                                                                                               \
    {                                                                                                         \
        const size_t sm = smem_row<N>();                                                                      \
        if (sm > 48 * 1024 &&                                                                                 \
            (e = cudaFuncSetAttribute(k_ytilde<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != \
                cudaSuccess)                                                                                  \
            return e;                                                                                         \
        k_ytilde<N><<<grid, RY * N / 16, sm, s>>>(y, lines, d.ny, d.nc, ms, nrows, yt1, tw_x);                \
        return cudaGetLastError();                                                                            \
    }
    switch (d.nx) {
        case 32: CALL(32)
        case 64: CALL(64)
        case 128: CALL(128)
        case 256: CALL(256)
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t launch_rss(const Dims& d, const SbFields& f, float2* x, const float2* tw_y, cudaStream_t s) {
    const dim3 grid(d.nx / TX, d.nb);
    cudaError_t e;
#define CALL(N)                                                                                            \
    {                                                                                                      \
        const size_t sm = (2 * N * TX + N) * sizeof(float2) + N * sizeof(int);                             \
        if (sm > 48 * 1024 &&                                                                              \
            (e = cudaFuncSetAttribute(k_rss<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != \
                cudaSuccess)                                                                               \
            return e;                                                                                      \
        k_rss<N><<<grid, TX * N / 16, sm, s>>>(f, d.nx, d.nc, x, tw_y);                                    \
        return cudaGetLastError();                                                                         \
    }
    switch (d.ny) {
        case 32: CALL(32)
        case 64: CALL(64)
        case 128: CALL(128)
        case 256: CALL(256)
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t launch_sb_update(const Dims& d, const SbFields& f, const float2* x, int levels, float lam, float gam,
                             float tau_tv, float tau_w, cudaStream_t s) {
    const dim3 grid(d.nx / 16, d.ny / 16, d.nb);
    k_sb_update<<<grid, 256, 0, s>>>(f, d.nx, d.ny, x, levels, lam, gam, tau_tv, tau_w);
    return cudaGetLastError();
}

}  // namespace sb
