// Split Bregman kernels (Algorithm 1) around the PCG solve.
//
// The k-space data live in the hybrid space (k_y, x): yt = F_x^H y, stored only on the sampled
// phase-encode lines ("slots").  With a line mask F^H R F = (F_y^H R_y F_y) (x) I_x, so every
// data-term operation of Algorithm 1 (step 4's sum_i S_i^H F^H R^H y_i, steps 12-14's
// y_i += y_i^[1] - R F S_i x) becomes a length-ny transform along y, done per column tile
// exactly like the data term of A.
//
//  k_ytilde     yt1 = F_x^H y on the sampled lines (once per reconstruction).
//  k_rss        x = sqrt(sum_i |F^H y_i|^2) (step 1) and the data term of b for y^[1],
//               bd1 = sum_i S_i^H F^H y_i^[1], from the same inverse transforms.
//  (the right-hand side and initial residual kernel is in k_rhs.cu)
//  (steps 6-11, shrink and Bregman updates, are in k_sbupd.cu)
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
    fft<NX, true>(v, t, buf, RowIdx<NX>{row}, tw);
    const float sc = rsqrtf((float)NX);
    if (ok)
#pragma unroll
        for (int e = 0; e < 16; ++e) yt1[(size_t)grow * NX + t + T * e] = cscale(v[e], sc);
}

// ------------------------------------------------------------------ root-sum-of-squares start
template <int NY>
__global__ void __launch_bounds__(TX * NY / 16)
k_rss(SbFields f, int nx, int nc, float2* __restrict__ x, int write_x, const float2* __restrict__ tw_g) {
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
    float2 bda[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        acc[e] = 0.f;
        bda[e] = make_float2(0.f, 0.f);
    }
    const ColIdx idx{col};
    const float sc = rsqrtf((float)NY);
    for (int c = 0; c < nc; ++c) {
        const float2* Y = f.yt1 + ((size_t)b * nc + c) * f.ms * nx;
        const float2* S = f.sens + ((size_t)b * nc + c) * NY * nx;
        float2 v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int s = sl[t + T * e];
            v[e] = s >= 0 ? Y[(size_t)s * nx + xg] : make_float2(0.f, 0.f);
        }
        fft<NY, true>(v, t, (c & 1) ? buf1 : buf0, idx, tw);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const float2 ci = cscale(v[e], sc);  // coil image F^H y_c
            acc[e] += cabs2(ci);
            bda[e] = cfmac(bda[e], __ldg(S + (size_t)(t + T * e) * nx + xg), ci);
        }
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const size_t gi = ((size_t)b * NY + t + T * e) * nx + xg;
        f.bd1[gi] = bda[e];
        f.bd[gi] = bda[e];
        if (write_x) x[gi] = make_float2(sqrtf(acc[e]), 0.f);
    }
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
            (e = set_smem_limit(k_ytilde<N>, (int)sm)) != \
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
        case 512: CALL(512)
        case 192: CALL(192)
        case 224: CALL(224)
        case 320: CALL(320)
        case 384: CALL(384)
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t launch_rss(const Dims& d, const SbFields& f, float2* x, int write_x, const float2* tw_y,
                       cudaStream_t s) {
    const dim3 grid(d.nx / TX, d.nb);
    cudaError_t e;
#define CALL(N)                                                                                            \
    {                                                                                                      \
        const size_t sm = (2 * N * TX + N) * sizeof(float2) + N * sizeof(int);                             \
        if (sm > 48 * 1024 &&                                                                              \
            (e = set_smem_limit(k_rss<N>, (int)sm)) != \
                cudaSuccess)                                                                               \
            return e;                                                                                      \
        k_rss<N><<<grid, TX * N / 16, sm, s>>>(f, d.nx, d.nc, x, write_x, tw_y);                           \
        return cudaGetLastError();                                                                         \
    }
    switch (d.ny) {
        case 32: CALL(32)
        case 64: CALL(64)
        case 128: CALL(128)
        case 256: CALL(256)
        case 512: CALL(512)
        case 192: CALL(192)
        case 224: CALL(224)
        case 320: CALL(320)
        case 384: CALL(384)
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

}  // namespace sb
