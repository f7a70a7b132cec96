// The Daubechies four-tap wavelet (the wavelet of the paper's experiments, Methods,
// "Reconstruction") for steps 8 and 11 of Algorithm 1 and the wavelet part of step 4's b:
//   W x:          per level l (band ny >> l by nx >> l, the low-pass corner), one analysis step
//                 along x on every band row, then along y on every band column (Mallat layout);
//   shrink:       d_w = shrink(W x + b_w, tau_w), b_w <- b_w + W x - d_w, u_w = d_w - b_w;
//   W^H u_w:      the levels undone coarsest first (y, then x), and g += gamma W^H u_w.
// One analysis step along an axis of length n (periodic):
//   a[k] = sum_m h_m s[(2k + m) mod n],  d[k] = sum_m g_m s[(2k + m) mod n],  k < n/2,
// h = (1 + sqrt 3, 3 + sqrt 3, 3 - sqrt 3, 1 - sqrt 3) / (4 sqrt 2), g_m = (-1)^m h_{3-m}.
// The synthesis step is its transpose, evaluated as a gather: s[j] receives the two taps
// m = j mod 2 and m + 2, from k = ((j - m) mod n) / 2.
// Unlike the Haar transform, the taps of neighbouring blocks overlap, so each band line is
// staged whole in shared memory (n <= 512).
#include "common.cuh"
#include "kernels.h"

namespace sb {
namespace {

__device__ __forceinline__ float d4h(int m) {
    // (1 + sqrt 3) / (4 sqrt 2), (3 + sqrt 3) / (4 sqrt 2), (3 - sqrt 3) / (4 sqrt 2), (1 - sqrt 3) / (4 sqrt 2)
    constexpr float h0 = 0.48296291314453414f, h1 = 0.83651630373780794f, h2 = 0.22414386804201339f,
                    h3 = -0.12940952255126037f;
    return m == 0 ? h0 : (m == 1 ? h1 : (m == 2 ? h2 : h3));
}
__device__ __forceinline__ float d4g(int m) {  // g_m = (-1)^m h_{3-m}
    return (m & 1) ? -d4h(3 - m) : d4h(3 - m);
}

// one analysis (INV = false) or synthesis step on a line of n values in shared memory `s`,
// writing the result to `out` at stride `ostride`
template <bool INV>
__device__ __forceinline__ void d4_line(const float2* s, int n, float2* out, size_t ostride, int lane, int nlanes) {
    const int h = n / 2;
    if (!INV) {
        for (int k = lane; k < h; k += nlanes) {
            float2 a = make_float2(0.f, 0.f), d = make_float2(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float2 v = s[(2 * k + m) % n];
                a = make_float2(fmaf(d4h(m), v.x, a.x), fmaf(d4h(m), v.y, a.y));
                d = make_float2(fmaf(d4g(m), v.x, d.x), fmaf(d4g(m), v.y, d.y));
            }
            out[(size_t)k * ostride] = a;
            out[(size_t)(h + k) * ostride] = d;
        }
    } else {
        for (int j = lane; j < n; j += nlanes) {
            float2 v = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int m = (j & 1) + 2 * q;
                const int k = ((j - m + n) % n) / 2;
                const float2 a = s[k], d = s[h + k];
                v.x = fmaf(d4h(m), a.x, fmaf(d4g(m), d.x, v.x));
                v.y = fmaf(d4h(m), a.y, fmaf(d4g(m), d.y, v.y));
            }
            out[(size_t)j * ostride] = v;
        }
    }
}

// rows of the band [by][bx] of slice b: src -> dst (may alias: the row is staged first)
template <bool INV>
__global__ void __launch_bounds__(256)
k_d4_rows(const float2* __restrict__ src, float2* dst, int nx, int ny, int bx) {
    __shared__ float2 s[512];
    const int y = blockIdx.x, b = blockIdx.y;
    const size_t row = ((size_t)b * ny + y) * nx;
    for (int i = threadIdx.x; i < bx; i += blockDim.x) s[i] = src[row + i];
    __syncthreads();
    d4_line<INV>(s, bx, dst + row, 1, threadIdx.x, blockDim.x);
}

// columns of the band [by][bx]: 16 columns per CTA, 16 threads per column, in place
template <bool INV>
__global__ void __launch_bounds__(256)
k_d4_cols(float2* c, int nx, int ny, int bx, int by) {
    extern __shared__ float2 sc[];  // [16][by]
    const int b = blockIdx.y;
    const int x0 = blockIdx.x * 16;
    const int cl = threadIdx.x % 16, ln = threadIdx.x / 16;
    const size_t img = (size_t)b * ny * nx;
    const bool ok = x0 + cl < bx;
    if (ok)
        for (int y = ln; y < by; y += 16) sc[cl * by + y] = c[img + (size_t)y * nx + x0 + cl];
    __syncthreads();
    if (ok) d4_line<INV>(sc + cl * by, by, c + img + x0 + cl, nx, ln, 16);
}

__device__ __forceinline__ float2 shrink_w(float2 z, float t) {
    const float m = sqrtf(cabs2(z));
    const float s = m > t ? (m - t) / m : 0.f;
    return cscale(z, s);
}

// steps 8 and 11 on every coefficient: w holds W x on entry and u_w = d_w - b_w on exit
__global__ void k_d4_shrink(float2* __restrict__ w, float2* __restrict__ bw, size_t n, float tau) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 u = w[i], bv = bw[i];
        const float2 dv = shrink_w(cadd(u, bv), tau);
        const float2 bn = csub(cadd(bv, u), dv);
        bw[i] = bn;
        w[i] = csub(dv, bn);
    }
}

__global__ void k_add_scaled(float2* __restrict__ g, const float2* __restrict__ w, size_t n, float gam) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 v = w[i];
        g[i] = make_float2(fmaf(gam, v.x, g[i].x), fmaf(gam, v.y, g[i].y));
    }
}

// The dynamic shared-memory limit of a kernel is one setting shared by every host thread, so it
// is always set to the largest size any launch needs (16 columns x 512 rows): a smaller,
// per-launch value could be lowered by another thread between its set and its launch.
constexpr int kColsSmemMax = 16 * 512 * (int)sizeof(float2);

unsigned blocks_for(size_t n) {
    const size_t b = (n + 255) / 256;
    return (unsigned)(b < 8192 ? b : 8192);
}

}  // namespace

cudaError_t launch_d4_update(const Dims& d, const float2* x, float2* w, float2* bw, float2* g, int levels, float gam,
                             float tau_w, cudaStream_t s) {
    if (levels < 1 || d.nx > 512 || d.ny > 512 || (d.nx >> (levels - 1)) < 4 || (d.ny >> (levels - 1)) < 4)
        return cudaErrorInvalidValue;
    const size_t n = (size_t)d.nb * d.nx * d.ny;
    cudaError_t e;
    // analysis, finest level first: rows (the first level reads x), then columns
    for (int l = 0; l < levels; ++l) {
        const int bx = d.nx >> l, by = d.ny >> l;
        k_d4_rows<false><<<dim3(by, d.nb), 256, 0, s>>>(l == 0 ? x : w, w, d.nx, d.ny, bx);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const size_t sm = (size_t)16 * by * sizeof(float2);
        if ((e = set_smem_limit(k_d4_cols<false>, kColsSmemMax)) !=
            cudaSuccess)
            return e;
        k_d4_cols<false><<<dim3((bx + 15) / 16, d.nb), 256, sm, s>>>(w, d.nx, d.ny, bx, by);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_d4_shrink<<<blocks_for(n), 256, 0, s>>>(w, bw, n, tau_w);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // synthesis, coarsest level first: columns, then rows
    for (int l = levels - 1; l >= 0; --l) {
        const int bx = d.nx >> l, by = d.ny >> l;
        const size_t sm = (size_t)16 * by * sizeof(float2);
        if ((e = set_smem_limit(k_d4_cols<true>, kColsSmemMax)) !=
            cudaSuccess)
            return e;
        k_d4_cols<true><<<dim3((bx + 15) / 16, d.nb), 256, sm, s>>>(w, d.nx, d.ny, bx, by);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_d4_rows<true><<<dim3(by, d.nb), 256, 0, s>>>(w, w, d.nx, d.ny, bx);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_add_scaled<<<blocks_for(n), 256, 0, s>>>(g, w, n, gam);
    return cudaGetLastError();
}

int d4_update_launches(int levels) { return 4 * levels + 2; }

}  // namespace sb
