// Once-per-plan kernels: mask analysis and the construction of k (Eq. Kdiag).
//
// k_c follows "Efficient Implementation of the Preconditioner" (Eq. diagonalelements): the
// diagonal of sum_i C_i^H R C_i, C_i = F S_i F^H BCCB, is the circular correlation
//   k_c[kappa] = sum_l r[l] g[l - kappa],   g = sum_i |DFT2(s_i)|^2 / N^2,
// evaluated as k_c = IDFT2( DFT2(r) conj(DFT2(g)) ) / N with unnormalised transforms.  k_d is
// the DFT of the first row of D_x^H D_x + D_y^H D_y, 4 - 2 cos(2 pi kx/nx) - 2 cos(2 pi ky/ny),
// and k_w = 1.  The generic row / column FFT kernels here reuse the register-resident Stockham
// transform of common.cuh.
#include <algorithm>

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

__global__ void k_mask_lines(const uint8_t* __restrict__ mask, int nx, int* line_val, int* line_uniform) {
    // one CTA per (slice, line): blockIdx.x = line, blockIdx.y = slice
    const size_t row = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    const uint8_t* m = mask + row * nx;
    const int v0 = m[0] != 0;
    int diff = 0;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) diff |= ((m[i] != 0) != v0);
    diff = __syncthreads_or(diff);
    if (threadIdx.x == 0) {
        line_val[row] = v0;
        line_uniform[row] = !diff;
    }
}

// src == dst transforms in place (each thread writes back only the values it read)
template <int NX, bool INV>
__global__ void __launch_bounds__(RY * NX / 16)
k_fft_rows(const float2* src, float2* dst, int nrows_total, const float2* __restrict__ tw_g) {
    constexpr int T = NX / 16;
    constexpr int NT = RY * T;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* buf = reinterpret_cast<float2*>(smem);
    float2* tw = buf + RY * (NX + NX / 16);
    const int tid = threadIdx.x, t = tid % T, row = tid / T;
    const int grow = blockIdx.x * RY + row;
    for (int i = tid; i < NX; i += NT) tw[i] = tw_g[i];
    float2 v[16];
    const bool ok = grow < nrows_total;
    const size_t base = (size_t)(ok ? grow : 0) * NX;
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = src[base + t + T * e];
    __syncthreads();
    fft<NX, INV>(v, t, buf, RowIdx<NX>{row}, tw);
    if (ok)
#pragma unroll
        for (int e = 0; e < 16; ++e) dst[base + t + T * e] = v[e];
}

template <int NY, bool INV>
__global__ void __launch_bounds__(TX * NY / 16)
k_fft_cols(float2* __restrict__ data, int nx, const float2* __restrict__ tw_g) {
    constexpr int T = NY / 16;
    constexpr int NT = TX * T;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* buf = reinterpret_cast<float2*>(smem);
    float2* tw = buf + NY * TX;
    const int tid = threadIdx.x, col = tid % TX, t = tid / TX;
    const int x = blockIdx.x * TX + col;
    for (int i = tid; i < NY; i += NT) tw[i] = tw_g[i];
    const size_t img = (size_t)blockIdx.y * NY * nx;
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = data[img + (size_t)(t + T * e) * nx + x];
    __syncthreads();
    fft<NY, INV>(v, t, buf, ColIdx{col}, tw);
#pragma unroll
    for (int e = 0; e < 16; ++e) data[img + (size_t)(t + T * e) * nx + x] = v[e];
}

// (a sum of nc non-negative FP32 terms: relative error below nc * 2^-24, no cancellation)
__global__ void k_coil_power(const float2* __restrict__ spec, float2* __restrict__ g, int n, int nc, float inv_n2) {
    const int b = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int c = 0; c < nc; ++c) acc += cabs2(spec[((size_t)b * nc + c) * n + i]);
        g[(size_t)b * n + i] = make_float2(acc * inv_n2, 0.f);
    }
}

// 2D planes: the column DFTs of every coil's row-transformed sensitivities and the coil power
// sum in one pass (the coil spectra are never written): per column tile of a slice, coil by coil,
// g += |DFT_y(column)|^2, then g / N^2
template <int NY>
__global__ void __launch_bounds__(TX * NY / 16)
k_coil_power_cols(const float2* __restrict__ spec, float2* __restrict__ g, int nx, int nc, float inv_n2,
                  const float2* __restrict__ tw_g) {
    constexpr int T = NY / 16;
    constexpr int NT = TX * T;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* buf = reinterpret_cast<float2*>(smem);
    float2* tw = buf + NY * TX;
    const int tid = threadIdx.x, col = tid % TX, t = tid / TX;
    const int x = blockIdx.x * TX + col, b = blockIdx.y;
    for (int i = tid; i < NY; i += NT) tw[i] = tw_g[i];
    float acc[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e] = 0.f;
    for (int c = 0; c < nc; ++c) {
        const size_t img = ((size_t)b * nc + c) * NY * nx;
        float2 v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = spec[img + (size_t)(t + T * e) * nx + x];
        __syncthreads();  // the twiddles are in place; the previous coil's exchange reads are done
        fft<NY, false>(v, t, buf, ColIdx{col}, tw);
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] += cabs2(v[e]);
    }
    const size_t out = (size_t)b * NY * nx;
#pragma unroll
    for (int e = 0; e < 16; ++e) g[out + (size_t)(t + T * e) * nx + x] = make_float2(acc[e] * inv_n2, 0.f);
}

__global__ void k_mask_to_complex(const uint8_t* __restrict__ mask, float2* __restrict__ out, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_float2(mask[i] ? 1.f : 0.f, 0.f);
}

__global__ void k_mul_conj(float2* __restrict__ R, const float2* __restrict__ G, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        R[i] = cmul(R[i], make_float2(G[i].x, -G[i].y));
}

// k = mu kc + lam kd + gam (first pass) and its per-slice maximum (non-negative floats compare
// as integers); kd is the geometry's table (volumes: k_d = 6 - 2 cos - 2 cos - 2 cos; with nz = 1
// the z term is 2 and this is the 2D formula), computed once per plan on the host
__global__ void k_form_k(const float2* __restrict__ kc_raw, const float* __restrict__ kd, int n, float mu, float lam,
                         float gam, float inv_n, float* __restrict__ k, unsigned* __restrict__ kmax) {
    const int b = blockIdx.y;
    float local = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float kc = kc_raw[(size_t)b * n + i].x * inv_n;
        const float v = fmaf(mu, kc, fmaf(lam, kd[i], gam));
        k[(size_t)b * n + i] = v;
        local = fmaxf(local, v);
    }
    // one atomic per block: atomics on one address serialise in L2 (one per warp over a 64-slice
    // batch, 2048 per slice, took 90 us), so the warps' maxima meet in shared memory first
    __shared__ unsigned wmax[32];
    const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(fmaxf(local, 0.f)));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        const unsigned v = __reduce_max_sync(0xffffffffu, threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0u);
        if (threadIdx.x == 0) atomicMax(kmax + b, v);
    }
}

// clamp k below at 1e-12 max(k) and store 1/(k N), the scale that turns the unnormalised
// DFT pair of the preconditioner into F^H diag(k)^{-1} F
__global__ void k_clamp_invert(float* __restrict__ k, float* __restrict__ invk, int n, const unsigned* __restrict__ kmax) {
    const int b = blockIdx.y;
    const float floor_v = 1e-12f * __uint_as_float(kmax[b]);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float v = fmaxf(k[(size_t)b * n + i], floor_v);
        k[(size_t)b * n + i] = v;
        invk[(size_t)b * n + i] = 1.f / (v * (float)n);
    }
}

// Jacobi: w = 1 / diag(A), diag(A)_j = mu (nnz(r)/N) sum_c |S_c[j]|^2 + 2 ndim lam + gam
// ((S^H F^H R F S)_jj = |s_j|^2 (F^H R F)_jj = |s_j|^2 nnz(r)/N; each D_a^H D_a adds 2).
// `ny` here counts the readout lines of one slice or volume (ny nz for a volume).
__global__ void k_jacobi_diag(const float2* __restrict__ sens, const float* __restrict__ maskw, int n, int ny, int nc,
                              float mu, float lam, float gam, float tvd, float* __restrict__ w) {
    const int b = blockIdx.y;
    __shared__ float frac_s;
    if (threadIdx.x < 32) {
        float s = 0.f;  // maskw holds 1/ny on sampled lines: its sum is nnz(r)/N
        for (int y = threadIdx.x; y < ny; y += 32) s += maskw[(size_t)b * ny + y];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) frac_s = s;
    }
    __syncthreads();
    const float frac = frac_s;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float p = 0.f;
        for (int c = 0; c < nc; ++c) p += cabs2(sens[((size_t)b * nc + c) * n + i]);
        w[(size_t)b * n + i] = 1.f / fmaf(mu * frac, p, tvd * lam + gam);
    }
}

template <int NX>
cudaError_t fft_rows_n(int ny, int nimg, const float2* src, float2* dst, const float2* tw, bool inv, cudaStream_t s) {
    const int rows = ny * nimg;
    const dim3 grid((rows + RY - 1) / RY), block(RY * NX / 16);
    const size_t sm = (RY * (NX + NX / 16) + NX) * sizeof(float2);
    cudaError_t e;
    if (inv) {
        if (sm > 48 * 1024 && (e = set_smem_limit(k_fft_rows<NX, true>, (int)sm)) != cudaSuccess) return e;
        k_fft_rows<NX, true><<<grid, block, sm, s>>>(src, dst, rows, tw);
    } else {
        if (sm > 48 * 1024 && (e = set_smem_limit(k_fft_rows<NX, false>, (int)sm)) != cudaSuccess) return e;
        k_fft_rows<NX, false><<<grid, block, sm, s>>>(src, dst, rows, tw);
    }
    return cudaGetLastError();
}

template <int NY>
cudaError_t coil_power_cols_n(const Dims& d, const float2* spec, float2* g, const float2* tw, cudaStream_t s) {
    const dim3 grid(d.nx / TX, d.nb), block(TX * NY / 16);
    const size_t sm = (NY * TX + NY) * sizeof(float2);
    cudaError_t e;
    if (sm > 48 * 1024 && (e = set_smem_limit(k_coil_power_cols<NY>, (int)sm)) != cudaSuccess) return e;
    const float n = (float)d.nx * (float)NY;
    k_coil_power_cols<NY><<<grid, block, sm, s>>>(spec, g, d.nx, d.nc, 1.f / (n * n), tw);
    return cudaGetLastError();
}

template <int NY>
cudaError_t fft_cols_n(int nx, int nimg, float2* data, const float2* tw, bool inv, cudaStream_t s) {
    const dim3 grid(nx / TX, nimg), block(TX * NY / 16);
    const size_t sm = (NY * TX + NY) * sizeof(float2);
    cudaError_t e;
    if (inv) {
        if (sm > 48 * 1024 && (e = set_smem_limit(k_fft_cols<NY, true>, (int)sm)) != cudaSuccess) return e;
        k_fft_cols<NY, true><<<grid, block, sm, s>>>(data, nx, tw);
    } else {
        if (sm > 48 * 1024 && (e = set_smem_limit(k_fft_cols<NY, false>, (int)sm)) != cudaSuccess) return e;
        k_fft_cols<NY, false><<<grid, block, sm, s>>>(data, nx, tw);
    }
    return cudaGetLastError();
}

unsigned elem_blocks(size_t n) {
    const size_t b = (n + 255) / 256;
    return (unsigned)(b < 4096 ? b : 4096);
}

}  // namespace

cudaError_t launch_mask_lines(const Dims& d, const uint8_t* mask, int* line_val, int* line_uniform, cudaStream_t s) {
    k_mask_lines<<<dim3(d.ny, d.nb), 128, 0, s>>>(mask, d.nx, line_val, line_uniform);
    return cudaGetLastError();
}

cudaError_t launch_fft_rows_from(int nx, int ny, int nimg, const float2* src, float2* dst, const float2* tw_x,
                                 bool inv, cudaStream_t s) {
    switch (nx) {
        case 32: return fft_rows_n<32>(ny, nimg, src, dst, tw_x, inv, s);
        case 64: return fft_rows_n<64>(ny, nimg, src, dst, tw_x, inv, s);
        case 128: return fft_rows_n<128>(ny, nimg, src, dst, tw_x, inv, s);
        case 256: return fft_rows_n<256>(ny, nimg, src, dst, tw_x, inv, s);
        case 512: return fft_rows_n<512>(ny, nimg, src, dst, tw_x, inv, s);
        case 192: return fft_rows_n<192>(ny, nimg, src, dst, tw_x, inv, s);
        case 224: return fft_rows_n<224>(ny, nimg, src, dst, tw_x, inv, s);
        case 320: return fft_rows_n<320>(ny, nimg, src, dst, tw_x, inv, s);
        case 384: return fft_rows_n<384>(ny, nimg, src, dst, tw_x, inv, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fft_rows(int nx, int ny, int nimg, float2* data, const float2* tw_x, bool inv, cudaStream_t s) {
    return launch_fft_rows_from(nx, ny, nimg, data, data, tw_x, inv, s);
}

cudaError_t launch_coil_power_cols(const Dims& d, const float2* spec, float2* g, const float2* tw_y, cudaStream_t s) {
    switch (d.ny) {
        case 32: return coil_power_cols_n<32>(d, spec, g, tw_y, s);
        case 64: return coil_power_cols_n<64>(d, spec, g, tw_y, s);
        case 128: return coil_power_cols_n<128>(d, spec, g, tw_y, s);
        case 256: return coil_power_cols_n<256>(d, spec, g, tw_y, s);
        case 512: return coil_power_cols_n<512>(d, spec, g, tw_y, s);
        case 192: return coil_power_cols_n<192>(d, spec, g, tw_y, s);
        case 224: return coil_power_cols_n<224>(d, spec, g, tw_y, s);
        case 320: return coil_power_cols_n<320>(d, spec, g, tw_y, s);
        case 384: return coil_power_cols_n<384>(d, spec, g, tw_y, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fft_cols(int nx, int ny, int nimg, float2* data, const float2* tw_y, bool inv, cudaStream_t s) {
    switch (ny) {
        case 32: return fft_cols_n<32>(nx, nimg, data, tw_y, inv, s);
        case 64: return fft_cols_n<64>(nx, nimg, data, tw_y, inv, s);
        case 128: return fft_cols_n<128>(nx, nimg, data, tw_y, inv, s);
        case 256: return fft_cols_n<256>(nx, nimg, data, tw_y, inv, s);
        case 512: return fft_cols_n<512>(nx, nimg, data, tw_y, inv, s);
        case 192: return fft_cols_n<192>(nx, nimg, data, tw_y, inv, s);
        case 224: return fft_cols_n<224>(nx, nimg, data, tw_y, inv, s);
        case 320: return fft_cols_n<320>(nx, nimg, data, tw_y, inv, s);
        case 384: return fft_cols_n<384>(nx, nimg, data, tw_y, inv, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_coil_power(const Dims& d, const float2* data, float2* g, cudaStream_t s) {
    const int n = d.nx * d.ny;
    const float inv_n2 = (float)(1.0 / ((double)n * (double)n));
    k_coil_power<<<dim3(elem_blocks(n), d.nb), 256, 0, s>>>(data, g, n, d.nc, inv_n2);
    return cudaGetLastError();
}

cudaError_t launch_mask_to_complex(const Dims& d, const uint8_t* mask, float2* out, cudaStream_t s) {
    const size_t n = (size_t)d.nx * d.ny * d.nb;
    k_mask_to_complex<<<elem_blocks(n), 256, 0, s>>>(mask, out, n);
    return cudaGetLastError();
}

cudaError_t launch_mul_conj(const Dims& d, float2* R, const float2* G, cudaStream_t s) {
    const size_t n = (size_t)d.nx * d.ny * d.nb;
    k_mul_conj<<<elem_blocks(n), 256, 0, s>>>(R, G, n);
    return cudaGetLastError();
}

cudaError_t launch_jacobi_diag(const Dims& d, int nz, const float2* sens, const float* maskw, float mu, float lam,
                               float gam, float* w, cudaStream_t s) {
    const int n = d.nx * d.ny * nz;
    k_jacobi_diag<<<dim3(elem_blocks(n), d.nb), 256, 0, s>>>(sens, maskw, n, d.ny * nz, d.nc, mu, lam, gam,
                                                             nz > 1 ? 6.f : 4.f, w);
    return cudaGetLastError();
}

cudaError_t launch_finish_k(const Dims& d, int nz, const float2* kc_raw, const float* kd, float mu, float lam,
                            float gam, float* k, float* invk, unsigned* kmax, cudaStream_t s) {
    const int n = d.nx * d.ny * nz;
    cudaError_t e = cudaMemsetAsync(kmax, 0, sizeof(unsigned) * d.nb, s);
    if (e != cudaSuccess) return e;
    const dim3 grid(elem_blocks(n), d.nb);
    // at most 64 blocks per slice for the maximum (each block one atomic; threads loop)
    k_form_k<<<dim3(std::min(elem_blocks(n), 64u), d.nb), 256, 0, s>>>(kc_raw, kd, n, mu, lam, gam, 1.f / n, k, kmax);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_clamp_invert<<<grid, 256, 0, s>>>(k, invk, n, kmax);
    return cudaGetLastError();
}

}  // namespace sb
