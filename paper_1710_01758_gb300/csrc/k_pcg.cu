// Kernels of one preconditioned-CG iteration (Theory, "Complexity": one application of A and
// one of M^{-1} per iteration) on a batch of slices.
//
//  (q = A p is in k_applyA.cu)
//  k_row_fwd      r -= alpha q, ||r||^2, then the DFT along x of r (first half of M^{-1}).
//  k_col_precond  DFT along y, scale by 1/(k N), inverse DFT along y (middle of M^{-1});
//                 rho = r^H M^{-1} r = sum |DFT2 r|^2 / (N k) is accumulated in k-space.
//  k_row_inv      inverse DFT along x gives z; x += alpha p, p = z + beta p.
//  k_vec_plain    the same CG updates with z = r (no preconditioner) or z = r / diag(A) (Jacobi).
// FP64 holds every CG scalar; vectors are complex64.  Cross-CTA sums use the last-CTA
// pattern (common.cuh), so a CG iteration needs no extra scalar launches and no host sync.
#include "common.cuh"
#include "kernels.h"

namespace sb {
namespace {

constexpr int RY = 16;  // rows per CTA in row kernels

template <int CT>
struct ColIdx {
    int col;
    __device__ __forceinline__ int operator()(int pos) const { return pos * CT + col; }
};
// Barrier of a row transform: a row's T = NX / 16 threads are consecutive, so for power-of-two
// NX <= 512 they lie within one warp (T divides 32) and its exchanges need only __syncwarp;
// otherwise (mixed radix, rows straddling warps) the whole CTA synchronises.
template <int NX>
struct RowBar {
    __device__ __forceinline__ void operator()() const {
        if constexpr (is_pow2(NX) && NX / 16 <= 32) __syncwarp();
        else __syncthreads();
    }
};

template <int N>
struct RowIdx {
    int row;
    __device__ __forceinline__ int operator()(int pos) const {
        return row * (N + N / 16) + pos + (pos >> 4);
    }
};

// ------------------------------------------------------------------------------ row pass F_x
// MODE 0: t = F_x(r), slices filtered by st if given.  MODE 1: r -= alpha q first (PCG step).
template <int NX, int MODE>
__global__ void __launch_bounds__(RY * NX / 16)
k_row_fwd(float2* __restrict__ r, const float2* __restrict__ q, float2* __restrict__ tout,
          const float2* __restrict__ tw_g, int ny, SliceState* st, double tol2, Red red) {
    constexpr int T = NX / 16;
    constexpr int NT = RY * T;
    const int b = blockIdx.y;
    if (st != nullptr && st[b].state != ST_ACTIVE) return;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* buf = reinterpret_cast<float2*>(smem);
    float2* tw = buf + RY * (NX + NX / 16);
    double* red_s = reinterpret_cast<double*>(tw + NX);
    __shared__ int flag;
    const int tid = threadIdx.x, t = tid % T, row = tid / T;
    const int y = blockIdx.x * RY + row;
    const size_t base = ((size_t)b * ny + y) * NX;
    for (int i = tid; i < NX; i += NT) tw[i] = tw_g[i];
    float2 v[16];
    float rr = 0.f;
    if constexpr (MODE == 1) {
        const float alpha = (float)st[b].alpha;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const size_t i = base + t + T * e;
            const float2 qq = q[i];
            float2 rv = r[i];
            rv.x = fmaf(-alpha, qq.x, rv.x);
            rv.y = fmaf(-alpha, qq.y, rv.y);
            r[i] = rv;
            v[e] = rv;
            rr += cabs2(rv);
        }
    } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = r[base + t + T * e];
    }
    __syncthreads();
    fft_bar<NX, false>(v, t, buf, RowIdx<NX>{row}, tw, RowBar<NX>{});
#pragma unroll
    for (int e = 0; e < 16; ++e) tout[base + t + T * e] = v[e];
    if constexpr (MODE == 1) {
        double vv[1] = {(double)rr}, tot[1];
        const int np = gridDim.x;
        if (last_block_total<1>(vv, red.part, np, b * np + blockIdx.x, red.counter + b, tot, red_s, &flag) &&
            threadIdx.x == 0) {
            SliceState& S = st[b];
            S.rnorm2 = tot[0];
            if (!isfinite(tot[0])) S.state = ST_NONFINITE;
            else if (tot[0] <= tol2 * S.bnorm2) S.state = ST_FINISHING;
        }
    }
}

// ------------------------------------------------------------------------------ column pass
// CT columns per CTA (8, 16 or 32: a tuning choice); the 1/(kN) weights are loaded with the data,
// before the forward transform, so their latency overlaps it.
template <int NY, bool PCG, int CT>
__global__ void __launch_bounds__(CT * NY / 16)
k_col_precond(float2* __restrict__ tb, const float* __restrict__ invk, const float2* __restrict__ tw_g,
              int nx, SliceState* st, int init, Red red) {
    constexpr int T = NY / 16;
    constexpr int NT = CT * T;
    const int b = blockIdx.y;
    if (PCG && st[b].state != ST_ACTIVE) return;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* buf0 = reinterpret_cast<float2*>(smem);
    float2* buf1 = buf0 + NY * CT;
    float2* tw = buf1 + NY * CT;
    double* red_s = reinterpret_cast<double*>(tw + NY);
    __shared__ int flag;
    const int tid = threadIdx.x, col = tid % CT, t = tid / CT;
    const int x = blockIdx.x * CT + col;
    for (int i = tid; i < NY; i += NT) tw[i] = tw_g[i];
    const size_t img = (size_t)b * NY * nx;
    float2 v[16];
    float wk[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        v[e] = tb[img + (size_t)(t + T * e) * nx + x];
        wk[e] = __ldg(invk + img + (size_t)(t + T * e) * nx + x);
    }
    __syncthreads();
    const ColIdx<CT> idx{col};
    fft<NY, false>(v, t, buf0, idx, tw);
    float rz = 0.f;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        rz = fmaf(cabs2(v[e]), wk[e], rz);
        v[e] = cscale(v[e], wk[e]);
    }
    fft<NY, true>(v, t, buf1, idx, tw);
#pragma unroll
    for (int e = 0; e < 16; ++e) tb[img + (size_t)(t + T * e) * nx + x] = v[e];
    if constexpr (PCG) {
        double vv[1] = {(double)rz}, tot[1];
        const int np = gridDim.x;
        if (last_block_total<1>(vv, red.part, np, b * np + blockIdx.x, red.counter + b, tot, red_s, &flag) &&
            threadIdx.x == 0) {
            SliceState& S = st[b];
            const double rho_new = tot[0];
            if (!isfinite(rho_new)) {
                S.state = ST_NONFINITE;
            } else {
                if (!init) S.beta = rho_new / S.rho;
                S.rho = rho_new;
            }
        }
    }
}

// ------------------------------------------------------------------------------ row pass F_x^H
// MODE 0: out = z.  MODE 1: p = z (CG start).  MODE 2: x += alpha p; p = z + beta p.
template <int NX, int MODE>
__global__ void __launch_bounds__(RY * NX / 16)
k_row_inv(const float2* __restrict__ tb, float2* __restrict__ out, float2* __restrict__ x,
          float2* __restrict__ p, const float2* __restrict__ tw_g, int ny, SliceState* st, Red red) {
    constexpr int T = NX / 16;
    constexpr int NT = RY * T;
    const int b = blockIdx.y;
    const int s = (MODE == 0) ? ST_ACTIVE : st[b].state;
    if (MODE == 1 && s != ST_ACTIVE) return;
    if (MODE == 2 && s != ST_ACTIVE && s != ST_FINISHING) return;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* buf = reinterpret_cast<float2*>(smem);
    float2* tw = buf + RY * (NX + NX / 16);
    double* red_s = reinterpret_cast<double*>(tw + NX);
    __shared__ int flag;
    const int tid = threadIdx.x, t = tid % T, row = tid / T;
    const int y = blockIdx.x * RY + row;
    const size_t base = ((size_t)b * ny + y) * NX;
    if (MODE == 2 && s == ST_FINISHING) {
        // last step of a converged slice: x += alpha p; then mark it done
        const float alpha = (float)st[b].alpha;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const size_t i = base + t + T * e;
            const float2 pp = p[i];
            float2 xv = x[i];
            xv.x = fmaf(alpha, pp.x, xv.x);
            xv.y = fmaf(alpha, pp.y, xv.y);
            x[i] = xv;
        }
        double vv[1] = {0.0}, tot[1];
        const int np = gridDim.x;
        if (last_block_total<1>(vv, red.part, np, b * np + blockIdx.x, red.counter + b, tot, red_s, &flag) &&
            threadIdx.x == 0)
            st[b].state = ST_DONE;
        return;
    }
    for (int i = tid; i < NX; i += NT) tw[i] = tw_g[i];
    float2 v[16], pp[MODE == 2 ? 16 : 1], xv[MODE == 2 ? 16 : 1];
    // every load of the pass is issued before the transform: one memory latency per CTA
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        v[e] = tb[base + t + T * e];
        if constexpr (MODE == 2) {
            pp[e] = p[base + t + T * e];
            xv[e] = x[base + t + T * e];
        }
    }
    __syncthreads();
    fft_bar<NX, true>(v, t, buf, RowIdx<NX>{row}, tw, RowBar<NX>{});
    if constexpr (MODE == 0) {
#pragma unroll
        for (int e = 0; e < 16; ++e) out[base + t + T * e] = v[e];
    } else if constexpr (MODE == 1) {
#pragma unroll
        for (int e = 0; e < 16; ++e) p[base + t + T * e] = v[e];
    } else {
        const float alpha = (float)st[b].alpha, beta = (float)st[b].beta;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const size_t i = base + t + T * e;
            x[i] = make_float2(fmaf(alpha, pp[e].x, xv[e].x), fmaf(alpha, pp[e].y, xv[e].y));
            p[i] = make_float2(fmaf(beta, pp[e].x, v[e].x), fmaf(beta, pp[e].y, v[e].y));
        }
    }
}

// ------------------------------------------------------------------------------ CG without
// the circulant preconditioner: z = w r with w = 1 (plain CG) or w = 1 / diag(A) (Jacobi)
template <int MODE>
__global__ void __launch_bounds__(kVecThreads)
k_vec_plain(float2* __restrict__ x, float2* __restrict__ r, float2* __restrict__ p,
            const float2* __restrict__ q, const float* __restrict__ w, int n, SliceState* st, double tol2, Red red) {
    const int b = blockIdx.y;
    const int s = st[b].state;
    if (MODE != 2 && s != ST_ACTIVE) return;
    if (MODE == 2 && s != ST_ACTIVE && s != ST_FINISHING) return;
    __shared__ double red_s[64];
    __shared__ int flag;
    const size_t img = (size_t)b * n;
    const int i0 = blockIdx.x * kVecThreads * kVecPerThread + threadIdx.x;
    float rr = 0.f, rz = 0.f;
    if constexpr (MODE == 0) {
#pragma unroll
        for (int k = 0; k < kVecPerThread; ++k) {
            const int i = i0 + k * kVecThreads;
            if (i < n) {
                const float2 rv = r[img + i];
                const float wv = w ? w[img + i] : 1.f;
                p[img + i] = cscale(rv, wv);
                rz += wv * cabs2(rv);
            }
        }
    } else if constexpr (MODE == 1) {
        const float alpha = (float)st[b].alpha;
#pragma unroll
        for (int k = 0; k < kVecPerThread; ++k) {
            const int i = i0 + k * kVecThreads;
            if (i < n) {
                const float2 qq = q[img + i];
                float2 rv = r[img + i];
                rv.x = fmaf(-alpha, qq.x, rv.x);
                rv.y = fmaf(-alpha, qq.y, rv.y);
                r[img + i] = rv;
                const float a2 = cabs2(rv);
                rr += a2;
                rz += (w ? w[img + i] : 1.f) * a2;
            }
        }
    } else {
        const float alpha = (float)st[b].alpha, beta = (float)st[b].beta;
        const bool upd_p = (s == ST_ACTIVE);
#pragma unroll
        for (int k = 0; k < kVecPerThread; ++k) {
            const int i = i0 + k * kVecThreads;
            if (i < n) {
                const float2 pp = p[img + i];
                float2 xv = x[img + i];
                xv.x = fmaf(alpha, pp.x, xv.x);
                xv.y = fmaf(alpha, pp.y, xv.y);
                x[img + i] = xv;
                if (upd_p) {
                    const float2 zv = cscale(r[img + i], w ? w[img + i] : 1.f);
                    p[img + i] = make_float2(fmaf(beta, pp.x, zv.x), fmaf(beta, pp.y, zv.y));
                }
            }
        }
    }
    double vv[2] = {(double)rr, (double)rz}, tot[2];
    const int np = gridDim.x;
    if (last_block_total<2>(vv, red.part, np, b * np + blockIdx.x, red.counter + b, tot, red_s, &flag) &&
        threadIdx.x == 0) {
        SliceState& S = st[b];
        if (MODE == 0) {
            S.rho = tot[1];
        } else if (MODE == 1) {
            S.rnorm2 = tot[0];
            if (!isfinite(tot[0]) || !isfinite(tot[1])) S.state = ST_NONFINITE;
            else if (tot[0] <= tol2 * S.bnorm2) S.state = ST_FINISHING;
            else {
                S.beta = tot[1] / S.rho;
                S.rho = tot[1];
            }
        } else if (s == ST_FINISHING) {
            S.state = ST_DONE;
        }
    }
}

__global__ void __launch_bounds__(kVecThreads)
k_resid_init(const float2* __restrict__ bvec, const float2* __restrict__ q, float2* __restrict__ r,
             int n, SliceState* st, double tol2, Red red) {
    const int b = blockIdx.y;
    __shared__ double red_s[64];
    __shared__ int flag;
    const size_t img = (size_t)b * n;
    const int i0 = blockIdx.x * kVecThreads * kVecPerThread + threadIdx.x;
    float bb = 0.f, rr = 0.f;
#pragma unroll
    for (int k = 0; k < kVecPerThread; ++k) {
        const int i = i0 + k * kVecThreads;
        if (i < n) {
            const float2 bv = bvec[img + i], qq = q[img + i];
            const float2 rv = csub(bv, qq);
            r[img + i] = rv;
            bb += cabs2(bv);
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

__global__ void __launch_bounds__(kVecThreads)
k_zero_rhs(float2* __restrict__ x, int n, const SliceState* st) {
    const int b = blockIdx.y;
    if (st[b].state != ST_ZERO) return;
    const int i0 = blockIdx.x * kVecThreads * kVecPerThread + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kVecPerThread; ++k) {
        const int i = i0 + k * kVecThreads;
        if (i < n) x[(size_t)b * n + i] = make_float2(0.f, 0.f);
    }
}

// ------------------------------------------------------------------------------ launch helpers
template <class K>
cudaError_t prepare(K kernel, size_t smem) {
    if (smem > 48 * 1024) return set_smem_limit(kernel, (int)smem);
    return cudaSuccess;
}

template <int NY, int CT>
size_t smem_col() { return (2 * NY * CT + NY) * sizeof(float2) + 64 * sizeof(double); }
template <int NX>
size_t smem_row() { return (RY * (NX + NX / 16) + NX) * sizeof(float2) + 64 * sizeof(double); }

template <int NX>
cudaError_t row_fwd_n(const Dims& d, int mode, float2* r, const float2* q, float2* t, const float2* tw,
                      SliceState* st, double tol2, Red red, cudaStream_t s) {
    const dim3 grid(d.ny / RY, d.nb), block(RY * NX / 16);
    const size_t sm = smem_row<NX>();
    cudaError_t e;
    if (mode == 1) {
        if ((e = prepare(k_row_fwd<NX, 1>, sm)) != cudaSuccess) return e;
        k_row_fwd<NX, 1><<<grid, block, sm, s>>>(r, q, t, tw, d.ny, st, tol2, red);
    } else {
        if ((e = prepare(k_row_fwd<NX, 0>, sm)) != cudaSuccess) return e;
        k_row_fwd<NX, 0><<<grid, block, sm, s>>>(r, q, t, tw, d.ny, st, tol2, red);
    }
    return cudaGetLastError();
}

template <int NY, int CT>
cudaError_t col_precond_ct(const Dims& d, float2* t, const float* invk, const float2* tw, SliceState* st,
                           int init, Red red, cudaStream_t s) {
    const dim3 grid(d.nx / CT, d.nb), block(CT * NY / 16);
    const size_t sm = smem_col<NY, CT>();
    cudaError_t e;
    if (st) {
        if ((e = prepare(k_col_precond<NY, true, CT>, sm)) != cudaSuccess) return e;
        k_col_precond<NY, true, CT><<<grid, block, sm, s>>>(t, invk, tw, d.nx, st, init, red);
    } else {
        if ((e = prepare(k_col_precond<NY, false, CT>, sm)) != cudaSuccess) return e;
        k_col_precond<NY, false, CT><<<grid, block, sm, s>>>(t, invk, tw, d.nx, st, init, red);
    }
    return cudaGetLastError();
}

template <int NY>
cudaError_t col_precond_n(const Dims& d, float2* t, const float* invk, const float2* tw, SliceState* st,
                          int init, Red red, cudaStream_t s, int ct) {
    if (!col_tile_ok(NY, d.nx, ct)) return cudaErrorInvalidValue;
    if (ct == 8) return col_precond_ct<NY, 8>(d, t, invk, tw, st, init, red, s);
    if (ct == 32) {
        if constexpr (NY * 32 / 16 <= 1024 && 2 * NY * 32 * 8 <= 160 * 1024)
            return col_precond_ct<NY, 32>(d, t, invk, tw, st, init, red, s);
        return cudaErrorInvalidValue;
    }
    return col_precond_ct<NY, 16>(d, t, invk, tw, st, init, red, s);
}

template <int NX>
cudaError_t row_inv_n(const Dims& d, int mode, const float2* t, float2* out, float2* x, float2* p,
                      const float2* tw, SliceState* st, Red red, cudaStream_t s) {
    const dim3 grid(d.ny / RY, d.nb), block(RY * NX / 16);
    const size_t sm = smem_row<NX>();
    cudaError_t e;
    switch (mode) {
        case 0:
            if ((e = prepare(k_row_inv<NX, 0>, sm)) != cudaSuccess) return e;
            k_row_inv<NX, 0><<<grid, block, sm, s>>>(t, out, x, p, tw, d.ny, st, red);
            break;
        case 1:
            if ((e = prepare(k_row_inv<NX, 1>, sm)) != cudaSuccess) return e;
            k_row_inv<NX, 1><<<grid, block, sm, s>>>(t, out, x, p, tw, d.ny, st, red);
            break;
        default:
            if ((e = prepare(k_row_inv<NX, 2>, sm)) != cudaSuccess) return e;
            k_row_inv<NX, 2><<<grid, block, sm, s>>>(t, out, x, p, tw, d.ny, st, red);
    }
    return cudaGetLastError();
}

dim3 vec_grid(const Dims& d) {
    const int n = d.nx * d.ny;
    return dim3((n + kVecThreads * kVecPerThread - 1) / (kVecThreads * kVecPerThread), d.nb);
}

}  // namespace

cudaError_t launch_row_fwd(const Dims& d, int mode, float2* r, const float2* q, float2* t, const float2* tw_x,
                           SliceState* st, double tol2, Red red, cudaStream_t s) {
#define CALL(N) row_fwd_n<N>(d, mode, r, q, t, tw_x, st, tol2, red, s)
    switch (d.nx) {
        case 32: return CALL(32);
        case 64: return CALL(64);
        case 128: return CALL(128);
        case 256: return CALL(256);
        case 512: return CALL(512);
        case 192: return CALL(192);
        case 224: return CALL(224);
        case 320: return CALL(320);
        case 384: return CALL(384);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

bool col_tile_ok(int ny, int nx, int ct) {
    if (ct != 8 && ct != 16 && ct != 32) return false;
    if (nx % ct != 0) return false;
    // one thread per 16 values: ct * ny / 16 threads and 2 ny ct complex values of shared memory
    return ct * ny / 16 <= 1024 && 2 * (size_t)ny * ct * 8 <= 160 * 1024;
}

cudaError_t launch_col_precond(const Dims& d, float2* t, const float* invk, const float2* tw_y, SliceState* st,
                               int init, Red red, cudaStream_t s, int ct) {
#define CALL(N) col_precond_n<N>(d, t, invk, tw_y, st, init, red, s, ct)
    switch (d.ny) {
        case 32: return CALL(32);
        case 64: return CALL(64);
        case 128: return CALL(128);
        case 256: return CALL(256);
        case 512: return CALL(512);
        case 192: return CALL(192);
        case 224: return CALL(224);
        case 320: return CALL(320);
        case 384: return CALL(384);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t launch_row_inv(const Dims& d, int mode, const float2* t, float2* out, float2* x, float2* p,
                           const float2* tw_x, SliceState* st, Red red, cudaStream_t s) {
#define CALL(N) row_inv_n<N>(d, mode, t, out, x, p, tw_x, st, red, s)
    switch (d.nx) {
        case 32: return CALL(32);
        case 64: return CALL(64);
        case 128: return CALL(128);
        case 256: return CALL(256);
        case 512: return CALL(512);
        case 192: return CALL(192);
        case 224: return CALL(224);
        case 320: return CALL(320);
        case 384: return CALL(384);
        default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t launch_vec_plain(const Dims& d, int mode, float2* x, float2* r, float2* p, const float2* q,
                             const float* w, SliceState* st, double tol2, Red red, cudaStream_t s) {
    const int n = d.nx * d.ny;
    const dim3 grid = vec_grid(d);
    switch (mode) {
        case 0: k_vec_plain<0><<<grid, kVecThreads, 0, s>>>(x, r, p, q, w, n, st, tol2, red); break;
        case 1: k_vec_plain<1><<<grid, kVecThreads, 0, s>>>(x, r, p, q, w, n, st, tol2, red); break;
        default: k_vec_plain<2><<<grid, kVecThreads, 0, s>>>(x, r, p, q, w, n, st, tol2, red);
    }
    return cudaGetLastError();
}

cudaError_t launch_resid_init(const Dims& d, const float2* b, const float2* q, float2* r, SliceState* st,
                              double tol2, Red red, cudaStream_t s) {
    k_resid_init<<<vec_grid(d), kVecThreads, 0, s>>>(b, q, r, d.nx * d.ny, st, tol2, red);
    return cudaGetLastError();
}

cudaError_t launch_zero_rhs_slices(const Dims& d, float2* x, SliceState* st, cudaStream_t s) {
    k_zero_rhs<<<vec_grid(d), kVecThreads, 0, s>>>(x, d.nx * d.ny, st);
    return cudaGetLastError();
}

}  // namespace sb
