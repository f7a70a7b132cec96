// One preconditioned-CG step after q = A p in a single launch (Theory, "Preconditioner":
// M^{-1} = F^H diag(k)^{-1} F; the CG recurrences are the textbook PCG the paper cites):
//
//   r -= alpha q,  ||r||^2 and the convergence test,
//   R = F2 r (2D DFT),  rho' = sum |R|^2 / (N k) = r^H M^{-1} r,  z = F2^H (R / (N k)),
//   beta = rho' / rho,  x += alpha p,  p = z + beta p.
//
// Each slice belongs to one thread-block cluster of C CTAs.  CTA c holds rows
// [c ny/C, (c+1) ny/C) for the transforms along x and columns [c nx/C, (c+1) nx/C) for the
// transforms along y; the two transposes between them read the other CTAs' shared memory
// directly (distributed shared memory), so the 2D spectrum never travels through HBM.  HBM
// sees r and q read, r written, 1/k read, x and p read and written: 60 B per pixel instead of
// the ~104 B of three separate passes.
//
// Cluster-wide sums: each CTA publishes its FP64 block sum in its own shared memory and every
// CTA adds the C partial sums in rank order, so all CTAs of a cluster hold bit-identical totals
// and take the same branch.  Every CTA of a cluster passes the same cluster barriers; a CTA
// leaves only after the last barrier that follows remote reads of its shared memory.
//
// MODE 0 starts CG: z = M^{-1} r, rho = r^H z, p = z (no r or x update).
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace sb {
namespace {

// launch shape of a slice of NX x NY pixels: 512 threads per CTA from 128 x 128 up
template <int NX, int NY>
struct Fused {
    static constexpr int kPix = NX * NY / 16;             // threads for one element per 16 pixels
    static constexpr int C = kPix / 512 < 1 ? 1 : kPix / 512;  // CTAs per slice (cluster size)
    static constexpr int RY = NY / C;                      // rows per CTA (x transforms)
    static constexpr int W = NX / C;                       // columns per CTA (y transforms)
    static constexpr int TXr = NX / 16;                    // threads per x transform
    static constexpr int TYc = NY / 16;                    // threads per y transform
    static constexpr int NT = RY * TXr;                    // threads per CTA
    static constexpr int RS = NX + NX / 16;                // padded row stride of the row buffer
    static_assert(NT == W * TYc, "row and column phases use the same threads");
    static_assert(C >= 1 && C <= 8 && RY >= 1 && W >= 16, "portable cluster sizes only");
    static constexpr size_t smem = (2 + 32) * sizeof(double) +
                                   ((size_t)RY * RS + (size_t)NY * W + NX + NY) * sizeof(float2);
};

// position -> index in the row buffer (padded row-major, one pad slot per 16 positions)
struct RowPos {
    int base;
    __device__ __forceinline__ int operator()(int pos) const { return base + pos + (pos >> 4); }
};
// position -> index in the column buffer ([NY][W], column `col`)
template <int W>
struct ColPos {
    int col;
    __device__ __forceinline__ int operator()(int pos) const { return pos * W + col; }
};

template <int NX, int NY, int MODE>
__global__ void __launch_bounds__(Fused<NX, NY>::NT, 1)
k_precond_fused(float2* __restrict__ x, float2* __restrict__ r, float2* __restrict__ p,
                const float2* __restrict__ q, const float* __restrict__ invk, const float2* __restrict__ twx_g,
                const float2* __restrict__ twy_g, SliceState* st, double tol2) {
    using F = Fused<NX, NY>;
    constexpr int C = F::C, RY = F::RY, W = F::W, TXr = F::TXr, TYc = F::TYc, NT = F::NT, RS = F::RS;
    const int b = blockIdx.y;
    // every CTA of the cluster reads the slice state before any of them passes the first
    // cluster barrier (the only writes come after it), so all take the same branch here
    if (st[b].state != ST_ACTIVE) return;
    const double alpha = st[b].alpha, rho = st[b].rho, bnorm2 = st[b].bnorm2;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();

    extern __shared__ __align__(16) unsigned char smem[];
    double* part = reinterpret_cast<double*>(smem);  // [0] ||r||^2, [1] r^H z of this CTA
    double* red_s = part + 2;                        // block_sum scratch (32 doubles)
    float2* rbuf = reinterpret_cast<float2*>(red_s + 32);  // [RY][RS] rows (x transforms)
    float2* cbuf = rbuf + RY * RS;                   // [NY][W] columns (y transforms)
    float2* twx = cbuf + NY * W;
    float2* twy = twx + NX;

    const int tid = threadIdx.x;
    for (int i = tid; i < NX; i += NT) twx[i] = twx_g[i];
    for (int i = tid; i < NY; i += NT) twy[i] = twy_g[i];

    // ---- rows: r update, DFT along x
    const int row = tid / TXr, t = tid % TXr;
    const size_t img = (size_t)b * NX * NY;
    const size_t rbase = img + (size_t)(rank * RY + row) * NX;
    const float af = (float)alpha;
    float2 v[16];
    float rr = 0.f;
    if constexpr (MODE == 1) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const size_t i = rbase + t + TXr * e;
            const float2 qq = q[i];
            float2 rv = r[i];
            rv.x = fmaf(-af, qq.x, rv.x);
            rv.y = fmaf(-af, qq.y, rv.y);
            r[i] = rv;
            v[e] = rv;
            rr += cabs2(rv);
        }
    } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = r[rbase + t + TXr * e];
    }
    __syncthreads();  // twiddles
    const RowPos rpos{row * RS};
    fft<NX, false>(v, t, rbuf, rpos, twx);
    __syncthreads();  // the transform's last exchange reads are done
#pragma unroll
    for (int e = 0; e < 16; ++e) rbuf[rpos(t + TXr * e)] = v[e];
    if constexpr (MODE == 1) {
        double vv[1] = {(double)rr};
        block_sum<1>(vv, red_s);
        if (tid == 0) part[0] = vv[0];
    }
    cluster.sync();  // row spectra and ||r||^2 partial sums are visible to the cluster

    double rr_tot = 0.0;
    if constexpr (MODE == 1) {
#pragma unroll
        for (int k = 0; k < C; ++k) rr_tot += *cluster.map_shared_rank(part, k);
        const bool finite = isfinite(rr_tot);
        if (!finite || rr_tot <= tol2 * bnorm2) {
            // converged (or broken): the last step x += alpha p, no new direction
            if (finite) {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const size_t i = rbase + t + TXr * e;
                    const float2 pp = p[i];
                    float2 xv = x[i];
                    xv.x = fmaf(af, pp.x, xv.x);
                    xv.y = fmaf(af, pp.y, xv.y);
                    x[i] = xv;
                }
            }
            if (rank == 0 && tid == 0) {
                st[b].rnorm2 = rr_tot;
                st[b].state = finite ? ST_DONE : ST_NONFINITE;
            }
            cluster.sync();  // no CTA leaves while another may still read its partial sum
            return;
        }
    }

    // ---- columns: gather from the cluster, DFT along y, 1/(N k), inverse DFT along y
    const int cl = tid % W, ty = tid / W;
    const int kx = rank * W + cl;
    const int kxo = kx + (kx >> 4);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int yy = ty + TYc * e;
        const float2* src = cluster.map_shared_rank(rbuf, yy / RY);
        v[e] = src[(yy % RY) * RS + kxo];
    }
    const ColPos<W> cpos{cl};
    fft<NY, false>(v, ty, cbuf, cpos, twy);
    float rz = 0.f;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const float w = __ldg(invk + img + (size_t)(ty + TYc * e) * NX + kx);
        rz = fmaf(cabs2(v[e]), w, rz);
        v[e] = cscale(v[e], w);
    }
    __syncthreads();  // a column's threads span warps: the forward exchange reads end before the inverse writes
    fft<NY, true>(v, ty, cbuf, cpos, twy);
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) cbuf[cpos(ty + TYc * e)] = v[e];
    {
        double vv[1] = {(double)rz};
        block_sum<1>(vv, red_s);
        if (tid == 0) part[1] = vv[0];
    }
    cluster.sync();  // column results and r^H z partial sums are visible; rbuf is free again

    double rz_tot = 0.0;
#pragma unroll
    for (int k = 0; k < C; ++k) rz_tot += *cluster.map_shared_rank(part + 1, k);
    // ---- rows again: gather, inverse DFT along x, CG updates
    const int yg = rank * RY + row;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int kx2 = t + TXr * e;
        const float2* src = cluster.map_shared_rank(cbuf, kx2 / W);
        v[e] = src[yg * W + (kx2 % W)];
    }
    cluster.sync();  // every remote read of this CTA's shared memory is done
    if (!isfinite(rz_tot)) {
        if (rank == 0 && tid == 0) {
            if (MODE == 1) st[b].rnorm2 = rr_tot;
            st[b].state = ST_NONFINITE;
        }
        return;
    }
    fft<NX, true>(v, t, rbuf, rpos, twx);
    if constexpr (MODE == 1) {
        const double beta = rz_tot / rho;
        const float bf = (float)beta;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const size_t i = rbase + t + TXr * e;
            const float2 pp = p[i];
            float2 xv = x[i];
            xv.x = fmaf(af, pp.x, xv.x);
            xv.y = fmaf(af, pp.y, xv.y);
            x[i] = xv;
            p[i] = make_float2(fmaf(bf, pp.x, v[e].x), fmaf(bf, pp.y, v[e].y));
        }
        if (rank == 0 && tid == 0) {
            st[b].rnorm2 = rr_tot;
            st[b].beta = beta;
            st[b].rho = rz_tot;
        }
    } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) p[rbase + t + TXr * e] = v[e];
        if (rank == 0 && tid == 0) st[b].rho = rz_tot;
    }
}

// launch (clusters == nullptr) or report how many clusters of this shape can be resident
template <int NX, int NY, int MODE>
cudaError_t fused_n(const Dims& d, float2* x, float2* r, float2* p, const float2* q, const float* invk,
                    const float2* twx, const float2* twy, SliceState* st, double tol2, cudaStream_t s,
                    int* clusters) {
    using F = Fused<NX, NY>;
    auto kern = k_precond_fused<NX, NY, MODE>;
    cudaError_t e = set_smem_limit(kern, (int)F::smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(F::C, d.nb);
    cfg.blockDim = dim3(F::NT);
    cfg.dynamicSmemBytes = F::smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = F::C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (clusters) return cudaOccupancyMaxActiveClusters(clusters, kern, &cfg);
    return cudaLaunchKernelEx(&cfg, kern, x, r, p, q, invk, twx, twy, st, tol2);
}

template <int NX, int NY>
cudaError_t fused_mode(const Dims& d, int mode, float2* x, float2* r, float2* p, const float2* q,
                       const float* invk, const float2* twx, const float2* twy, SliceState* st, double tol2,
                       cudaStream_t s, int* clusters) {
    return mode == 0 ? fused_n<NX, NY, 0>(d, x, r, p, q, invk, twx, twy, st, tol2, s, clusters)
                     : fused_n<NX, NY, 1>(d, x, r, p, q, invk, twx, twy, st, tol2, s, clusters);
}

template <int NX>
cudaError_t fused_ny(const Dims& d, int mode, float2* x, float2* r, float2* p, const float2* q,
                     const float* invk, const float2* twx, const float2* twy, SliceState* st, double tol2,
                     cudaStream_t s, int* clusters) {
    switch (d.ny) {
        case 32: return fused_mode<NX, 32>(d, mode, x, r, p, q, invk, twx, twy, st, tol2, s, clusters);
        case 64: return fused_mode<NX, 64>(d, mode, x, r, p, q, invk, twx, twy, st, tol2, s, clusters);
        case 128: return fused_mode<NX, 128>(d, mode, x, r, p, q, invk, twx, twy, st, tol2, s, clusters);
        case 256: return fused_mode<NX, 256>(d, mode, x, r, p, q, invk, twx, twy, st, tol2, s, clusters);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t fused_dispatch(const Dims& d, int mode, float2* x, float2* r, float2* p, const float2* q,
                           const float* invk, const float2* twx, const float2* twy, SliceState* st, double tol2,
                           cudaStream_t s, int* clusters) {
    switch (d.nx) {
        case 32: return fused_ny<32>(d, mode, x, r, p, q, invk, twx, twy, st, tol2, s, clusters);
        case 64: return fused_ny<64>(d, mode, x, r, p, q, invk, twx, twy, st, tol2, s, clusters);
        case 128: return fused_ny<128>(d, mode, x, r, p, q, invk, twx, twy, st, tol2, s, clusters);
        case 256: return fused_ny<256>(d, mode, x, r, p, q, invk, twx, twy, st, tol2, s, clusters);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool precond_fused_shape_ok(const Dims& d) {
    auto ok = [](int n) { return n == 32 || n == 64 || n == 128 || n == 256; };
    return ok(d.nx) && ok(d.ny);
}

int precond_fused_clusters(const Dims& d) {
    if (!precond_fused_shape_ok(d)) return 0;
    int n0 = 0, n1 = 0;
    if (fused_dispatch(d, 0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, nullptr,
                       &n0) != cudaSuccess ||
        fused_dispatch(d, 1, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, nullptr,
                       &n1) != cudaSuccess) {
        cudaGetLastError();  // a refused query is an answer, not a sticky error
        return 0;
    }
    return n0 < n1 ? n0 : n1;
}

cudaError_t launch_precond_fused(const Dims& d, int mode, float2* x, float2* r, float2* p, const float2* q,
                                 const float* invk, const float2* tw_x, const float2* tw_y, SliceState* st,
                                 double tol2, cudaStream_t s) {
    return fused_dispatch(d, mode, x, r, p, q, invk, tw_x, tw_y, st, tol2, s, nullptr);
}

}  // namespace sb
