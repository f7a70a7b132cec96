// Volumes (nz planes of ny x nx) whose mask is constant along the readout axis x: sampled
// (k_y, k_z) lines.  With R = R_yz (x) I_x the data term is F^H R F = (F_yz^H R_yz F_yz) (x) I_x
// (the readout shortcut of the 2D path, one dimension up), so every data-term operation is a
// 2D transform over (y, z) per x column, and the mask is a general 2D pattern in (k_y, k_z).
// Each operation runs as three passes through a per-coil scratch U [nb][Nc][nz][ny][nx]:
//
//  k_g3_fwd_y   U_c = DFT_y(S_c v) per plane (v = p for A, x for the right-hand side).
//  k_g3_z       DFT_z, the (k_y, k_z) mask operation, IDFT_z, per (y, x-tile) column:
//                 MODE 0 (A):    U <- IDFT_z(R DFT_z U) / (ny nz)
//                 MODE 1 (RHS):  on sampled lines tt = DFT_z U / sqrt(ny nz) (= R F_yz S x);
//                                yt <- yt + yt1 - tt (ADDBACK); U <- IDFT_z((yt - tt) / sqrt(ny nz))
//                 MODE 2 (back-projection): U <- IDFT_z(yt1 on sampled lines / sqrt(ny nz))
//  k_g3_inv_y   u_c = IDFT_y(U_c), acc = sum_c conj(S_c) u_c, then per MODE:
//                 MODE 0: q = mu acc + lam (D^H D) p + gam p (7-point periodic stencil),
//                         Re(p^H q) and alpha = rho / p^H q (last CTA of the volume)
//                 MODE 1: the Split Bregman right-hand side and initial residual (as in 2D)
//                 MODE 2: bd1 = bd = acc and, optionally, x = sqrt(sum_c |u_c|^2) (step 1)
//
// The same passes serve 2D slices with an arbitrary mask (nz = 1): k_g2_x replaces k_g3_z with
// the transform along x and a per-point mask in (k_y, k_x), the k-space data kept whole
// ([nb][Nc][ny][nx], no hybrid space); the 7-point stencil of k_g3_inv_y reduces to the 5-point
// one when nz = 1 (both z neighbours are the plane itself).
//
// k_col_dft is a plain per-plane DFT along y (the y passes of the 3D preconditioner and of the
// 3D k construction); k_sb_update3 is steps 6-11 of Algorithm 1 on 16^3 tiles (anisotropic TV
// in x, y, z and the 3D Haar transform in place, levels <= 4).
#include "common.cuh"
#include "kernels.h"

namespace sb {
namespace {

constexpr int TX = kColTile;

struct ColIdx {
    int col;
    __device__ __forceinline__ int operator()(int pos) const { return pos * TX + col; }
};

// ---------------------------------------------------------------------- y transforms per plane
template <int NY, bool INV>
__global__ void __launch_bounds__(TX * NY / 16)
k_col_dft(float2* __restrict__ data, int nx, int nz, const float2* __restrict__ tw_g, const SliceState* st) {
    constexpr int T = NY / 16;
    constexpr int NT = TX * T;
    const int plane = blockIdx.y;  // over [nb][nz]
    if (st && st[plane / nz].state != ST_ACTIVE) return;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* buf = reinterpret_cast<float2*>(smem);
    float2* tw = buf + NY * TX;
    const int tid = threadIdx.x, col = tid % TX, t = tid / TX;
    const int x = blockIdx.x * TX + col;
    for (int i = tid; i < NY; i += NT) tw[i] = tw_g[i];
    const size_t img = (size_t)plane * NY * nx;
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = data[img + (size_t)(t + T * e) * nx + x];
    __syncthreads();
    fft<NY, INV>(v, t, buf, ColIdx{col}, tw);
#pragma unroll
    for (int e = 0; e < 16; ++e) data[img + (size_t)(t + T * e) * nx + x] = v[e];
}

// ---------------------------------------------------------------------- pass A
template <int NY>
__global__ void __launch_bounds__(TX * NY / 16)
k_g3_fwd_y(const float2* __restrict__ sens, const float2* __restrict__ v, float2* __restrict__ U, int nx, int nz,
           int nc, const float2* __restrict__ tw_g, const SliceState* st) {
    constexpr int T = NY / 16;
    constexpr int NT = TX * T;
    const int z = blockIdx.y, bc = blockIdx.z, b = bc / nc;
    if (st && st[b].state != ST_ACTIVE) return;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* buf = reinterpret_cast<float2*>(smem);
    float2* tw = buf + NY * TX;
    const int tid = threadIdx.x, col = tid % TX, t = tid / TX;
    const int x = blockIdx.x * TX + col;
    for (int i = tid; i < NY; i += NT) tw[i] = tw_g[i];
    const size_t plane = (size_t)NY * nx;
    const size_t vimg = ((size_t)b * nz + z) * plane;
    const size_t simg = ((size_t)bc * nz + z) * plane;
    float2 u[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const size_t o = (size_t)(t + T * e) * nx + x;
        u[e] = cmul(__ldg(sens + simg + o), v[vimg + o]);
    }
    __syncthreads();
    fft<NY, false>(u, t, buf, ColIdx{col}, tw);
#pragma unroll
    for (int e = 0; e < 16; ++e) U[simg + (size_t)(t + T * e) * nx + x] = u[e];
}

// ---------------------------------------------------------------------- pass B (along z)
template <int NZ, int MODE, bool ADDBACK>
__global__ void __launch_bounds__(TX * NZ / 16)
k_g3_z(float2* __restrict__ U, const int* __restrict__ slot, float2* __restrict__ yt, const float2* __restrict__ yt1,
       int ms, int nx, int ny, int nc, const float2* __restrict__ tw_g, const SliceState* st) {
    constexpr int T = NZ / 16;
    constexpr int NT = TX * T;
    const int ky = blockIdx.y, bc = blockIdx.z, b = bc / nc;
    if (st && st[b].state != ST_ACTIVE) return;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* buf0 = reinterpret_cast<float2*>(smem);
    float2* buf1 = buf0 + NZ * TX;
    float2* tw = buf1 + NZ * TX;
    const int tid = threadIdx.x, col = tid % TX, t = tid / TX;
    const int x = blockIdx.x * TX + col;
    for (int i = tid; i < NZ; i += NT) tw[i] = tw_g[i];
    const size_t zs = (size_t)ny * nx;  // plane stride
    const size_t base = (size_t)bc * NZ * zs + (size_t)ky * nx + x;
    const int* sl = slot + (size_t)b * NZ * ny;
    const size_t ybase = (size_t)bc * ms * nx + x;
    const ColIdx idx{col};
    float2 u[16];
    if constexpr (MODE != 2) {
#pragma unroll
        for (int e = 0; e < 16; ++e) u[e] = U[base + (size_t)(t + T * e) * zs];
    }
    __syncthreads();
    if constexpr (MODE != 2) fft<NZ, false>(u, t, buf0, idx, tw);
    const float n_yz = (float)(ny * NZ);
    const float isq = rsqrtf(n_yz);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int s = sl[(size_t)(t + T * e) * ny + ky];
        if (s < 0) {
            u[e] = make_float2(0.f, 0.f);
        } else if constexpr (MODE == 0) {
            u[e] = cscale(u[e], 1.f / n_yz);
        } else if constexpr (MODE == 1) {
            const float2 tt = cscale(u[e], isq);
            float2 yv = yt[ybase + (size_t)s * nx];
            if (ADDBACK) {
                yv = csub(cadd(yv, yt1[ybase + (size_t)s * nx]), tt);
                yt[ybase + (size_t)s * nx] = yv;
            }
            u[e] = cscale(csub(yv, tt), isq);
        } else {
            u[e] = cscale(yt1[ybase + (size_t)s * nx], isq);
        }
    }
    fft<NZ, true>(u, t, buf1, idx, tw);
#pragma unroll
    for (int e = 0; e < 16; ++e) U[base + (size_t)(t + T * e) * zs] = u[e];
}

// ---------------------------------------------------------------------- pass B (along x, 2D)
template <int N>
struct RowIdx {
    int row;
    __device__ __forceinline__ int operator()(int pos) const { return row * (N + N / 16) + pos + (pos >> 4); }
};
constexpr int RY2 = 16;  // rows per CTA

template <int NX, int MODE, bool ADDBACK>
__global__ void __launch_bounds__(RY2 * NX / 16)
k_g2_x(float2* __restrict__ U, const uint8_t* __restrict__ mask, float2* __restrict__ yt,
       const float2* __restrict__ yt1, int ny, int nc, const float2* __restrict__ tw_g, const SliceState* st) {
    constexpr int T = NX / 16;
    constexpr int NT = RY2 * T;
    const int bc = blockIdx.y, b = bc / nc;
    if (st && st[b].state != ST_ACTIVE) return;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* buf0 = reinterpret_cast<float2*>(smem);
    float2* buf1 = buf0 + RY2 * (NX + NX / 16);
    float2* tw = buf1 + RY2 * (NX + NX / 16);
    const int tid = threadIdx.x, t = tid % T, row = tid / T;
    const int ky = blockIdx.x * RY2 + row;
    for (int i = tid; i < NX; i += NT) tw[i] = tw_g[i];
    const size_t base = ((size_t)bc * ny + ky) * NX;
    const uint8_t* m = mask + ((size_t)b * ny + ky) * NX;
    const RowIdx<NX> idx{row};
    float2 u[16];
    if constexpr (MODE != 2) {
#pragma unroll
        for (int e = 0; e < 16; ++e) u[e] = U[base + t + T * e];
    }
    __syncthreads();
    if constexpr (MODE != 2) fft<NX, false>(u, t, buf0, idx, tw);
    const float nn = (float)NX * (float)ny;
    const float isq = rsqrtf(nn);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int kx = t + T * e;
        if (!m[kx]) {
            u[e] = make_float2(0.f, 0.f);
        } else if constexpr (MODE == 0) {
            u[e] = cscale(u[e], 1.f / nn);
        } else if constexpr (MODE == 1) {
            const float2 tt = cscale(u[e], isq);
            float2 yv = yt[base + kx];
            if (ADDBACK) {
                yv = csub(cadd(yv, yt1[base + kx]), tt);
                yt[base + kx] = yv;
            }
            u[e] = cscale(csub(yv, tt), isq);
        } else {
            u[e] = cscale(yt1[base + kx], isq);
        }
    }
    fft<NX, true>(u, t, buf1, idx, tw);
#pragma unroll
    for (int e = 0; e < 16; ++e) U[base + t + T * e] = u[e];
}

// ---------------------------------------------------------------------- pass C
// 7-point periodic stencil (D_x^H D_x + D_y^H D_y + D_z^H D_z) v at (z, y, x) for element e of
// this thread: x and y neighbours from the shared tile `vt` (+ column halos), z neighbours from
// global memory
struct Stencil3 {
    const float2* vt;
    const float2* halo;
    int NYv, col;
    __device__ __forceinline__ float2 at(int y, int c) const {
        if (c < 0) return halo[y];
        if (c >= TX) return halo[NYv + y];
        return vt[y * TX + c];
    }
};

template <int NY, int MODE, bool FLAG>
__global__ void __launch_bounds__(TX * NY / 16)
k_g3_inv_y(const float2* __restrict__ U, SbFields f, int nx, int nz, int nc, const float2* __restrict__ vin,
           float2* __restrict__ out, int write_x, const float2* __restrict__ tw_g, float mu, float lam, float gam,
           SliceState* st, double tol2, Red red) {
    constexpr int T = NY / 16;
    constexpr int NT = TX * T;
    const int z = blockIdx.y, b = blockIdx.z;
    if (MODE == 0 && FLAG && st[b].state != ST_ACTIVE) return;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* buf0 = reinterpret_cast<float2*>(smem);
    float2* buf1 = buf0 + NY * TX;
    float2* tw = buf1 + NY * TX;
    float2* vt = tw + NY;       // [NY][TX] tile of v (p or x)
    float2* halo = vt + NY * TX;  // [2][NY]: columns x0 - 1 and x0 + TX
    double* red_s = reinterpret_cast<double*>(halo + 2 * NY);
    __shared__ int flag;
    const int tid = threadIdx.x, col = tid % TX, t = tid / TX;
    const int x0 = blockIdx.x * TX, x = x0 + col;
    for (int i = tid; i < NY; i += NT) tw[i] = tw_g[i];
    const size_t plane = (size_t)NY * nx;
    const size_t img = ((size_t)b * nz + z) * plane;
    __syncthreads();
    const ColIdx idx{col};
    float2 acc[16];
    float ss[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        acc[e] = make_float2(0.f, 0.f);
        ss[e] = 0.f;
    }
    for (int c = 0; c < nc; ++c) {
        const size_t cimg = (((size_t)b * nc + c) * nz + z) * plane;
        float2 u[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) u[e] = U[cimg + (size_t)(t + T * e) * nx + x];
        fft<NY, true>(u, t, (c & 1) ? buf1 : buf0, idx, tw);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            acc[e] = cfmac(acc[e], __ldg(f.sens + cimg + (size_t)(t + T * e) * nx + x), u[e]);
            if (MODE == 2) ss[e] += cabs2(u[e]);
        }
    }
    if constexpr (MODE == 2) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const size_t gi = img + (size_t)(t + T * e) * nx + x;
            f.bd1[gi] = acc[e];
            f.bd[gi] = acc[e];
            if (write_x) out[gi] = make_float2(sqrtf(ss[e]), 0.f);
        }
        return;
    } else {
        // the 7-point stencil needs v on the tile, its column halos and the planes z -+ 1
        float2 vv[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            vv[e] = vin[img + (size_t)(t + T * e) * nx + x];
            vt[(t + T * e) * TX + col] = vv[e];
        }
        for (int i = tid; i < NY; i += NT) {
            halo[i] = vin[img + (size_t)i * nx + (x0 == 0 ? nx - 1 : x0 - 1)];
            halo[NY + i] = vin[img + (size_t)i * nx + (x0 + TX == nx ? 0 : x0 + TX)];
        }
        __syncthreads();
        const size_t zm = ((size_t)b * nz + (z == 0 ? nz - 1 : z - 1)) * plane;
        const size_t zp = ((size_t)b * nz + (z == nz - 1 ? 0 : z + 1)) * plane;
        const Stencil3 S3{vt, halo, NY, col};
        float v0 = 0.f, v1 = 0.f;  // MODE 0: Re(p^H q); MODE 1: ||b||^2, ||r||^2
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int yy = t + T * e;
            const size_t o = (size_t)yy * nx + x;
            const float2 up = S3.at(yy == 0 ? NY - 1 : yy - 1, col);
            const float2 dn = S3.at(yy == NY - 1 ? 0 : yy + 1, col);
            const float2 lf = S3.at(yy, col - 1), rt = S3.at(yy, col + 1);
            const float2 zb = vin[zm + o], zf = vin[zp + o];
            const float tvx = 6.f * vv[e].x - up.x - dn.x - lf.x - rt.x - zb.x - zf.x;
            const float tvy = 6.f * vv[e].y - up.y - dn.y - lf.y - rt.y - zb.y - zf.y;
            const size_t gi = img + o;
            if constexpr (MODE == 0) {
                float2 q;
                q.x = fmaf(mu, acc[e].x, fmaf(lam, tvx, gam * vv[e].x));
                q.y = fmaf(mu, acc[e].y, fmaf(lam, tvy, gam * vv[e].y));
                out[gi] = q;
                v0 = fmaf(vv[e].x, q.x, fmaf(vv[e].y, q.y, v0));
            } else {
                const float2 gv = f.g[gi];
                float2 bdv = f.bd[gi];
                if (FLAG) {  // after an outer update: bd' = (racc + bd + bd1) / 2
                    const float2 b1 = f.bd1[gi];
                    bdv = make_float2(0.5f * (acc[e].x + bdv.x + b1.x), 0.5f * (acc[e].y + bdv.y + b1.y));
                    f.bd[gi] = bdv;
                }
                const float2 bvec = make_float2(fmaf(mu, bdv.x, gv.x), fmaf(mu, bdv.y, gv.y));
                float2 rv;
                rv.x = fmaf(mu, acc[e].x, gv.x) - fmaf(lam, tvx, gam * vv[e].x);
                rv.y = fmaf(mu, acc[e].y, gv.y) - fmaf(lam, tvy, gam * vv[e].y);
                out[gi] = rv;
                v0 += cabs2(bvec);
                v1 += cabs2(rv);
            }
        }
        const int np = gridDim.x * gridDim.y;
        const int slot = b * np + blockIdx.y * gridDim.x + blockIdx.x;
        if constexpr (MODE == 0) {
            if (!FLAG) return;
            double vd[1] = {(double)v0}, tot[1];
            if (last_block_total<1>(vd, red.part, np, slot, red.counter + b, tot, red_s, &flag) && tid == 0) {
                SliceState& S = st[b];
                const double pq = tot[0];
                S.pq = pq;
                if (!isfinite(pq) || !isfinite(S.rho)) S.state = ST_NONFINITE;
                else if (!(pq > 0.0)) S.state = ST_BREAKDOWN;
                else {
                    S.alpha = S.rho / pq;
                    S.iters += 1;
                }
            }
        } else {
            double vd[2] = {(double)v0, (double)v1}, tot[2];
            if (last_block_total<2>(vd, red.part, np, slot, red.counter + b, tot, red_s, &flag) && tid == 0) {
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
    }
}

// ---------------------------------------------------------------------- steps 6-11 in 3D
constexpr int VT = 16;  // tile edge
constexpr float kH3 = 0.35355339059327377f;  // (1/sqrt 2)^3

__device__ __forceinline__ float2 shrink3(float2 z, float t) {
    const float m = sqrtf(cabs2(z));
    const float s = m > t ? (m - t) / m : 0.f;
    return cscale(z, s);
}

// orthonormal Haar butterfly of a 2x2x2 group, v[(dz << 2) | (dy << 1) | dx]; v[0] becomes the
// approximation.  The matrix is symmetric and orthogonal, so it is also its own inverse.
__device__ __forceinline__ void haar8(float2 (&v)[8]) {
#pragma unroll
    for (int m = 1; m < 8; m <<= 1)
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (!(i & m)) {
                const float2 a = v[i], c = v[i | m];
                v[i] = cadd(a, c);
                v[i | m] = csub(a, c);
            }
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = cscale(v[i], kH3);
}

struct Sb3Smem {
    float2 xs[VT + 2][VT + 2][VT + 2];  // x with a one-voxel periodic halo
    union {
        struct {
            float2 ux[VT][VT][VT + 1];  // d_x - b_x (new) on the tile and its +1 halo in x
            float2 uy[VT][VT + 1][VT];
            float2 uz[VT + 1][VT][VT];
        } tv;
        float2 ws[VT][VT][VT];  // Haar work area (levels >= 2)
    } u;
};

__global__ void __launch_bounds__(512)
k_sb_update3(SbFields f, int nx, int ny, int nz, const float2* __restrict__ x, int levels, float lam, float gam,
             float tau_tv, float tau_w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sb3Smem& sm = *reinterpret_cast<Sb3Smem*>(smem_raw);
    const int tz = nz / VT;
    const int b = blockIdx.z / tz;
    const int z0 = (blockIdx.z % tz) * VT, y0 = blockIdx.y * VT, x0 = blockIdx.x * VT;
    const int tid = threadIdx.x;
    const size_t img = (size_t)b * nz * ny * nx;
    auto gidx = [&](int gz, int gy, int gx) { return img + ((size_t)gz * ny + gy) * nx + gx; };
    for (int i = tid; i < (VT + 2) * (VT + 2) * (VT + 2); i += 512) {
        const int lz = i / ((VT + 2) * (VT + 2)), ly = (i / (VT + 2)) % (VT + 2), lx = i % (VT + 2);
        sm.xs[lz][ly][lx] = x[gidx((z0 - 1 + lz + nz) % nz, (y0 - 1 + ly + ny) % ny, (x0 - 1 + lx + nx) % nx)];
    }
    __syncthreads();
    // this thread's 2x2x2 group
    const int gz = 2 * (tid / 64), gy = 2 * ((tid / 8) % 8), gx = 2 * (tid % 8);
    float2 g8[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) g8[k] = make_float2(0.f, 0.f);

    if (lam != 0.f) {
        // one direction at a time: the tile plus a +1 halo along that direction
        auto tv_dir = [&](int dir) {
            const int ex = dir == 0, ey = dir == 1, ez = dir == 2;
            const int nxl = VT + ex, nyl = VT + ey, nzl = VT + ez;
            const float2* bo = dir == 0 ? f.bx : (dir == 1 ? f.by : f.bz);
            float2* bn_out = dir == 0 ? f.bx_new : (dir == 1 ? f.by_new : f.bz_new);
            for (int i = tid; i < nxl * nyl * nzl; i += 512) {
                const int lz = i / (nxl * nyl), ly = (i / nxl) % nyl, lx = i % nxl;
                const float2 xc = sm.xs[lz + 1][ly + 1][lx + 1];
                const float2 xm = sm.xs[lz + 1 - ez][ly + 1 - ey][lx + 1 - ex];
                const float2 dv = csub(xc, xm);  // D_a x (backward difference)
                const size_t g = gidx((z0 + lz) % nz, (y0 + ly) % ny, (x0 + lx) % nx);
                const float2 bv = bo[g];
                const float2 dd = shrink3(cadd(dv, bv), tau_tv);
                const float2 bn = csub(cadd(bv, dv), dd);
                const float2 uu = csub(dd, bn);
                if (dir == 0) sm.u.tv.ux[lz][ly][lx] = uu;
                else if (dir == 1) sm.u.tv.uy[lz][ly][lx] = uu;
                else sm.u.tv.uz[lz][ly][lx] = uu;
                if (lx < VT && ly < VT && lz < VT) bn_out[g] = bn;
            }
        };
        tv_dir(0);
        tv_dir(1);
        tv_dir(2);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int lz = gz + (k >> 2), ly = gy + ((k >> 1) & 1), lx = gx + (k & 1);
            const float2 a = csub(sm.u.tv.ux[lz][ly][lx], sm.u.tv.ux[lz][ly][lx + 1]);
            const float2 bq = csub(sm.u.tv.uy[lz][ly][lx], sm.u.tv.uy[lz][ly + 1][lx]);
            const float2 c = csub(sm.u.tv.uz[lz][ly][lx], sm.u.tv.uz[lz + 1][ly][lx]);
            g8[k] = cscale(cadd(cadd(a, bq), c), lam);
        }
        __syncthreads();  // the TV area is reused by the Haar levels below
    }

    if (gam != 0.f) {
        float2 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = sm.xs[gz + (k >> 2) + 1][gy + ((k >> 1) & 1) + 1][gx + (k & 1) + 1];
        float2* bw = f.bw;
        auto update = [&](float2& w, size_t g) {
            const float2 bv = bw[g];
            const float2 dw = shrink3(cadd(w, bv), tau_w);
            const float2 bn = csub(cadd(bv, w), dw);
            bw[g] = bn;
            w = csub(dw, bn);  // u_w = d_w - b_w
        };
        auto pos = [&](int lz, int ly, int lx) { return gidx(z0 + lz, y0 + ly, x0 + lx); };
        if (levels >= 1) haar8(v);
        // details of level 1 (or, without levels, the voxels themselves)
#pragma unroll
        for (int k = 1; k < 8; ++k) update(v[k], pos(gz + (k >> 2), gy + ((k >> 1) & 1), gx + (k & 1)));
        if (levels <= 1) {
            update(v[0], pos(gz, gy, gx));
        } else {
            sm.u.ws[gz][gy][gx] = v[0];
            __syncthreads();
            for (int l = 1; l < levels; ++l) {  // coarser levels, stride s, in place
                const int s = 1 << l, per = VT / (2 * s);
                if (tid < per * per * per) {
                    const int bz = (tid / (per * per)) * 2 * s, by = ((tid / per) % per) * 2 * s,
                              bx = (tid % per) * 2 * s;
                    float2 w[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) w[k] = sm.u.ws[bz + (k >> 2) * s][by + ((k >> 1) & 1) * s][bx + (k & 1) * s];
                    haar8(w);
#pragma unroll
                    for (int k = 1; k < 8; ++k)
                        update(w[k], pos(bz + (k >> 2) * s, by + ((k >> 1) & 1) * s, bx + (k & 1) * s));
                    if (l == levels - 1) update(w[0], pos(bz, by, bx));
#pragma unroll
                    for (int k = 0; k < 8; ++k) sm.u.ws[bz + (k >> 2) * s][by + ((k >> 1) & 1) * s][bx + (k & 1) * s] = w[k];
                }
                __syncthreads();
            }
            for (int l = levels - 1; l >= 1; --l) {  // synthesis, coarsest first
                const int s = 1 << l, per = VT / (2 * s);
                if (tid < per * per * per) {
                    const int bz = (tid / (per * per)) * 2 * s, by = ((tid / per) % per) * 2 * s,
                              bx = (tid % per) * 2 * s;
                    float2 w[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) w[k] = sm.u.ws[bz + (k >> 2) * s][by + ((k >> 1) & 1) * s][bx + (k & 1) * s];
                    haar8(w);
#pragma unroll
                    for (int k = 0; k < 8; ++k) sm.u.ws[bz + (k >> 2) * s][by + ((k >> 1) & 1) * s][bx + (k & 1) * s] = w[k];
                }
                __syncthreads();
            }
            v[0] = sm.u.ws[gz][gy][gx];
        }
        if (levels >= 1) haar8(v);
#pragma unroll
        for (int k = 0; k < 8; ++k) g8[k] = cadd(g8[k], cscale(v[k], gam));
    }
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        const size_t g = gidx(z0 + gz + (k >> 2), y0 + gy + ((k >> 1) & 1), x0 + gx);
        reinterpret_cast<float4*>(f.g + g)[0] = make_float4(g8[k].x, g8[k].y, g8[k + 1].x, g8[k + 1].y);
    }
}

// ---------------------------------------------------------------------- launch helpers
template <class K>
cudaError_t prep(K kernel, size_t smem) {
    if (smem > 48 * 1024) return set_smem_limit(kernel, (int)smem);
    return cudaSuccess;
}

template <int NY, bool INV>
cudaError_t col_dft_n(int nx, int nplanes, int nz, float2* data, const float2* tw, const SliceState* st,
                      cudaStream_t s) {
    const size_t sm = (NY * TX + NY) * sizeof(float2);
    cudaError_t e = prep(k_col_dft<NY, INV>, sm);
    if (e != cudaSuccess) return e;
    k_col_dft<NY, INV><<<dim3(nx / TX, nplanes), TX * NY / 16, sm, s>>>(data, nx, nz, tw, st);
    return cudaGetLastError();
}

template <int NY>
cudaError_t fwd_y_n(const Dims& d, int nz, const float2* sens, const float2* v, float2* U, const float2* tw,
                    const SliceState* st, cudaStream_t s) {
    const size_t sm = (NY * TX + NY) * sizeof(float2);
    cudaError_t e = prep(k_g3_fwd_y<NY>, sm);
    if (e != cudaSuccess) return e;
    k_g3_fwd_y<NY><<<dim3(d.nx / TX, nz, d.nb * d.nc), TX * NY / 16, sm, s>>>(sens, v, U, d.nx, nz, d.nc, tw, st);
    return cudaGetLastError();
}

template <int NZ, int MODE, bool AB>
cudaError_t z_n(const Dims& d, float2* U, const int* slot, float2* yt, const float2* yt1, int ms, const float2* tw,
                const SliceState* st, cudaStream_t s) {
    const size_t sm = (2 * NZ * TX + NZ) * sizeof(float2);
    cudaError_t e = prep(k_g3_z<NZ, MODE, AB>, sm);
    if (e != cudaSuccess) return e;
    k_g3_z<NZ, MODE, AB><<<dim3(d.nx / TX, d.ny, d.nb * d.nc), TX * NZ / 16, sm, s>>>(U, slot, yt, yt1, ms, d.nx,
                                                                                        d.ny, d.nc, tw, st);
    return cudaGetLastError();
}

template <int NY, int MODE, bool FLAG>
cudaError_t inv_y_n(const Dims& d, int nz, const float2* U, const SbFields& f, const float2* vin, float2* out,
                    int write_x, const float2* tw, float mu, float lam, float gam, SliceState* st, double tol2,
                    Red red, cudaStream_t s) {
    const size_t sm = (3 * NY * TX + 3 * NY) * sizeof(float2) + 64 * sizeof(double);
    cudaError_t e = prep(k_g3_inv_y<NY, MODE, FLAG>, sm);
    if (e != cudaSuccess) return e;
    k_g3_inv_y<NY, MODE, FLAG><<<dim3(d.nx / TX, nz, d.nb), TX * NY / 16, sm, s>>>(
        U, f, d.nx, nz, d.nc, vin, out, write_x, tw, mu, lam, gam, st, tol2, red);
    return cudaGetLastError();
}

template <int NX, int MODE, bool AB>
cudaError_t x_n(const Dims& d, float2* U, const uint8_t* mask, float2* yt, const float2* yt1, const float2* tw,
                const SliceState* st, cudaStream_t s) {
    const size_t sm = (2 * RY2 * (NX + NX / 16) + NX) * sizeof(float2);
    cudaError_t e = prep(k_g2_x<NX, MODE, AB>, sm);
    if (e != cudaSuccess) return e;
    k_g2_x<NX, MODE, AB><<<dim3(d.ny / RY2, d.nb * d.nc), RY2 * NX / 16, sm, s>>>(U, mask, yt, yt1, d.ny, d.nc, tw, st);
    return cudaGetLastError();
}

#define VOL_SIZES(X) X(32) X(64) X(128) X(192) X(224) X(256) X(320) X(384) X(512)

}  // namespace

cudaError_t launch_col_dft(int nx, int ny, int nplanes, int nz, float2* data, const float2* tw_y, bool inv,
                           const SliceState* st, cudaStream_t s) {
    switch (ny) {
#define C_(N) \
    case N: return inv ? col_dft_n<N, true>(nx, nplanes, nz, data, tw_y, st, s) : col_dft_n<N, false>(nx, nplanes, nz, data, tw_y, st, s);
        VOL_SIZES(C_)
#undef C_
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_g3_fwd_y(const Dims& d, int nz, const float2* sens, const float2* v, float2* U, const float2* tw_y,
                            const SliceState* st, cudaStream_t s) {
    switch (d.ny) {
#define C_(N) \
    case N: return fwd_y_n<N>(d, nz, sens, v, U, tw_y, st, s);
        VOL_SIZES(C_)
#undef C_
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_g3_z(const Dims& d, int nz, int mode, int addback, float2* U, const int* slot, float2* yt,
                        const float2* yt1, int ms, const float2* tw_z, const SliceState* st, cudaStream_t s) {
    switch (nz) {
#define C_(N)                                                                      \
    case N:                                                                        \
        if (mode == 0) return z_n<N, 0, false>(d, U, slot, yt, yt1, ms, tw_z, st, s); \
        if (mode == 2) return z_n<N, 2, false>(d, U, slot, yt, yt1, ms, tw_z, st, s); \
        return addback ? z_n<N, 1, true>(d, U, slot, yt, yt1, ms, tw_z, st, s)         \
                       : z_n<N, 1, false>(d, U, slot, yt, yt1, ms, tw_z, st, s);
        VOL_SIZES(C_)
#undef C_
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_g2_x(const Dims& d, int mode, int addback, float2* U, const uint8_t* mask, float2* yt,
                        const float2* yt1, const float2* tw_x, const SliceState* st, cudaStream_t s) {
    switch (d.nx) {
#define C_(N)                                                                   \
    case N:                                                                     \
        if (mode == 0) return x_n<N, 0, false>(d, U, mask, yt, yt1, tw_x, st, s); \
        if (mode == 2) return x_n<N, 2, false>(d, U, mask, yt, yt1, tw_x, st, s); \
        return addback ? x_n<N, 1, true>(d, U, mask, yt, yt1, tw_x, st, s)         \
                       : x_n<N, 1, false>(d, U, mask, yt, yt1, tw_x, st, s);
        VOL_SIZES(C_)
#undef C_
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_g3_inv_y(const Dims& d, int nz, int mode, int flag, const float2* U, const SbFields& f,
                            const float2* vin, float2* out, int write_x, const float2* tw_y, float mu, float lam,
                            float gam, SliceState* st, double tol2, Red red, cudaStream_t s) {
    switch (d.ny) {
#define C_(N)                                                                                                   \
    case N:                                                                                                     \
        if (mode == 0)                                                                                          \
            return flag ? inv_y_n<N, 0, true>(d, nz, U, f, vin, out, write_x, tw_y, mu, lam, gam, st, tol2, red, s) \
                        : inv_y_n<N, 0, false>(d, nz, U, f, vin, out, write_x, tw_y, mu, lam, gam, st, tol2, red, s); \
        if (mode == 1)                                                                                          \
            return flag ? inv_y_n<N, 1, true>(d, nz, U, f, vin, out, write_x, tw_y, mu, lam, gam, st, tol2, red, s) \
                        : inv_y_n<N, 1, false>(d, nz, U, f, vin, out, write_x, tw_y, mu, lam, gam, st, tol2, red, s); \
        return inv_y_n<N, 2, false>(d, nz, U, f, vin, out, write_x, tw_y, mu, lam, gam, st, tol2, red, s);
        VOL_SIZES(C_)
#undef C_
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sb_update3(const Dims& d, int nz, const SbFields& f, const float2* x, int levels, float lam,
                              float gam, float tau_tv, float tau_w, cudaStream_t s) {
    if (levels > 4 || d.nx % VT || d.ny % VT || nz % VT) return cudaErrorInvalidValue;
    const size_t sm = sizeof(Sb3Smem);
    cudaError_t e = prep(k_sb_update3, sm);
    if (e != cudaSuccess) return e;
    k_sb_update3<<<dim3(d.nx / VT, d.ny / VT, d.nb * (nz / VT)), 512, sm, s>>>(f, d.nx, d.ny, nz, x, levels, lam, gam,
                                                                             tau_tv, tau_w);
    return cudaGetLastError();
}

}  // namespace sb
