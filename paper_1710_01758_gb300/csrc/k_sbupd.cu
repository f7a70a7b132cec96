// Steps 6-11 of Algorithm 1 in one pass per 32x32 tile of a slice:
//   d_a = shrink(D_a x + b_a, tau_tv),  b_a <- b_a + D_a x - d_a       (a = x, y; anisotropic TV)
//   d_w = shrink(W x + b_w, tau_w),     b_w <- b_w + W x - d_w         (orthonormal Haar W)
// and the non-data part of the next right-hand side (step 4):
//   g = lambda (D_x^H (d_x - b_x) + D_y^H (d_y - b_y)) + gamma W^H (d_w - b_w).
//
// Each thread owns a 2x2 pixel group.  The Haar transform is computed in place: a level maps
// the four values of a 2x2 group (stride s = 2^level) to the approximation (kept at the
// group's first position) and three details (kept at the other three), which is the same
// coefficient set as the Mallat layout, only arranged differently.  Level 1 runs in
// registers, the coarser levels in shared memory with one barrier per level.  A 32x32 tile is
// a union of whole Haar blocks for up to 5 levels, so tiles are independent.  b_w is stored in
// this tile-local arrangement (it is internal state; only x is an output).
//
// The TV update needs u = d - b at the +1 neighbours, which belong to neighbouring tiles; they
// are recomputed here from x and the old b (read from the `bx`/`by` buffers, written to
// `bx_new`/`by_new`), so concurrent tiles never read a value another tile is updating.
#include "common.cuh"
#include "kernels.h"

namespace sb {
namespace {

constexpr int ST = 32;  // tile edge

__device__ __forceinline__ float2 shrink(float2 z, float t) {
    const float m = sqrtf(cabs2(z));
    const float s = m > t ? (m - t) / m : 0.f;
    return cscale(z, s);
}

// forward Haar butterfly of a 2x2 group (a b / c d): approximation and x-, y-, xy-details
__device__ __forceinline__ void haar2x2(float2& a, float2& b, float2& c, float2& d) {
    const float2 s0 = cadd(a, b), d0 = csub(a, b), s1 = cadd(c, d), d1 = csub(c, d);
    a = cscale(cadd(s0, s1), 0.5f);
    b = cscale(cadd(d0, d1), 0.5f);
    c = cscale(csub(s0, s1), 0.5f);
    d = cscale(csub(d0, d1), 0.5f);
}

// inverse of haar2x2 (the matrix is symmetric and orthogonal: it is its own inverse)
__device__ __forceinline__ void ihaar2x2(float2& a, float2& b, float2& c, float2& d) { haar2x2(a, b, c, d); }

__device__ __forceinline__ float4 pack2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// TV step at tile position (ly, lx) in [0, ST]^2 from the old b_x, b_y values there: returns the
// new b values and leaves u = d - b in ux / uy
__device__ __forceinline__ void tv_point(float2 (&xs)[ST + 2][ST + 2], float2 (&ux)[ST + 1][ST + 1],
                                         float2 (&uy)[ST + 1][ST + 1], int ly, int lx, float2 bxv, float2 byv,
                                         float tau_tv, float2& bxn, float2& byn) {
    const float2 xc = xs[ly + 1][lx + 1];
    const float2 dxv = csub(xc, xs[ly + 1][lx]);  // D_x x
    const float2 dyv = csub(xc, xs[ly][lx + 1]);  // D_y x
    const float2 dx = shrink(cadd(dxv, bxv), tau_tv);
    const float2 dy = shrink(cadd(dyv, byv), tau_tv);
    bxn = csub(cadd(bxv, dxv), dx);
    byn = csub(cadd(byv, dyv), dy);
    ux[ly][lx] = csub(dx, bxn);
    uy[ly][lx] = csub(dy, byn);
}

// Memory access: each thread's 2 x 2 group of the tile interior is two 16-byte row pairs (x0 + c0
// even, nx even, buffers 16-byte aligned), read and written with float4; only the one-pixel
// periodic halo (132 positions of x, 65 of b_x / b_y) uses wrapped scalar indices.
__global__ void __launch_bounds__(256)
k_sb_update(SbFields f, int nx, int ny, const float2* __restrict__ x, int levels, float lam, float gam,
            float tau_tv, float tau_w) {
    __shared__ float2 xs[ST + 2][ST + 2];  // x, one-pixel periodic halo on every side
    __shared__ float2 ux[ST + 1][ST + 1];  // d_x - b_x (new) on the tile and its +1 halo
    __shared__ float2 uy[ST + 1][ST + 1];
    __shared__ float2 ws[ST][ST];          // Haar work area (levels >= 2)
    const int b = blockIdx.z;
    const int y0 = blockIdx.y * ST, x0 = blockIdx.x * ST;
    const int tid = threadIdx.x;
    const size_t img = (size_t)b * ny * nx;
    const int gi = tid / 16, gj = tid % 16;     // 2x2 group: rows 2gi, 2gi+1; cols 2gj, 2gj+1
    const int r0 = 2 * gi, c0 = 2 * gj;
    const size_t p00 = img + (size_t)(y0 + r0) * nx + x0 + c0;
    const size_t p10 = p00 + nx;
    {
        const float4 xa = __ldg(reinterpret_cast<const float4*>(x + p00));
        const float4 xb = __ldg(reinterpret_cast<const float4*>(x + p10));
        xs[r0 + 1][c0 + 1] = lo2(xa);
        xs[r0 + 1][c0 + 2] = hi2(xa);
        xs[r0 + 2][c0 + 1] = lo2(xb);
        xs[r0 + 2][c0 + 2] = hi2(xb);
    }
    if (tid < 4 * (ST + 1)) {  // the ring of the 34 x 34 tile: rows 0 and 33, columns 0 and 33
        int ly, lx;
        if (tid < ST + 2) { ly = 0; lx = tid; }
        else if (tid < 2 * (ST + 2)) { ly = ST + 1; lx = tid - (ST + 2); }
        else if (tid < 2 * (ST + 2) + ST) { lx = 0; ly = tid - 2 * (ST + 2) + 1; }
        else { lx = ST + 1; ly = tid - 2 * (ST + 2) - ST + 1; }
        const int gy = (y0 - 1 + ly + ny) % ny, gx = (x0 - 1 + lx + nx) % nx;
        xs[ly][lx] = x[img + (size_t)gy * nx + gx];
    }
    __syncthreads();
    float2 g4[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};

    if (lam != 0.f) {
        {  // the thread's 2 x 2 group of the interior
            const float4 bxa = reinterpret_cast<const float4*>(f.bx + p00)[0];
            const float4 bxb = reinterpret_cast<const float4*>(f.bx + p10)[0];
            const float4 bya = reinterpret_cast<const float4*>(f.by + p00)[0];
            const float4 byb = reinterpret_cast<const float4*>(f.by + p10)[0];
            float2 nx0, ny0, nx1, ny1, nx2, ny2, nx3, ny3;
            tv_point(xs, ux, uy, r0, c0, lo2(bxa), lo2(bya), tau_tv, nx0, ny0);
            tv_point(xs, ux, uy, r0, c0 + 1, hi2(bxa), hi2(bya), tau_tv, nx1, ny1);
            tv_point(xs, ux, uy, r0 + 1, c0, lo2(bxb), lo2(byb), tau_tv, nx2, ny2);
            tv_point(xs, ux, uy, r0 + 1, c0 + 1, hi2(bxb), hi2(byb), tau_tv, nx3, ny3);
            reinterpret_cast<float4*>(f.bx_new + p00)[0] = pack2(nx0, nx1);
            reinterpret_cast<float4*>(f.bx_new + p10)[0] = pack2(nx2, nx3);
            reinterpret_cast<float4*>(f.by_new + p00)[0] = pack2(ny0, ny1);
            reinterpret_cast<float4*>(f.by_new + p10)[0] = pack2(ny2, ny3);
        }
        if (tid < 2 * ST + 1) {  // the +1 halo: row ST (columns 0..ST) and column ST (rows 0..ST-1)
            const int ly = tid <= ST ? ST : tid - (ST + 1);
            const int lx = tid <= ST ? tid : ST;
            const size_t gidx = img + (size_t)((y0 + ly) % ny) * nx + (x0 + lx) % nx;
            float2 bxn, byn;
            tv_point(xs, ux, uy, ly, lx, f.bx[gidx], f.by[gidx], tau_tv, bxn, byn);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int ly = r0 + (k >> 1), lx = c0 + (k & 1);
            const float2 tv = cadd(csub(ux[ly][lx], ux[ly][lx + 1]), csub(uy[ly][lx], uy[ly + 1][lx]));
            g4[k] = cscale(tv, lam);
        }
    }

    if (gam != 0.f) {
        // pixel values of the group, then level 1 in registers
        float2 a = xs[r0 + 1][c0 + 1], bq = xs[r0 + 1][c0 + 2], c = xs[r0 + 2][c0 + 1], d = xs[r0 + 2][c0 + 2];
        if (levels >= 1) haar2x2(a, bq, c, d);
        // shrink + Bregman update of every coefficient this group holds at the finest level
        // (the approximation a is shrunk only when no coarser level follows)
        float2* bw = f.bw;
        auto upd = [&](float2& w, float2 bv) {
            const float2 dw = shrink(cadd(w, bv), tau_w);
            const float2 bn = csub(cadd(bv, w), dw);
            w = csub(dw, bn);  // u_w = d_w - b_w
            return bn;
        };
        {
            // the group's four b_w slots as two row pairs; the slot of a is rewritten unchanged
            // when a coarser level owns it (that level updates it after the next barrier)
            const float4 ba = reinterpret_cast<const float4*>(bw + p00)[0];
            const float4 bb = reinterpret_cast<const float4*>(bw + p10)[0];
            const float2 n01 = upd(bq, hi2(ba));
            const float2 n10 = upd(c, lo2(bb));
            const float2 n11 = upd(d, hi2(bb));
            const float2 n00 = levels <= 1 ? upd(a, lo2(ba)) : lo2(ba);
            reinterpret_cast<float4*>(bw + p00)[0] = pack2(n00, n01);
            reinterpret_cast<float4*>(bw + p10)[0] = pack2(n10, n11);
        }
        auto update = [&](float2& w, size_t gidx) { bw[gidx] = upd(w, bw[gidx]); };
        if (levels > 1) {
            ws[r0][c0] = a;
            __syncthreads();
            for (int l = 1; l < levels; ++l) {  // coarser levels, stride s, in place
                const int s = 1 << l, per = ST / (2 * s);
                if (tid < per * per) {
                    const int rr = (tid / per) * 2 * s, cc = (tid % per) * 2 * s;
                    float2 A = ws[rr][cc], B = ws[rr][cc + s], C = ws[rr + s][cc], D = ws[rr + s][cc + s];
                    haar2x2(A, B, C, D);
                    const size_t q = img + (size_t)(y0 + rr) * nx + x0 + cc;
                    update(B, q + s);
                    update(C, q + (size_t)s * nx);
                    update(D, q + (size_t)s * nx + s);
                    if (l == levels - 1) update(A, q);
                    ws[rr][cc] = A;
                    ws[rr][cc + s] = B;
                    ws[rr + s][cc] = C;
                    ws[rr + s][cc + s] = D;
                }
                __syncthreads();
            }
            for (int l = levels - 1; l >= 1; --l) {  // synthesis, coarsest first
                const int s = 1 << l, per = ST / (2 * s);
                if (tid < per * per) {
                    const int rr = (tid / per) * 2 * s, cc = (tid % per) * 2 * s;
                    float2 A = ws[rr][cc], B = ws[rr][cc + s], C = ws[rr + s][cc], D = ws[rr + s][cc + s];
                    ihaar2x2(A, B, C, D);
                    ws[rr][cc] = A;
                    ws[rr][cc + s] = B;
                    ws[rr + s][cc] = C;
                    ws[rr + s][cc + s] = D;
                }
                __syncthreads();
            }
            a = ws[r0][c0];
        }
        if (levels >= 1) ihaar2x2(a, bq, c, d);
        g4[0] = cadd(g4[0], cscale(a, gam));
        g4[1] = cadd(g4[1], cscale(bq, gam));
        g4[2] = cadd(g4[2], cscale(c, gam));
        g4[3] = cadd(g4[3], cscale(d, gam));
    }
    reinterpret_cast<float4*>(f.g + p00)[0] = pack2(g4[0], g4[1]);
    reinterpret_cast<float4*>(f.g + p10)[0] = pack2(g4[2], g4[3]);
}

}  // namespace

cudaError_t launch_sb_update(const Dims& d, const SbFields& f, const float2* x, int levels, float lam, float gam,
                             float tau_tv, float tau_w, cudaStream_t s) {
    if (levels > 5 || d.nx % ST || d.ny % ST) return cudaErrorInvalidValue;
    const dim3 grid(d.nx / ST, d.ny / ST, d.nb);
    k_sb_update<<<grid, 256, 0, s>>>(f, d.nx, d.ny, x, levels, lam, gam, tau_tv, tau_w);
    return cudaGetLastError();
}

}  // namespace sb
