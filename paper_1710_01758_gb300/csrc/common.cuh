// Shared device helpers: complex arithmetic, small DFTs, the register-resident Stockham FFTs
// (two stages up to 256 points, three at 512, a radix-16 stage plus two shared-memory stages for
// 192, 224, 320 and 384 points), and deterministic block / cross-CTA reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sb {

// ------------------------------------------------------------------ complex helpers
// Complex addition and subtraction as packed FP32 pair instructions (add / sub .f32x2, sm_100+):
// one instruction for both components, each rounded exactly like the scalar operation, so the
// results are bitwise those of two scalar adds; the transforms are bound by instruction issue,
// and most of their arithmetic is these adds.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    unsigned long long ra, rb, rd;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
    return d;
}
// a * (s, s) for a pair (s, s) held as one float2 (packed multiply)
__device__ __forceinline__ float2 cscale2(float2 a, float2 ss) { return __fmul2_rn(a, ss); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
// acc + conj(a) * b
__device__ __forceinline__ float2 cfmac(float2 acc, float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
// multiply by W4 = -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ float2 mul_w4(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// a + W4 x and a - W4 x without forming W4 x: the product swaps x's components, which a packed
// add could only take after two moves; two scalar adds each are as cheap and give the same bits.
template <bool INV> __device__ __forceinline__ float2 add_w4(float2 a, float2 x) {
    return INV ? make_float2(a.x - x.y, a.y + x.x) : make_float2(a.x + x.y, a.y - x.x);
}
template <bool INV> __device__ __forceinline__ float2 sub_w4(float2 a, float2 x) {
    return INV ? make_float2(a.x + x.y, a.y - x.x) : make_float2(a.x - x.y, a.y + x.x);
}
// cos(2 pi m / 16) and sin(2 pi m / 16): cos(pi/8), sin(pi/8) and sqrt(1/2) are the only
// irrational values needed.
__host__ __device__ constexpr float w16_cos(int m) {
    constexpr float C1 = 0.92387953251128674f, S1 = 0.38268343236508977f, R2 = 0.70710678118654752f;
    switch (m & 15) {
        case 0: return 1.f;  case 1: return C1;  case 2: return R2;  case 3: return S1;
        case 4: return 0.f;  case 5: return -S1; case 6: return -R2; case 7: return -C1;
        case 8: return -1.f; case 9: return -C1; case 10: return -R2; case 11: return -S1;
        case 12: return 0.f; case 13: return S1; case 14: return R2; default: return C1;
    }
}
__host__ __device__ constexpr float w16_sin(int m) { return w16_cos(m - 4); }

// multiply by the constant exp(-2 pi i m / 16) (forward) or its conjugate (inverse)
template <bool INV, int M> __device__ __forceinline__ float2 mul_w16(float2 a) {
    constexpr int m = M & 15;
    if constexpr (m == 0) return a;
    else if constexpr (m == 4) return mul_w4<INV>(a);
    else if constexpr (m == 8) return make_float2(-a.x, -a.y);
    else if constexpr (m == 12) return mul_w4<!INV>(a);
    else if constexpr ((m & 3) == 2) {
        // W16^m = r (c' + i s') with r = sqrt(1/2) and c', s' = +-1: two adds and one packed
        // multiply by (r, r) instead of two multiplies and two fused multiply-adds
        constexpr float cs = w16_cos(m) > 0.f ? 1.f : -1.f;
        constexpr float sn = (INV ? w16_sin(m) : -w16_sin(m)) > 0.f ? 1.f : -1.f;
        const float2 t = make_float2(cs * a.x - sn * a.y, sn * a.x + cs * a.y);
        return __fmul2_rn(t, make_float2(0.70710678118654752f, 0.70710678118654752f));
    } else {
        constexpr float c = w16_cos(m);
        constexpr float s = INV ? w16_sin(m) : -w16_sin(m);
        return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
    }
}

// ------------------------------------------------------------------ small DFTs in registers
// Unnormalised DFT of R points, forward sign negative (INV: positive), in natural order.
template <bool INV> __device__ __forceinline__ void dft2(float2& a0, float2& a1) {
    const float2 t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

template <bool INV> __device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
    const float2 t2 = cadd(a1, a3), d = csub(a1, a3);
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = add_w4<INV>(t1, d);
    a3 = sub_w4<INV>(t1, d);
}

// dft4 of (a0, a1, W4 r2, a3): the third input arrives before its multiplication by W4
template <bool INV> __device__ __forceinline__ void dft4_w4in2(float2& a0, float2& a1, float2& r2, float2& a3) {
    const float2 t0 = add_w4<INV>(a0, r2), t1 = sub_w4<INV>(a0, r2);
    const float2 t2 = cadd(a1, a3), d = csub(a1, a3);
    a0 = cadd(t0, t2);
    r2 = csub(t0, t2);
    a1 = add_w4<INV>(t1, d);
    a3 = sub_w4<INV>(t1, d);
}

template <bool INV> __device__ __forceinline__ void dft8(float2 (&a)[8]) {
    float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    float2 o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = mul_w16<INV, 2>(o1);
    o3 = mul_w16<INV, 6>(o3);
    a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
    a[1] = cadd(e1, o1); a[5] = csub(e1, o1);
    a[2] = add_w4<INV>(e2, o2); a[6] = sub_w4<INV>(e2, o2);  // o2 times W16^4 = W4
    a[3] = cadd(e3, o3); a[7] = csub(e3, o3);
}

// 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2.
template <bool INV> __device__ __forceinline__ void dft16(float2 (&a)[16]) {
    // length-4 DFTs over n1 for each n2 (in place: a[n2 + 4 k1] holds Y[n2][k1])
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(a[n2], a[n2 + 4], a[n2 + 8], a[n2 + 12]);
    // twiddles W16^(n2 k1) (a[10]'s, W16^4 = W4, is folded into its length-4 DFT below)
    a[5] = mul_w16<INV, 1>(a[5]);  a[9] = mul_w16<INV, 2>(a[9]);   a[13] = mul_w16<INV, 3>(a[13]);
    a[6] = mul_w16<INV, 2>(a[6]);                                  a[14] = mul_w16<INV, 6>(a[14]);
    a[7] = mul_w16<INV, 3>(a[7]);  a[11] = mul_w16<INV, 6>(a[11]); a[15] = mul_w16<INV, 9>(a[15]);
    // length-4 DFTs over n2 for each k1: inputs a[4 k1 + n2], outputs X[k1 + 4 k2]
    float2 y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        // element (n2, k1) sits at a[n2 + 4 k1]
        float2 b0 = a[4 * k1], b1 = a[1 + 4 * k1], b2 = a[2 + 4 * k1], b3 = a[3 + 4 * k1];
        if (k1 == 2) dft4_w4in2<INV>(b0, b1, b2, b3);
        else dft4<INV>(b0, b1, b2, b3);
        y[k1] = b0; y[k1 + 4] = b1; y[k1 + 8] = b2; y[k1 + 12] = b3;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = y[i];
}

template <int R, bool INV> __device__ __forceinline__ void dftR(float2 (&a)[R]) {
    if constexpr (R == 2) dft2<INV>(a[0], a[1]);
    else if constexpr (R == 4) dft4<INV>(a[0], a[1], a[2], a[3]);
    else if constexpr (R == 8) dft8<INV>(a);
    else if constexpr (R == 16) dft16<INV>(a);
}

// ------------------------------------------------------------------ two-stage Stockham FFT
// An N-point transform (N = 16 * R2, R2 in {2, 4, 8, 16}) is carried by T = N/16 threads;
// thread t holds v[e] = x[t + T e], e = 0..15, and receives X[t + T e] (unnormalised DFT).
// Stage 1 is a radix-16 butterfly on the registers; its outputs go to shared memory at
// positions 16 t + r; stage 2 is radix R2 with twiddles W_N^{r j} read from `tw`
// (tw[r * 16 + j] = exp(-2 pi i r j / N), conjugated for INV) and lands back in registers.
// `idx(pos)` maps a position of this transform to its shared-memory slot.  One
// __syncthreads() separates the two stages; callers alternate two buffers between
// consecutive transforms so that no second barrier is needed.
template <int N, bool INV, class Idx>
__device__ __forceinline__ void fft_2stage(float2 (&v)[16], int t, float2* buf, Idx idx,
                                           const float2* tw) {
    constexpr int R2 = N / 16;
    constexpr int T = N / 16;
    constexpr int BF = 16 / R2;  // stage-2 butterflies per thread
    dft16<INV>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[idx(16 * t + r)] = v[r];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < BF; ++m) {
        const int j = t + T * m;
        float2 a[R2];
#pragma unroll
        for (int r = 0; r < R2; ++r) a[r] = buf[idx(j + 16 * r)];
#pragma unroll
        for (int r = 1; r < R2; ++r) {
            float2 w = tw[r * 16 + j];
            if (INV) w.y = -w.y;
            a[r] = cmul(a[r], w);
        }
        dftR<R2, INV>(a);
#pragma unroll
        for (int r = 0; r < R2; ++r) v[m + r * BF] = a[r];
    }
}

// The same transform with a caller-supplied barrier between the two stages (for transforms
// whose threads are a subset of the CTA).
template <int N, bool INV, class Idx, class Bar>
__device__ __forceinline__ void fft_2stage_bar(float2 (&v)[16], int t, float2* buf, Idx idx, const float2* tw,
                                               Bar bar) {
    constexpr int R2 = N / 16;
    constexpr int T = N / 16;
    constexpr int BF = 16 / R2;
    dft16<INV>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[idx(16 * t + r)] = v[r];
    bar();
#pragma unroll
    for (int m = 0; m < BF; ++m) {
        const int j = t + T * m;
        float2 a[R2];
#pragma unroll
        for (int r = 0; r < R2; ++r) a[r] = buf[idx(j + 16 * r)];
#pragma unroll
        for (int r = 1; r < R2; ++r) {
            float2 w = tw[r * 16 + j];
            if (INV) w.y = -w.y;
            a[r] = cmul(a[r], w);
        }
        dftR<R2, INV>(a);
#pragma unroll
        for (int r = 0; r < R2; ++r) v[m + r * BF] = a[r];
    }
}

// fft_2stage_bar for N = 256 (16 threads per transform, t < 16) with the thread's stage-2
// twiddles held in registers, twr[r - 1] = W_256^{r t} for r = 1 .. 15: it saves the transform's
// 15 shared-memory twiddle loads, at the cost of 30 registers.
template <bool INV, class Idx, class Bar>
__device__ __forceinline__ void fft256_bar_rtw(float2 (&v)[16], int t, float2* buf, Idx idx, const float2 (&twr)[15],
                                               Bar bar) {
    dft16<INV>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[idx(16 * t + r)] = v[r];
    bar();
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = buf[idx(t + 16 * r)];
#pragma unroll
    for (int r = 1; r < 16; ++r) {
        float2 w = twr[r - 1];
        if (INV) w.y = -w.y;
        v[r] = cmul(v[r], w);
    }
    dft16<INV>(v);
}

// Three-stage transform for N = 16 * 16 * R3 (N = 512: R3 = 2), T = N / 16 threads per
// transform, the same register layout (thread t holds x[t + T e] in and X[t + T e] out).
// Stage 1: radix 16 on registers; stage 2: radix 16 over the 256-point sub-transforms (span 16,
// twiddles tw[r * 16 + k] = W_256^{r k}); stage 3: radix R3 (span 256, twiddles tw[256 + k] =
// W_N^{k}) back into registers.  Both exchanges go through `buf`; `bar()` separates every
// write phase from the following reads and the stage-2 reads from the stage-2 writes.
template <int N, bool INV, class Idx, class Bar>
__device__ __forceinline__ void fft_3stage_bar(float2 (&v)[16], int t, float2* buf, Idx idx, const float2* tw,
                                               Bar bar) {
    constexpr int T = N / 16;
    constexpr int R3 = N / 256;
    constexpr int BF3 = 16 / R3;  // stage-3 butterflies per thread
    static_assert(N == 256 * R3 && T * R3 == 16 * R3 * (T / 16), "N = 16 * 16 * R3");
    // stage 1: Ns = 1, butterfly j = t, inputs x[t + T r], outputs y[16 t + r]
    dft16<INV>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[idx(16 * t + r)] = v[r];
    bar();
    // stage 2: Ns = 16, butterfly j = t, k = t % 16, inputs x[t + T r], outputs
    // y[(t / 16) * 256 + k + 16 r]
    {
        const int k = t & 15;
        float2 a[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) a[r] = buf[idx(t + T * r)];
#pragma unroll
        for (int r = 1; r < 16; ++r) {
            float2 w = tw[r * 16 + k];
            if (INV) w.y = -w.y;
            a[r] = cmul(a[r], w);
        }
        dft16<INV>(a);
        bar();  // every stage-2 read is done before the stage-2 writes
        const int base = (t >> 4) * 256 + k;
#pragma unroll
        for (int r = 0; r < 16; ++r) buf[idx(base + 16 * r)] = a[r];
    }
    bar();
    // stage 3: Ns = 256, butterflies j = t + T m, k = j, inputs x[j + 256 r], outputs y[j + 256 r]
#pragma unroll
    for (int m = 0; m < BF3; ++m) {
        const int j = t + T * m;
        float2 a[R3];
#pragma unroll
        for (int r = 0; r < R3; ++r) a[r] = buf[idx(j + 256 * r)];
#pragma unroll
        for (int r = 1; r < R3; ++r) {
            float2 w = tw[256 + (r * j) % 256];
            if (INV) w.y = -w.y;
            a[r] = cmul(a[r], w);
        }
        dftR<R3, INV>(a);
#pragma unroll
        for (int r = 0; r < R3; ++r) v[m + r * BF3] = a[r];
    }
}

// fft_3stage_bar for N = 512 (32 threads per transform) with the thread's stage-2 twiddles in
// registers, twr[r - 1] = W_256^{r (t mod 16)} for r = 1 .. 15
template <bool INV, class Idx, class Bar>
__device__ __forceinline__ void fft512_bar_rtw(float2 (&v)[16], int t, float2* buf, Idx idx, const float2* tw,
                                               const float2 (&twr)[15], Bar bar) {
    constexpr int T = 32;
    dft16<INV>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[idx(16 * t + r)] = v[r];
    bar();
    {
        const int k = t & 15;
        float2 a[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) a[r] = buf[idx(t + T * r)];
#pragma unroll
        for (int r = 1; r < 16; ++r) {
            float2 w = twr[r - 1];
            if (INV) w.y = -w.y;
            a[r] = cmul(a[r], w);
        }
        dft16<INV>(a);
        bar();  // every stage-2 read is done before the stage-2 writes
        const int base = (t >> 4) * 256 + k;
#pragma unroll
        for (int r = 0; r < 16; ++r) buf[idx(base + 16 * r)] = a[r];
    }
    bar();
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int j = t + T * m;
        float2 a0 = buf[idx(j)], a1 = buf[idx(j + 256)];
        float2 w = tw[256 + j];
        if (INV) w.y = -w.y;
        a1 = cmul(a1, w);
        dft2<INV>(a0, a1);
        v[m] = a0;
        v[m + 8] = a1;
    }
}

// ------------------------------------------------------------------ lengths 16 x {12, 14, 20, 24}
// cos and sin of 2 pi m / R for the odd radices (values of the functions, to float precision)
template <int R> __host__ __device__ constexpr float cos_r(int m);
template <int R> __host__ __device__ constexpr float sin_r(int m);
template <> __host__ __device__ constexpr float cos_r<3>(int m) { return m % 3 == 0 ? 1.f : -0.5f; }
template <> __host__ __device__ constexpr float sin_r<3>(int m) {
    return m % 3 == 0 ? 0.f : (m % 3 == 1 ? 0.86602540378443865f : -0.86602540378443865f);
}
template <> __host__ __device__ constexpr float cos_r<5>(int m) {
    switch (m % 5) {
        case 0: return 1.f; case 1: case 4: return 0.30901699437494742f; default: return -0.80901699437494742f;
    }
}
template <> __host__ __device__ constexpr float sin_r<5>(int m) {
    switch (m % 5) {
        case 0: return 0.f; case 1: return 0.95105651629515357f; case 2: return 0.58778525229247313f;
        case 3: return -0.58778525229247313f; default: return -0.95105651629515357f;
    }
}
template <> __host__ __device__ constexpr float cos_r<7>(int m) {
    switch (m % 7) {
        case 0: return 1.f; case 1: case 6: return 0.62348980185873353f;
        case 2: case 5: return -0.22252093395631440f; default: return -0.90096886790241913f;
    }
}
template <> __host__ __device__ constexpr float sin_r<7>(int m) {
    switch (m % 7) {
        case 0: return 0.f; case 1: return 0.78183148246802981f; case 2: return 0.97492791218182361f;
        case 3: return 0.43388373911755812f; case 4: return -0.43388373911755812f;
        case 5: return -0.97492791218182361f; default: return -0.78183148246802981f;
    }
}

// Odd-length DFT from the definition, folding x_j and x_{R-j}: with s_j = x_j + x_{R-j},
// d_j = x_j - x_{R-j}, A_k = x_0 + sum_j cos(2 pi j k / R) s_j and B_k = sum_j sin(..) d_j,
// X_k = A_k - i B_k and X_{R-k} = A_k + i B_k (forward; signs swapped for INV).
template <int R, bool INV> __device__ __forceinline__ void dft_odd(float2 (&a)[R]) {
    constexpr int H = (R - 1) / 2;
    float2 sj[H], dj[H];
#pragma unroll
    for (int j = 1; j <= H; ++j) {
        sj[j - 1] = cadd(a[j], a[R - j]);
        dj[j - 1] = csub(a[j], a[R - j]);
    }
    const float2 x0 = a[0];
    float2 s0 = x0;
#pragma unroll
    for (int j = 0; j < H; ++j) s0 = cadd(s0, sj[j]);
    a[0] = s0;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        float2 A = x0, B = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 1; j <= H; ++j) {
            const float c = cos_r<R>(j * k), sn = sin_r<R>(j * k);
            A = make_float2(fmaf(c, sj[j - 1].x, A.x), fmaf(c, sj[j - 1].y, A.y));
            B = make_float2(fmaf(sn, dj[j - 1].x, B.x), fmaf(sn, dj[j - 1].y, B.y));
        }
        const float2 mib = make_float2(B.y, -B.x);  // -i B
        a[k] = INV ? csub(A, mib) : cadd(A, mib);
        a[R - k] = INV ? cadd(A, mib) : csub(A, mib);
    }
}

template <int R, bool INV> __device__ __forceinline__ void dft_any(float2 (&a)[R]) {
    if constexpr (R % 2 == 1) dft_odd<R, INV>(a);
    else dftR<R, INV>(a);
}

// radices after the first radix-16 stage
template <int N> struct GenericPlan;
template <> struct GenericPlan<192> { static constexpr int R2 = 4, R3 = 3; };
template <> struct GenericPlan<224> { static constexpr int R2 = 2, R3 = 7; };
template <> struct GenericPlan<320> { static constexpr int R2 = 4, R3 = 5; };
template <> struct GenericPlan<384> { static constexpr int R2 = 8, R3 = 3; };

// One in-place Stockham stage of radix R and span NS on the shared-memory transform: butterfly
// j (of N / R, spread over the T threads, the last ones idle where T does not divide N / R)
// reads x[j + (N / R) r], applies W_{NS R}^{(j mod NS) r} = tw[(j mod NS) r N / (NS R)] with
// tw[m] = W_N^m, and writes y[(j / NS) NS R + j mod NS + NS r].  All reads finish (bar) before
// the writes, and the writes (bar) before the next stage.
template <int N, int R, int NS, int T, bool INV, class Idx, class Bar>
__device__ __forceinline__ void stockham_stage(float2* buf, Idx idx, const float2* tw, int t, Bar bar) {
    constexpr int NB = N / R;
    constexpr int PER = (NB + T - 1) / T;
    float2 a[PER][R];
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        const int j = t + T * m;
        if (PER * T == NB || j < NB) {
            const int k = j % NS;
#pragma unroll
            for (int r = 0; r < R; ++r) a[m][r] = buf[idx(j + NB * r)];
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[k * r * (N / (NS * R))];
                if (INV) w.y = -w.y;
                a[m][r] = cmul(a[m][r], w);
            }
            dft_any<R, INV>(a[m]);
        }
    }
    bar();
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        const int j = t + T * m;
        if (PER * T == NB || j < NB) {
            const int base = (j / NS) * NS * R + j % NS;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[idx(base + NS * r)] = a[m][r];
        }
    }
    bar();
}

// N = 16 x {12, 14, 20, 24}: the same register layout as the power-of-two transforms (thread t
// of T = N / 16 holds x[t + T e] in and X[t + T e] out); radix 16 on the registers, then the
// two stages of GenericPlan<N> in shared memory (tw[m] = W_N^m, m < N).
template <int N, bool INV, class Idx, class Bar>
__device__ __forceinline__ void fft_generic_bar(float2 (&v)[16], int t, float2* buf, Idx idx, const float2* tw,
                                                Bar bar) {
    constexpr int T = N / 16;
    constexpr int R2 = GenericPlan<N>::R2, R3 = GenericPlan<N>::R3;
    static_assert(16 * R2 * R3 == N, "plan covers N");
    dft16<INV>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[idx(16 * t + r)] = v[r];
    bar();
    stockham_stage<N, R2, 16, T, INV>(buf, idx, tw, t, bar);
    stockham_stage<N, R3, 16 * R2, T, INV>(buf, idx, tw, t, bar);
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = buf[idx(t + T * e)];
}

// Out-of-place form of the two shared-memory stages (src -> dst, one butterfly at a time, so only
// R values are live): the callers that can spare a second exchange buffer avoid holding every
// butterfly's values across the stage barrier.
template <int N, int R, int NS, int T, bool INV, class Idx>
__device__ __forceinline__ void stockham_stage_oop(const float2* src, float2* dst, Idx idx, const float2* tw, int t) {
    constexpr int NB = N / R;
    constexpr int PER = (NB + T - 1) / T;
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        const int j = t + T * m;
        if (PER * T == NB || j < NB) {
            const int k = j % NS;
            float2 a[R];
#pragma unroll
            for (int r = 0; r < R; ++r) a[r] = src[idx(j + NB * r)];
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[k * r * (N / (NS * R))];
                if (INV) w.y = -w.y;
                a[r] = cmul(a[r], w);
            }
            dft_any<R, INV>(a);
            const int base = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[idx(base + NS * r)] = a[r];
        }
    }
}

// fft_generic_bar with the stages out of place through buf2 (same layout as buf): three barriers
// instead of five; the result and the register layout are those of fft_generic_bar.
template <int N, bool INV, class Idx, class Bar>
__device__ __forceinline__ void fft_generic_oop_bar(float2 (&v)[16], int t, float2* buf, float2* buf2, Idx idx,
                                                    const float2* tw, Bar bar) {
    constexpr int T = N / 16;
    constexpr int R2 = GenericPlan<N>::R2, R3 = GenericPlan<N>::R3;
    static_assert(16 * R2 * R3 == N, "plan covers N");
    dft16<INV>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[idx(16 * t + r)] = v[r];
    bar();
    stockham_stage_oop<N, R2, 16, T, INV>(buf, buf2, idx, tw, t);
    bar();
    stockham_stage_oop<N, R3, 16 * R2, T, INV>(buf2, buf, idx, tw, t);
    bar();
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = buf[idx(t + T * e)];
}

__host__ __device__ constexpr bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Size dispatch: two stages for powers of two up to 256, three for 512, the generic
// mixed-radix transform for 192, 224, 320 and 384.
template <int N, bool INV, class Idx, class Bar>
__device__ __forceinline__ void fft_bar(float2 (&v)[16], int t, float2* buf, Idx idx, const float2* tw, Bar bar) {
    if constexpr (is_pow2(N) && N <= 256) fft_2stage_bar<N, INV>(v, t, buf, idx, tw, bar);
    else if constexpr (N == 512) fft_3stage_bar<N, INV>(v, t, buf, idx, tw, bar);
    else fft_generic_bar<N, INV>(v, t, buf, idx, tw, bar);
}

// fft_bar, with a second exchange buffer for the mixed-radix sizes (unused by the others)
template <int N, bool INV, class Idx, class Bar>
__device__ __forceinline__ void fft_bar2(float2 (&v)[16], int t, float2* buf, float2* buf2, Idx idx, const float2* tw,
                                         Bar bar) {
    if constexpr (is_pow2(N)) fft_bar<N, INV>(v, t, buf, idx, tw, bar);
    else fft_generic_oop_bar<N, INV>(v, t, buf, buf2, idx, tw, bar);
}

struct CtaBar {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

template <int N, bool INV, class Idx>
__device__ __forceinline__ void fft(float2 (&v)[16], int t, float2* buf, Idx idx, const float2* tw) {
    fft_bar<N, INV>(v, t, buf, idx, tw, CtaBar{});
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum K doubles over the block in a fixed order; result valid in thread 0.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* scratch /* >= 32*K */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) scratch[wid * K + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += scratch[w * K + k];
            v[k] = s;
        }
    }
}

// Cross-CTA reduction without a second launch: every CTA of slice `b` stores its block sums
// into part[(b * nparts + blockIdx.x) * K + k]; the last CTA to arrive (atomic ticket) sums all
// parts of the slice in index order and returns true with the totals in `tot` (thread 0).
// The ticket counter is reset by the last CTA, so the same counter serves the next launch.
template <int K>
__device__ __forceinline__ bool last_block_total(double (&v)[K], double* part, int nparts, int slot,
                                                 unsigned* counter, double (&tot)[K], double* scratch,
                                                 int* flag_smem) {
    block_sum<K>(v, scratch);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) part[(size_t)slot * K + k] = v[k];
        __threadfence();
        const unsigned ticket = atomicAdd(counter, 1u);
        *flag_smem = (ticket == (unsigned)nparts - 1u);
    }
    __syncthreads();
    const bool last = *flag_smem != 0;
    if (last && threadIdx.x == 0) {
        __threadfence();
        const double* base = part + (size_t)(slot - (slot % nparts)) * K;
#pragma unroll
        for (int k = 0; k < K; ++k) tot[k] = 0.0;
        for (int i = 0; i < nparts; ++i)
#pragma unroll
            for (int k = 0; k < K; ++k) tot[k] += __ldcg(base + (size_t)i * K + k);
        *counter = 0u;
    }
    return last;
}

}  // namespace sb
