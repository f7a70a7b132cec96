// Coil compression (Methods, "Coil Compression"; Discussion): the coil data and the coil
// sensitivity maps are mapped onto virtual coils by a compression matrix built from the
// principal components of the coil data, and only the nv most dominant virtual coils are kept.
//
//   C = sum over all samples of y y^H         (Nc x Nc, Hermitian)  k_coil_cov, k_coil_cov_reduce
//   C = V diag(s) V^H, s descending           cyclic complex Jacobi on the host, FP64
//   A = V[:, :nv]^H                           (nv x Nc)
//   y_v = A y,  S_v = A S                     k_coil_project
//
// A virtual coil is defined up to a unit phase (its eigenvector's); the reconstruction does not
// depend on it.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "sb.h"

namespace sb {
namespace {

constexpr int kChunk = 128;    // samples per CTA of the covariance kernel
constexpr int kMaxCoils = 32;

// partial covariance of one chunk: part[(b * nchunks + chunk) * npairs + pair] for the pairs
// c <= d in row order, C[c][d] = sum_i y_c[i] conj(y_d[i]); FP32 inside the chunk
__global__ void __launch_bounds__(256)
k_coil_cov(const float2* __restrict__ y, size_t npts, int nc, int nchunks, double2* __restrict__ part) {
    __shared__ float2 s[kMaxCoils][kChunk];
    const int b = blockIdx.y, chunk = blockIdx.x;
    const size_t i0 = (size_t)chunk * kChunk;
    for (int k = threadIdx.x; k < nc * kChunk; k += blockDim.x) {
        const int c = k / kChunk, j = k % kChunk;
        s[c][j] = (i0 + j < npts) ? y[((size_t)b * nc + c) * npts + i0 + j] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int npairs = nc * (nc + 1) / 2;
    for (int pr = threadIdx.x; pr < npairs; pr += blockDim.x) {
        int c = 0, rem = pr;
        while (rem >= nc - c) {
            rem -= nc - c;
            ++c;
        }
        const int d = c + rem;
        float re = 0.f, im = 0.f;
        for (int j = 0; j < kChunk; ++j) {
            const float2 a = s[c][j], e = s[d][j];
            re = fmaf(a.x, e.x, fmaf(a.y, e.y, re));
            im = fmaf(a.y, e.x, fmaf(-a.x, e.y, im));
        }
        part[((size_t)b * nchunks + chunk) * npairs + pr] = make_double2(re, im);
    }
}

// cov[b][pair] = sum over chunks, in chunk order (FP64, deterministic)
__global__ void k_coil_cov_reduce(const double2* __restrict__ part, int nchunks, int npairs, int nb,
                                  double2* __restrict__ cov) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb * npairs) return;
    const int b = i / npairs, pr = i % npairs;
    double re = 0.0, im = 0.0;
    for (int ch = 0; ch < nchunks; ++ch) {
        const double2 v = part[((size_t)b * nchunks + ch) * npairs + pr];
        re += v.x;
        im += v.y;
    }
    cov[i] = make_double2(re, im);
}

// out[b][v][i] = sum_c A[b][v][c] in[b][c][i]
__global__ void __launch_bounds__(256)
k_coil_project(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ A, size_t npts,
               int nc, int nv) {
    __shared__ float2 a[kMaxCoils * kMaxCoils];
    const int b = blockIdx.y;
    for (int k = threadIdx.x; k < nv * nc; k += blockDim.x) a[k] = A[(size_t)b * nv * nc + k];
    __syncthreads();
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npts; i += (size_t)gridDim.x * blockDim.x) {
        float2 v[kMaxCoils];  // fixed trip counts keep v in registers
#pragma unroll
        for (int c = 0; c < kMaxCoils; ++c)
            v[c] = c < nc ? in[((size_t)b * nc + c) * npts + i] : make_float2(0.f, 0.f);
        for (int o = 0; o < nv; ++o) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < kMaxCoils; ++c)
                if (c < nc) acc = cadd(acc, cmul(a[o * nc + c], v[c]));
            out[((size_t)b * nv + o) * npts + i] = acc;
        }
    }
}

using cd = std::complex<double>;

// device scratch of sb_coil_compress, kept per device and grown on demand (a cudaFree per call
// would synchronise the device); the mutex also serialises concurrent calls on one device
struct Scratch {
    void* ptr = nullptr;
    size_t bytes = 0;
};
std::mutex g_scratch_mu;
std::map<int, Scratch> g_scratch;

cudaError_t scratch_get(size_t bytes, void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    Scratch& s = g_scratch[dev];
    if (s.bytes < bytes) {
        if (s.ptr) cudaFree(s.ptr);
        s.ptr = nullptr;
        s.bytes = 0;
        if ((e = cudaMalloc(&s.ptr, bytes)) != cudaSuccess) return e;
        s.bytes = bytes;
    }
    *out = s.ptr;
    return cudaSuccess;
}

// Eigen-decomposition of a Hermitian n x n matrix (row-major) by cyclic Jacobi rotations.  Each
// rotation zeroes a[p][q]: with a[p][q] = |b| e^{i phi}, D = diag(1, e^{-i phi}) makes the 2 x 2
// block real symmetric, and the symmetric Schur rotation J = [[c, s], [-s, c]] with
// tau = (a_qq - a_pp) / (2 |b|), t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2),
// s = t c diagonalises it; U = D J is applied as a <- U^H a U, v <- v U.
void hermitian_jacobi(std::vector<cd>& a, int n, std::vector<cd>& v, std::vector<double>& w) {
    v.assign((size_t)n * n, cd(0.0, 0.0));
    for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
    auto A = [&](int r, int c) -> cd& { return a[(size_t)r * n + c]; };
    double total = 0.0;
    for (const cd& z : a) total += std::norm(z);
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += std::norm(A(p, q));
        if (off <= 1e-26 * total || total == 0.0) break;  // off-diagonal 1e-13 of the norm
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const cd b = A(p, q);
                const double mb = std::abs(b);
                if (mb <= 1e-300) continue;
                const cd e = b / mb;  // e^{i phi}
                const double tau = (A(q, q).real() - A(p, p).real()) / (2.0 * mb);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                const cd upp = c, upq = s, uqp = -s * std::conj(e), uqq = c * std::conj(e);
                for (int r = 0; r < n; ++r) {  // columns: a <- a U
                    const cd ap = A(r, p), aq = A(r, q);
                    A(r, p) = ap * upp + aq * uqp;
                    A(r, q) = ap * upq + aq * uqq;
                }
                for (int r = 0; r < n; ++r) {  // rows: a <- U^H a
                    const cd ap = A(p, r), aq = A(q, r);
                    A(p, r) = std::conj(upp) * ap + std::conj(uqp) * aq;
                    A(q, r) = std::conj(upq) * ap + std::conj(uqq) * aq;
                }
                A(p, q) = A(q, p) = 0.0;
                for (int r = 0; r < n; ++r) {
                    const cd vp = v[(size_t)r * n + p], vq = v[(size_t)r * n + q];
                    v[(size_t)r * n + p] = vp * upp + vq * uqp;
                    v[(size_t)r * n + q] = vp * upq + vq * uqq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A(i, i).real();
}

// compression matrix (nv x nc, row-major) and descending eigenvalues of a covariance
void compression_from_cov(const std::vector<cd>& cov, int nc, int nv, std::vector<cd>& mat, std::vector<double>& eig) {
    std::vector<cd> a = cov, v;
    std::vector<double> w;
    hermitian_jacobi(a, nc, v, w);
    std::vector<int> order(nc);
    for (int i = 0; i < nc; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return w[i] > w[j]; });
    mat.assign((size_t)nv * nc, cd(0.0, 0.0));
    for (int o = 0; o < nv; ++o)
        for (int c = 0; c < nc; ++c) mat[(size_t)o * nc + c] = std::conj(v[(size_t)c * nc + order[o]]);
    eig.resize(nc);
    for (int i = 0; i < nc; ++i) eig[i] = w[order[i]];
}

}  // namespace
}  // namespace sb

using namespace sb;

extern "C" {

sb_status sb_coil_compression_matrix(const double* cov, int nc, int nv, double* mat_out, double* eig_out) {
    if (!cov || !mat_out || nc < 1 || nc > kMaxCoils || nv < 1 || nv > nc) return SB_ERR_INVALID_ARG;
    std::vector<cd> c((size_t)nc * nc);
    for (size_t i = 0; i < c.size(); ++i) c[i] = cd(cov[2 * i], cov[2 * i + 1]);
    std::vector<cd> mat;
    std::vector<double> eig;
    compression_from_cov(c, nc, nv, mat, eig);
    for (size_t i = 0; i < mat.size(); ++i) {
        mat_out[2 * i] = mat[i].real();
        mat_out[2 * i + 1] = mat[i].imag();
    }
    if (eig_out)
        for (int i = 0; i < nc; ++i) eig_out[i] = eig[i];
    return SB_OK;
}

sb_status sb_coil_compress(const void* d_y, const void* d_sens, size_t npix, int nc, int nbatch, int nv,
                           void* d_y_out, void* d_sens_out, void* h_matrix, double* h_eig, void* cuda_stream) {
    if (!d_y || !d_sens || !d_y_out || !d_sens_out || npix == 0 || nbatch < 1 || nc < 1 || nc > kMaxCoils || nv < 1 ||
        nv > nc)
        return SB_ERR_INVALID_ARG;
    if (d_y_out == d_y || d_sens_out == d_sens) return SB_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int nchunks = (int)((npix + kChunk - 1) / kChunk);
    const int npairs = nc * (nc + 1) / 2;
    const size_t nparts = (size_t)nbatch * nchunks * npairs;
    const size_t ncov = (size_t)nbatch * npairs;
    // partial sums, the per-slice sums and the compression matrices in one scratch block
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    void* base = nullptr;
    if (scratch_get((nparts + ncov) * sizeof(double2) + (size_t)nbatch * nv * nc * sizeof(float2), &base) !=
        cudaSuccess)
        return SB_ERR_CUDA;
    double2* part = static_cast<double2*>(base);
    double2* dcov = part + nparts;
    float2* dmat = reinterpret_cast<float2*>(dcov + ncov);
    sb_status st = SB_OK;
    std::vector<double2> hp(ncov);
    std::vector<float2> hm((size_t)nbatch * nv * nc);
    do {
        k_coil_cov<<<dim3(nchunks, nbatch), 256, 0, s>>>(static_cast<const float2*>(d_y), npix, nc, nchunks, part);
        k_coil_cov_reduce<<<(unsigned)((ncov + 255) / 256), 256, 0, s>>>(part, nchunks, npairs, nbatch, dcov);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(hp.data(), dcov, ncov * sizeof(double2), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = SB_ERR_CUDA;
            break;
        }
        // one small eigenproblem per slice, independent: spread over host threads
        auto solve = [&](int b) {
            std::vector<cd> cov((size_t)nc * nc, cd(0.0, 0.0));
            const double2* pp = hp.data() + (size_t)b * npairs;
            int pr = 0;
            for (int c = 0; c < nc; ++c)
                for (int d = c; d < nc; ++d, ++pr) cov[(size_t)c * nc + d] = cd(pp[pr].x, pp[pr].y);
            for (int c = 0; c < nc; ++c)
                for (int d = 0; d < c; ++d) cov[(size_t)c * nc + d] = std::conj(cov[(size_t)d * nc + c]);
            std::vector<cd> mat;
            std::vector<double> eig;
            compression_from_cov(cov, nc, nv, mat, eig);
            for (size_t i = 0; i < mat.size(); ++i)
                hm[(size_t)b * nv * nc + i] = make_float2((float)mat[i].real(), (float)mat[i].imag());
            if (h_eig)
                for (int i = 0; i < nc; ++i) h_eig[(size_t)b * nc + i] = eig[i];
        };
        const int nthr = std::max(1, std::min<int>(nbatch, (int)std::thread::hardware_concurrency()));
        std::vector<std::thread> pool;
        for (int k = 1; k < nthr; ++k)
            pool.emplace_back([&, k] {
                for (int b = k; b < nbatch; b += nthr) solve(b);
            });
        for (int b = 0; b < nbatch; b += nthr) solve(b);
        for (auto& th : pool) th.join();
        if (h_matrix) std::copy(hm.begin(), hm.end(), static_cast<float2*>(h_matrix));
        if (cudaMemcpyAsync(dmat, hm.data(), hm.size() * sizeof(float2), cudaMemcpyHostToDevice, s) != cudaSuccess) {
            st = SB_ERR_CUDA;
            break;
        }
        const unsigned blocks = (unsigned)std::min<size_t>((npix + 255) / 256, 4096);
        k_coil_project<<<dim3(blocks, nbatch), 256, 0, s>>>(static_cast<const float2*>(d_y),
                                                              static_cast<float2*>(d_y_out), dmat, npix, nc, nv);
        k_coil_project<<<dim3(blocks, nbatch), 256, 0, s>>>(static_cast<const float2*>(d_sens),
                                                              static_cast<float2*>(d_sens_out), dmat, npix, nc, nv);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) st = SB_ERR_CUDA;
    } while (false);
    return st;
}

}  // extern "C"
