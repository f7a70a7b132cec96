// sb_apply_precond_noalloc: z = F^H diag(k)^{-1} F r without any device allocation.
//
// Some callers cannot call cudaMalloc at the point where they need the preconditioner: code
// that runs with a frozen memory budget after start-up (an acquisition-time reconstruction
// pipeline), hosts that hand a plugin only pre-allocated buffers, or frameworks that own the
// device memory pool.  sb_apply_precond needs a plan, and a plan allocates its workspace.
// This entry point needs no plan: the caller passes r, k and z, and the intermediate of the
// two-pass transform (the row DFTs of r) lives in g_noalloc_scratch, a file-scope device array
// of fixed size that every GPU loading this library holds until the process exits.
//
// Set-up: the first call on each device resolves the array's device address with
// cudaGetSymbolAddress (the array's name in host code is only a host-side stand-in), writes
// the DFT twiddle tables into it and waits for the device to finish that copy (a copy from
// pageable host memory may return before the data has landed, and the caller's stream need not
// be ordered after the copy's stream); so that first call must not be made while a stream is
// being captured.  Later calls only enqueue three kernels on `stream`.  The set-up is kept per
// device ordinal: the entry point serves the device's primary context (the one the CUDA
// runtime uses) and does not survive cudaDeviceReset.
// Every call shares the array and leaves its contents behind; nothing in it has to start at
// zero (the intermediate is fully written before it is read).  Calls whose kernels overlap on
// the GPU (different streams, or different threads without ordering) race on the array.
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "sb.h"

namespace sb {
namespace {

constexpr int TX = kColTile;
constexpr int kMaxDevices = 64;
// Layout of the scratch array (float2 units): DFT twiddle tables for n = 32, 64, 128, 256 at
// offsets 0, 32, 96, 224 (480 entries, padded to 512), then the row-DFT intermediate.
constexpr size_t kTwiddleRegion = 512;
constexpr size_t kNoAllocMaxElems = size_t(1) << 20;  // complex64 elements: 8 MiB

static __device__ __align__(256) float2 g_noalloc_scratch[kTwiddleRegion + kNoAllocMaxElems];

size_t twiddle_offset(int n) {
    switch (n) {
        case 32: return 0;
        case 64: return 32;
        case 128: return 96;
        default: return 224;
    }
}

struct DeviceScratch {
    float2* base = nullptr;  // device address of g_noalloc_scratch on this device
    bool ready = false;
};
DeviceScratch g_dev[kMaxDevices];
std::mutex g_mu;

// Column pass with k itself as input: t <- IDFT_y( DFT_y(t) / (k N) ), in place.
template <int NY>
__global__ void __launch_bounds__(TX * NY / 16)
k_col_precond_k(float2* __restrict__ tb, const float* __restrict__ kdiag, const float2* __restrict__ tw_g, int nx) {
    constexpr int T = NY / 16;
    constexpr int NT = TX * T;
    extern __shared__ __align__(128) unsigned char smem[];
    float2* buf0 = reinterpret_cast<float2*>(smem);
    float2* buf1 = buf0 + NY * TX;
    float2* tw = buf1 + NY * TX;
    const int tid = threadIdx.x, col = tid % TX, t = tid / TX;
    const int x = blockIdx.x * TX + col;
    for (int i = tid; i < NY; i += NT) tw[i] = tw_g[i];
    const size_t img = (size_t)blockIdx.y * NY * nx;
    const float n = (float)(NY * nx);
    float2 v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = tb[img + (size_t)(t + T * e) * nx + x];
    __syncthreads();
    struct Idx {
        int col;
        __device__ __forceinline__ int operator()(int pos) const { return pos * TX + col; }
    } idx{col};
    fft_2stage<NY, false>(v, t, buf0, idx, tw);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const float kv = __ldg(kdiag + img + (size_t)(t + T * e) * nx + x);
        v[e] = cscale(v[e], 1.f / (kv * n));
    }
    fft_2stage<NY, true>(v, t, buf1, idx, tw);
#pragma unroll
    for (int e = 0; e < 16; ++e) tb[img + (size_t)(t + T * e) * nx + x] = v[e];
}

template <int NY>
cudaError_t col_k_n(int nx, int nb, float2* t, const float* k, const float2* tw, cudaStream_t s) {
    const size_t sm = (2 * NY * TX + NY) * sizeof(float2);
    if (sm > 48 * 1024) {
        cudaError_t e = set_smem_limit(k_col_precond_k<NY>, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_col_precond_k<NY><<<dim3(nx / TX, nb), TX * NY / 16, sm, s>>>(t, k, tw, nx);
    return cudaGetLastError();
}

// Once per device, with that device current: resolve the array's address and fill the
// twiddle tables (tw[r * 16 + j] = exp(-2 pi i r j / n), the layout fft_2stage reads).
cudaError_t setup_device(int dev, float2** base) {
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceScratch& d = g_dev[dev];
    if (!d.ready) {
        float2* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        std::vector<float2> tw(kTwiddleRegion, make_float2(0.f, 0.f));
        for (int n : {32, 64, 128, 256})
            for (int r = 0; r < n / 16; ++r)
                for (int j = 0; j < 16; ++j) {
                    const double a = -2.0 * M_PI * (double)r * j / n;
                    tw[twiddle_offset(n) + r * 16 + j] = make_float2((float)std::cos(a), (float)std::sin(a));
                }
        e = cudaMemcpy(p, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
        // the tables must be in device memory before any stream, blocking or not, reads them
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return e;
        d.base = p;
        d.ready = true;
    }
    *base = d.base;
    return cudaSuccess;
}

bool supported(int n) { return n == 32 || n == 64 || n == 128 || n == 256; }

}  // namespace
}  // namespace sb

extern "C" sb_status sb_apply_precond_noalloc(const void* d_r, const float* d_k, void* d_z, int nx, int ny,
                                              int nbatch, void* cuda_stream) {
    using namespace sb;
    if (!d_r || !d_k || !d_z || nbatch < 1) return SB_ERR_INVALID_ARG;
    if (!supported(nx) || !supported(ny)) return SB_ERR_UNSUPPORTED;
    if ((size_t)nx * ny * nbatch > kNoAllocMaxElems) return SB_ERR_INVALID_ARG;  // beyond the fixed scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SB_ERR_CUDA;
    float2* base = nullptr;
    if (setup_device(dev, &base) != cudaSuccess) return SB_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    float2* tb = base + kTwiddleRegion;
    const Dims d{nx, ny, 1, nbatch};
    const Red none{nullptr, nullptr, nullptr};
    cudaError_t e = launch_row_fwd(d, 0, const_cast<float2*>(static_cast<const float2*>(d_r)), nullptr, tb,
                                   base + twiddle_offset(nx), nullptr, 0.0, none, s);
    if (e == cudaSuccess) {
        switch (ny) {
            case 32: e = col_k_n<32>(nx, nbatch, tb, d_k, base + twiddle_offset(ny), s); break;
            case 64: e = col_k_n<64>(nx, nbatch, tb, d_k, base + twiddle_offset(ny), s); break;
            case 128: e = col_k_n<128>(nx, nbatch, tb, d_k, base + twiddle_offset(ny), s); break;
            default: e = col_k_n<256>(nx, nbatch, tb, d_k, base + twiddle_offset(ny), s); break;
        }
    }
    if (e == cudaSuccess)
        e = launch_row_inv(d, 0, tb, static_cast<float2*>(d_z), nullptr, nullptr, base + twiddle_offset(nx), nullptr,
                           none, s);
    return e == cudaSuccess ? SB_OK : SB_ERR_CUDA;
}
