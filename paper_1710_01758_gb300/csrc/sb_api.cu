// C-ABI layer (include/sb.h): plan object, workspace, argument checks, and the host-side
// drivers of preconditioned CG and of Split Bregman (Algorithm 1).  Every numerical step runs
// in the kernels of k_*.cu; the host only sequences launches and reads the per-slice CG state
// back to decide when to stop.
//
// Execution contexts: the batch is split into contiguous slice groups, each with its own stream
// and its own host thread for sb_pcg_solve and sb_split_bregman.  Slices converge after
// different numbers of PCG iterations; within one group the later iterations run with few
// active slices, and the concurrent groups fill the GPU meanwhile.  The groups fork from and
// join back into the plan's stream, so callers see ordinary stream-ordered calls.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <tuple>
#include <string>
#include <thread>
#include <vector>

#include "kernels.h"
#include "sb.h"

using namespace sb;

namespace sb {
cudaError_t set_smem_limit(const void* kernel, int bytes) {
    static std::mutex mu;
    static std::set<std::tuple<const void*, int, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const auto key = std::make_tuple(kernel, dev, bytes);
    {
        std::lock_guard<std::mutex> lock(mu);
        if (done.count(key)) return cudaSuccess;
    }
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(mu);
        done.insert(key);
    }
    return e;
}
}  // namespace sb

namespace {

std::atomic<uint64_t> g_launches{0};
thread_local uint64_t t_launches = 0;  // this host thread's launches (sizes a graph capture)

// PCG iterations enqueued between two reads of the per-slice state
#ifndef SB_POLL_EVERY
#define SB_POLL_EVERY 4
#endif
constexpr int kPollEvery = SB_POLL_EVERY;

bool supported_n(int n) {
    return n == 32 || n == 64 || n == 128 || n == 256 || n == 512 || n == 192 || n == 224 || n == 320 || n == 384;
}

struct Pending {
    int cls;
    cudaEvent_t a, b;
};

}  // namespace

// A contiguous range of slices [b0, b0 + d.nb) driven on one stream.
// A captured block of PCG iterations (CUDA graph), replayed while its parameters hold
struct PcgGraph {
    const void* sens;  // the coil maps (TMA descriptors) are captured by value
    bool general;      // line-mask or general data-term path
    const void* x;
    double tol2;
    int precond, fixed, iters;
    cudaGraphExec_t exec;
    uint64_t launches;  // kernels per replay
};

struct Exec {
    sb_plan pl = nullptr;
    int b0 = 0;
    Dims d{};
    cudaStream_t s = nullptr;
    bool own_stream = false;
    CUtensorMap smap{}, ymap{}, y1map{};  // TMA maps whose first row belongs to slice b0
    CUtensorMap ymap8{}, y1map8{};        // compact k-space rows as 8-column boxes, 64-byte swizzle (ny 256, 512)
    CUtensorMap smap_sw{};                // coil tiles with the 128-byte swizzle (q = A p)
    CUtensorMap smap_sw64{};              // 8-column coil tiles, 64-byte swizzle (split-precision q = A p)
    SliceState* st = nullptr;             // device state of the range
    SliceState* h_st = nullptr;           // pinned mirror of the range
    Red red{};
    unsigned h_err = 0;
    std::string err;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> ev_pool;
    cudaEvent_t join = nullptr;
    std::vector<PcgGraph> graphs;  // captured PCG iteration blocks of this context
    bool primed = false;           // one block ran uncaptured (kernel attributes are set)
};

struct sb_plan_s {
    sb_plan_desc d{};
    cudaStream_t stream = nullptr;
    int device = 0;
    Dims dims{};
    size_t n = 0;  // pixels per slice
    const float2* sens = nullptr;
    bool have_coils = false, have_mask = false;
    bool fused_precond = false;  // circulant M^{-1} as one cluster launch per PCG iteration
    bool graphs = true;          // PCG iteration blocks replayed as CUDA graphs
    int col_tile = kColTile;     // columns per CTA of the preconditioner's column pass (tuning)
    int poll_every = kPollEvery; // PCG iterations between convergence polls (tuning)
    int apply_tile = 8;          // columns per CTA of q = A p at ny = 256 (tuning: 8 or 16)
    // volumes: dims is the rows view {nx, ny nz, Nc, nb}; the planes are ny_plane x nx, nz of them
    int nz = 1, ny_plane = 0;
    size_t maxparts = kMaxParts;  // per-slice capacity of the cross-CTA partial sums
    float2* tw_z = nullptr;
    float2* tw_full = nullptr;  // W_ny^m, m < ny, and the DFT-matrix operands (split-precision modes)
    void* bmat = nullptr;
    float2* bz[2] = {nullptr, nullptr};
    // 2D slices whose mask varies along x (the paper's random 2D sampling): the data term runs
    // as the three passes of the volumes with a per-point mask (copied here)
    bool general = false;
    bool general_cluster = false;  // q = A p of the general path as one cluster launch (k_general.cu)
    int general_passes = 1;        // tuning: 1 = the cluster launch where the shape allows, 3 = three passes
    uint8_t* mask8 = nullptr;
    float2* wb = nullptr;  // Daubechies-4 coefficient scratch [nb][ny][nx]
    bool passes() const { return nz > 1 || general; }
    std::string err;

    float2* tw_x = nullptr;
    float2* tw_y = nullptr;
    float* maskw = nullptr;  // [nb][ny]
    int* slot = nullptr;     // [nb][ny]
    int* lines = nullptr;    // [nb][ms]
    int ms = 0;
    float* k = nullptr;      // [nb][N]
    float* invk = nullptr;   // [nb][N]
    float* kd = nullptr;     // [N] k_d of the geometry (the same for every slice)
    float* jw = nullptr;     // [nb][N] 1 / diag(A) (Jacobi)
    bool jw_ready = false;   // jw matches the current coils and mask (built by the first Jacobi solve)
    float2 *r = nullptr, *p = nullptr, *q = nullptr, *tb = nullptr;
    float2* bx[2] = {nullptr, nullptr};
    float2* by[2] = {nullptr, nullptr};
    float2 *bw = nullptr, *g = nullptr;
    float2 *bd = nullptr, *bd1 = nullptr;  // data term of b for y^[j] and for y^[1]
    float2 *yt = nullptr, *yt1 = nullptr;
    size_t yt_elems = 0;
    SliceState* st = nullptr;
    SliceState* h_st = nullptr;  // pinned mirror
    double* part = nullptr;
    unsigned* counter = nullptr;
    unsigned* kmax = nullptr;
    unsigned* derr = nullptr;  // device error word
    uint32_t wait_limit = kWaitLimit;  // polls of each bounded device wait (sb_set_wait_check)
    uint32_t red_flags = 0;            // Red::flags of every launch (sb_set_wait_check)
    // k construction scratch (kept after the first sb_set_mask so later calls do not allocate)
    float2 *spec = nullptr, *gb = nullptr, *rb = nullptr;
    int *line_val = nullptr, *line_uni = nullptr;

    Exec whole;                 // the full batch on the plan's stream
    std::vector<Exec> groups;   // concurrent slice groups
    cudaEvent_t fork = nullptr;

    // event timer per kernel class (totals over all contexts)
    unsigned tmask = 0;
    std::mutex tmu;
    uint64_t tcount[SB_KCLASS_COUNT] = {};
    double tms[SB_KCLASS_COUNT] = {};
};

namespace {

sb_status fail(sb_plan pl, sb_status s, const std::string& msg) {
    if (pl) pl->err = msg;
    return s;
}

sb_status xfail(Exec& ex, sb_status s, const std::string& msg) {
    ex.err = msg;
    return s;
}

std::string cuda_msg(const char* what, cudaError_t e) {
    return std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}

#define SB_CK(pl, call)                                                            \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) return fail((pl), SB_ERR_CUDA, cuda_msg(#call, e_)); \
    } while (0)

#define SB_XCK(ex, call)                                                             \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) return xfail((ex), SB_ERR_CUDA, cuda_msg(#call, e_)); \
    } while (0)

cudaEvent_t timer_begin(Exec& ex, int cls) {
    if (!(ex.pl->tmask & (1u << cls))) return nullptr;
    cudaEvent_t a = nullptr;
    if (!ex.ev_pool.empty()) {
        a = ex.ev_pool.back();
        ex.ev_pool.pop_back();
    } else if (cudaEventCreate(&a) != cudaSuccess) {
        return nullptr;
    }
    if (cudaEventRecord(a, ex.s) != cudaSuccess) {
        ex.ev_pool.push_back(a);
        return nullptr;
    }
    return a;
}

void timer_end(Exec& ex, int cls, cudaEvent_t a) {
    if (!a) return;
    cudaEvent_t b = nullptr;
    if (!ex.ev_pool.empty()) {
        b = ex.ev_pool.back();
        ex.ev_pool.pop_back();
    } else if (cudaEventCreate(&b) != cudaSuccess) {
        ex.ev_pool.push_back(a);
        return;
    }
    cudaEventRecord(b, ex.s);
    ex.pending.push_back({cls, a, b});
}

// accumulate the recorded event pairs; call only after ex.s has been synchronised
void timer_harvest(Exec& ex) {
    if (ex.pending.empty()) return;
    double ms_c[SB_KCLASS_COUNT] = {};
    uint64_t n_c[SB_KCLASS_COUNT] = {};
    for (const auto& p : ex.pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            ms_c[p.cls] += ms;
            n_c[p.cls] += 1;
        }
        ex.ev_pool.push_back(p.a);
        ex.ev_pool.push_back(p.b);
    }
    ex.pending.clear();
    std::lock_guard<std::mutex> lock(ex.pl->tmu);
    for (int c = 0; c < SB_KCLASS_COUNT; ++c) {
        ex.pl->tms[c] += ms_c[c];
        ex.pl->tcount[c] += n_c[c];
    }
}

// launch helper: counts kernels and, when enabled for the class, times them with events
#define SB_LAUNCH(ex, cls, nk, call)                                               \
    do {                                                                           \
        cudaEvent_t ta_ = timer_begin((ex), (cls));                                \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) return xfail((ex), SB_ERR_CUDA, cuda_msg(#call, e_)); \
        timer_end((ex), (cls), ta_);                                               \
        g_launches.fetch_add((nk), std::memory_order_relaxed);                     \
        t_launches += (nk);                                                        \
    } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16);
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

// Twiddle tables of the register-resident transforms (common.cuh), computed in double:
// n <= 256: tw[r * 16 + j] = exp(-2 pi i r j / n), r < n/16, j < 16 (the second stage);
// n = 512: tw[r * 16 + k] = exp(-2 pi i r k / 256) (second stage), tw[256 + k] =
// exp(-2 pi i k / 512), k < 256 (third stage);
// n = 192, 224, 320, 384 (mixed radix): tw[m] = exp(-2 pi i m / n), m < n.
std::vector<float2> twiddles(int n) {
    std::vector<float2> t(n);
    auto w = [](double num, double den) {
        const double a = -2.0 * M_PI * num / den;
        return make_float2((float)std::cos(a), (float)std::sin(a));
    };
    if ((n & (n - 1)) != 0) {
        for (int m = 0; m < n; ++m) t[m] = w(m, n);
        return t;
    }
    const int m = n <= 256 ? n : 256;
    for (int r = 0; r < m / 16; ++r)
        for (int j = 0; j < 16; ++j) t[r * 16 + j] = w((double)r * j, m);
    if (n > 256)
        for (int k = 0; k < 256; ++k) t[256 + k] = w(k, n);
    return t;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, resolved once through the runtime (no link against libcuda)
EncodeTiledFn tensor_map_encoder() {
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// float32 view [rows][2 nx] of complex rows starting at base; box = box_rows x one column tile
bool encode_rows(CUtensorMap* m, const void* base, int nx, size_t rows, int box_rows, bool swizzle = false,
                 int box_cols = kColTile, CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_128B) {
    auto encode = tensor_map_encoder();
    if (!encode) return false;
    const cuuint64_t gdim[2] = {(cuuint64_t)2 * nx, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)2 * nx * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)2 * box_cols, (cuuint32_t)box_rows};
    const cuuint32_t estride[2] = {1, 1};
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), gdim, gstride, box, estride,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle ? sw : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void bind_exec(sb_plan pl, Exec& ex, int b0, int nb, cudaStream_t s) {
    ex.pl = pl;
    ex.b0 = b0;
    ex.d = Dims{pl->dims.nx, pl->dims.ny, pl->dims.nc, nb};
    ex.s = s;
    ex.st = pl->st + b0;
    ex.h_st = pl->h_st + b0;
    ex.red = Red{pl->part + (size_t)b0 * pl->maxparts * 2, pl->counter + b0, pl->derr, pl->wait_limit, pl->red_flags};
}

// pointer to slice b0 of an array whose slices hold `per` elements
template <class T>
T* at(T* base, const Exec& ex, size_t per) {
    return base + (size_t)ex.b0 * per;
}

// q = A p on 2D slices with a line mask: the FP32 kernel, or in the split-precision modes the
// kernel whose radix-16 DFT stages run on the tensor cores
cudaError_t apply_A_2d(const sb_plan_s* pl, const Exec& ex, const Dims& d, const float2* p, float2* q,
                       const float* maskw, SliceState* st, Red red, cudaStream_t s) {
    const float mu = (float)pl->d.mu, lam = (float)pl->d.lambda, gam = (float)pl->d.gamma;
    if (pl->d.prec != SB_PREC_FP32) {
        const TcOperands tc{&ex.smap_sw64, pl->tw_full, pl->bmat, pl->d.prec == SB_PREC_SPLIT_BF16};
        return launch_apply_A_tc(d, tc, p, q, maskw, mu, lam, gam, st, red, s);
    }
    return launch_apply_A(d, ex.smap_sw, ex.smap_sw64, p, q, maskw, pl->tw_y, mu, lam, gam, st, red, s,
                          pl->apply_tile);
}

// ---- volumes (nz > 1) and 2D arbitrary masks: the data term as three passes through the coil
// scratch (k_vol.cu)
Dims plane_dims(const Exec& ex) { return Dims{ex.d.nx, ex.pl->ny_plane, ex.d.nc, ex.d.nb}; }

// The middle of the general path (a mask that varies along x) on the coil scratch U, after DFT_y
// of every plane: DFT_z (volumes), then along x the per-point mask operation `mode` of k_g2_x
// over the rows of every plane, then IDFT_z.  mode 2 (back-projection) reads no U, so it skips
// the forward DFT_z.  The z passes run over every volume of the context (converged ones too: U
// is scratch).
sb_status general_mid(Exec& ex, int cls, int mode, int addback, float2* U, float2* yt, const float2* yt1,
                      const SliceState* stf) {
    sb_plan pl = ex.pl;
    const Dims dp = plane_dims(ex);
    const Dims rows{dp.nx, dp.ny * pl->nz, dp.nc, dp.nb};  // the rows of all planes
    const int ncols = dp.nx * dp.ny, nimg = dp.nb * dp.nc;
    if (pl->nz > 1 && mode != 2)
        SB_LAUNCH(ex, cls, 1, launch_fft_cols(ncols, pl->nz, nimg, U, pl->tw_z, false, ex.s));
    SB_LAUNCH(ex, cls, 1,
              launch_g2_x(rows, mode, addback, U, at(pl->mask8, ex, pl->n), yt, yt1, pl->tw_x, stf, ex.s));
    if (pl->nz > 1) SB_LAUNCH(ex, cls, 1, launch_fft_cols(ncols, pl->nz, nimg, U, pl->tw_z, true, ex.s));
    return SB_OK;
}

// out = A v on the context's volumes; pcg: PCG mode (inactive volumes skipped, p^H q, alpha)
sb_status vol_apply_A(Exec& ex, const float2* v, float2* out, bool pcg) {
    sb_plan pl = ex.pl;
    const Dims dp = plane_dims(ex);
    const size_t n = pl->n;
    float2* U = at(pl->spec, ex, (size_t)dp.nc * n);
    const float2* sens = at(pl->sens, ex, (size_t)dp.nc * n);
    const SliceState* stf = pcg ? ex.st : nullptr;
    SbFields f{};
    f.sens = sens;
    const float mu = (float)pl->d.mu, lam = (float)pl->d.lambda, gam = (float)pl->d.gamma;
    if (pl->general_cluster && pl->general_passes == 1) {  // one launch, spectra in distributed shared memory
        SB_LAUNCH(ex, SB_KCLASS_APPLY_A, 1,
                  launch_apply_A_general(dp, sens, v, out, at(pl->mask8, ex, n), pl->tw_x, pl->tw_y, mu, lam, gam,
                                         pcg ? ex.st : nullptr, ex.red, ex.s));
        return SB_OK;
    }
    SB_LAUNCH(ex, SB_KCLASS_APPLY_A, 1, launch_g3_fwd_y(dp, pl->nz, sens, v, U, pl->tw_y, stf, ex.s));
    if (pl->general) {
        if (sb_status e = general_mid(ex, SB_KCLASS_APPLY_A, 0, 0, U, nullptr, nullptr, stf)) return e;
    } else
        SB_LAUNCH(ex, SB_KCLASS_APPLY_A, 1,
                  launch_g3_z(dp, pl->nz, 0, 0, U, at(pl->slot, ex, (size_t)ex.d.ny), nullptr, nullptr, pl->ms,
                              pl->tw_z, stf, ex.s));
    SB_LAUNCH(ex, SB_KCLASS_APPLY_A, 1,
              launch_g3_inv_y(dp, pl->nz, 0, pcg ? 1 : 0, U, f, v, out, 0, pl->tw_y, mu, lam, gam, ex.st, 0.0, ex.red,
                              ex.s));
    return SB_OK;
}

// M^{-1} = F^H diag(k)^{-1} F on volumes: DFT along x (rows), y (per plane), z with 1/(kN) and
// r^H z, then the inverses.  phase 0: out = M^{-1} r; 1: CG start (p = z, rho); 2: CG step
// (r -= alpha q and the stop test first; x += alpha p, p = z + beta p after).
sb_status vol_precond(Exec& ex, int phase, float2* r, const float2* q, float2* x, float2* p, float2* out,
                      double tol2) {
    sb_plan pl = ex.pl;
    const Dims& d = ex.d;  // rows view
    const int nyp = pl->ny_plane, nz = pl->nz;
    const Dims dz{d.nx * nyp, nz, d.nc, d.nb};  // z columns
    SliceState* st = phase ? ex.st : nullptr;
    float2* tb = at(pl->tb, ex, pl->n);
    const float* invk = at(pl->invk, ex, pl->n);
    SB_LAUNCH(ex, SB_KCLASS_PRECOND_ROW_FWD, 1,
              launch_row_fwd(d, phase == 2 ? 1 : 0, r, q, tb, pl->tw_x, st, tol2, ex.red, ex.s));
    SB_LAUNCH(ex, SB_KCLASS_PRECOND_COL, 1, launch_col_dft(d.nx, nyp, d.nb * nz, nz, tb, pl->tw_y, false, st, ex.s));
    SB_LAUNCH(ex, SB_KCLASS_PRECOND_COL, 1,
              launch_col_precond(dz, tb, invk, pl->tw_z, st, phase == 1 ? 1 : 0, ex.red, ex.s));
    SB_LAUNCH(ex, SB_KCLASS_PRECOND_COL, 1, launch_col_dft(d.nx, nyp, d.nb * nz, nz, tb, pl->tw_y, true, st, ex.s));
    SB_LAUNCH(ex, SB_KCLASS_PRECOND_ROW_INV, 1, launch_row_inv(d, phase, tb, out, x, p, pl->tw_x, st, ex.red, ex.s));
    return SB_OK;
}

// Sequence CG on the context's slices from the state left by launch_resid_init / launch_rhs
// (r = r0, bnorm2, state).  x and the result arrays are the full-batch ones.
sb_status pcg_run(Exec& ex, const sb_pcg_opts& o, float2* x_full, sb_pcg_result* h_results, int* iters_out,
                  int iters_stride) {
    sb_plan pl = ex.pl;
    const Dims& d = ex.d;
    const size_t n = pl->n;
    cudaStream_t s = ex.s;
    const bool fixed = o.fixed_iters > 0;
    const double tol2 = fixed ? -1.0 : o.tol * o.tol;
    const bool circ = o.precond == SB_PRECOND_CIRCULANT;
    const float* w = o.precond == SB_PRECOND_JACOBI ? at(pl->jw, ex, n) : nullptr;
    const Red red = ex.red;
    const float mu = (float)pl->d.mu, lam = (float)pl->d.lambda, gam = (float)pl->d.gamma;
    float2* x = at(x_full, ex, n);
    float2 *r = at(pl->r, ex, n), *p = at(pl->p, ex, n), *q = at(pl->q, ex, n), *tb = at(pl->tb, ex, n);
    const float* invk = at(pl->invk, ex, n);
    const float* maskw = at(pl->maskw, ex, (size_t)d.ny);

    SB_LAUNCH(ex, SB_KCLASS_VEC, 1, launch_zero_rhs_slices(d, x, ex.st, s));
    const bool fused = circ && pl->fused_precond;
    const bool vol = pl->nz > 1, passes = pl->passes();
    if (circ && vol) {
        if (sb_status e = vol_precond(ex, 1, r, nullptr, x, p, nullptr, tol2)) return e;
    } else if (fused) {
        SB_LAUNCH(ex, SB_KCLASS_PRECOND_FUSED, 1,
                  launch_precond_fused(d, 0, x, r, p, nullptr, invk, pl->tw_x, pl->tw_y, ex.st, tol2, s));
    } else if (circ) {
        SB_LAUNCH(ex, SB_KCLASS_PRECOND_ROW_FWD, 1, launch_row_fwd(d, 0, r, nullptr, tb, pl->tw_x, ex.st, tol2, red, s));
        SB_LAUNCH(ex, SB_KCLASS_PRECOND_COL, 1, launch_col_precond(d, tb, invk, pl->tw_y, ex.st, 1, red, s, pl->col_tile));
        SB_LAUNCH(ex, SB_KCLASS_PRECOND_ROW_INV, 1, launch_row_inv(d, 1, tb, nullptr, x, p, pl->tw_x, ex.st, red, s));
    } else {
        SB_LAUNCH(ex, SB_KCLASS_VEC, 1, launch_vec_plain(d, 0, x, r, p, nullptr, w, ex.st, tol2, red, s));
    }
    const int nit = fixed ? o.fixed_iters : o.maxit;
    // one PCG iteration: q = A p (with p^H q and alpha), then M^{-1} (r update, stop test, z,
    // rho, beta, x and p updates); slices that are not active skip every kernel
    auto body = [&]() -> sb_status {
        if (passes) {
            if (sb_status e = vol_apply_A(ex, p, q, true)) return e;
        } else {
            SB_LAUNCH(ex, SB_KCLASS_APPLY_A, 1,
                      apply_A_2d(pl, ex, d, p, q, maskw, ex.st, red, s));
        }
        if (circ && vol) {
            if (sb_status e = vol_precond(ex, 2, r, q, x, p, nullptr, tol2)) return e;
        } else if (fused) {
            SB_LAUNCH(ex, SB_KCLASS_PRECOND_FUSED, 1,
                      launch_precond_fused(d, 1, x, r, p, q, invk, pl->tw_x, pl->tw_y, ex.st, tol2, s));
        } else if (circ) {
            SB_LAUNCH(ex, SB_KCLASS_PRECOND_ROW_FWD, 1, launch_row_fwd(d, 1, r, q, tb, pl->tw_x, ex.st, tol2, red, s));
            SB_LAUNCH(ex, SB_KCLASS_PRECOND_COL, 1, launch_col_precond(d, tb, invk, pl->tw_y, ex.st, 0, red, s, pl->col_tile));
            SB_LAUNCH(ex, SB_KCLASS_PRECOND_ROW_INV, 1, launch_row_inv(d, 2, tb, nullptr, x, p, pl->tw_x, ex.st, red, s));
        } else {
            SB_LAUNCH(ex, SB_KCLASS_VEC, 1, launch_vec_plain(d, 1, x, r, p, q, w, ex.st, tol2, red, s));
            SB_LAUNCH(ex, SB_KCLASS_VEC, 1, launch_vec_plain(d, 2, x, r, p, q, w, ex.st, tol2, red, s));
        }
        return SB_OK;
    };
    // g iterations between two polls: replayed from a CUDA graph captured on this context's
    // stream once its parameters (x, tol, preconditioner, schedule, g) repeat; direct launches
    // while the per-kernel timer is on and for the context's first block (which also sets the
    // kernels' shared-memory attributes outside any capture)
    auto block = [&](int g) -> sb_status {
        // the legacy and per-thread default streams cannot be captured: direct launches there
        const bool use_graph = pl->graphs && pl->tmask == 0 && s != nullptr && s != cudaStreamLegacy &&
                               s != cudaStreamPerThread;
        PcgGraph* hit = nullptr;
        if (use_graph)
            for (auto& pg : ex.graphs)
                if (pg.sens == pl->sens && pg.general == pl->general && pg.x == x && pg.tol2 == tol2 && pg.precond == (int)o.precond && pg.fixed == (int)fixed &&
                    pg.iters == g)
                    hit = &pg;
        if (!hit && (!use_graph || !ex.primed)) {
            for (int i = 0; i < g; ++i)
                if (sb_status e = body()) return e;
            ex.primed = true;
            return SB_OK;
        }
        if (!hit) {
            cudaError_t ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (ce != cudaSuccess) return xfail(ex, SB_ERR_CUDA, cuda_msg("cudaStreamBeginCapture", ce));
            const uint64_t l0 = t_launches;
            sb_status st = SB_OK;
            for (int i = 0; i < g && st == SB_OK; ++i) st = body();
            cudaGraph_t graph = nullptr;
            ce = cudaStreamEndCapture(s, &graph);
            const uint64_t nk = t_launches - l0;
            t_launches = l0;
            g_launches.fetch_sub(nk);  // captured, not launched
            if (st != SB_OK || ce != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return st != SB_OK ? st : xfail(ex, SB_ERR_CUDA, cuda_msg("cudaStreamEndCapture", ce));
            }
            cudaGraphExec_t exec = nullptr;
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return xfail(ex, SB_ERR_CUDA, cuda_msg("cudaGraphInstantiate", ce));
            if (ex.graphs.size() >= 8) {  // a bounded cache: drop the oldest, once nothing of it runs
                cudaStreamSynchronize(s);
                cudaGraphExecDestroy(ex.graphs.front().exec);
                ex.graphs.erase(ex.graphs.begin());
            }
            ex.graphs.push_back(PcgGraph{pl->sens, pl->general, x, tol2, (int)o.precond, (int)fixed, g, exec, nk});
            hit = &ex.graphs.back();
        }
        const cudaError_t ce = cudaGraphLaunch(hit->exec, s);
        if (ce != cudaSuccess) return xfail(ex, SB_ERR_CUDA, cuda_msg("cudaGraphLaunch", ce));
        g_launches.fetch_add(hit->launches, std::memory_order_relaxed);
        return SB_OK;
    };
    int it = 0;
    while (it < nit) {
        const int g = std::min(pl->poll_every, nit - it);
        if (sb_status e = block(g)) return e;
        it += g;
        if (!fixed || it >= nit) {
            SB_XCK(ex, cudaMemcpyAsync(ex.h_st, ex.st, sizeof(SliceState) * d.nb, cudaMemcpyDeviceToHost, s));
            SB_XCK(ex, cudaMemcpyAsync(&ex.h_err, pl->derr, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
            SB_XCK(ex, cudaStreamSynchronize(s));
            timer_harvest(ex);
            if (ex.h_err) return xfail(ex, SB_ERR_TIMEOUT, "a bounded device wait gave up (TMA tile never arrived)");
            bool running = false;
            for (int b = 0; b < d.nb; ++b)
                running |= (ex.h_st[b].state == ST_ACTIVE || ex.h_st[b].state == ST_FINISHING);
            if (!running) break;
        }
    }
    sb_status worst = SB_OK;
    for (int b = 0; b < d.nb; ++b) {
        const SliceState& S = ex.h_st[b];
        sb_status sl = SB_OK;
        if (S.state == ST_BREAKDOWN) sl = SB_ERR_BREAKDOWN;
        else if (S.state == ST_NONFINITE) sl = SB_ERR_NONFINITE;
        else if (S.state == ST_ACTIVE && !fixed) sl = SB_ERR_NOT_CONVERGED;
        if (worst == SB_OK) worst = sl;
        const double rel = S.bnorm2 > 0 ? std::sqrt(S.rnorm2 / S.bnorm2) : 0.0;
        const int gb = ex.b0 + b;
        if (h_results) {
            h_results[gb].iters = S.iters;
            h_results[gb].rel_resid = rel;
            h_results[gb].converged = (sl == SB_OK) ? 1 : 0;
        }
        if (iters_out) iters_out[(size_t)gb * iters_stride] = S.iters;
    }
    if (worst == SB_ERR_NOT_CONVERGED) ex.err = "PCG reached maxit before the tolerance";
    else if (worst != SB_OK) ex.err = std::string("PCG stopped: ") + sb_status_string(worst);
    return worst;
}

sb_status check_ready(sb_plan pl) {
    if (!pl) return SB_ERR_INVALID_ARG;
    if (!pl->have_coils || !pl->have_mask) return fail(pl, SB_ERR_NOT_READY, "call sb_set_coils and sb_set_mask first");
    return SB_OK;
}

sb_status check_opts(sb_plan pl, const sb_pcg_opts* o) {
    if (!o) return fail(pl, SB_ERR_INVALID_ARG, "null PCG options");
    if (o->fixed_iters < 0 || (o->fixed_iters == 0 && (o->maxit < 1 || !(o->tol >= 0.0))))
        return fail(pl, SB_ERR_INVALID_ARG, "PCG options: need fixed_iters > 0, or maxit >= 1 and tol >= 0");
    if (o->precond != SB_PRECOND_CIRCULANT && o->precond != SB_PRECOND_NONE && o->precond != SB_PRECOND_JACOBI)
        return fail(pl, SB_ERR_UNSUPPORTED, "preconditioner kind not implemented");
    return SB_OK;
}

// Run fn(exec) for every slice group concurrently (one host thread per extra group), forking
// from and joining back into the plan's stream.  Returns the first non-OK status in group order.
template <class Fn>
sb_status run_groups(sb_plan pl, Fn fn) {
    const int G = (int)pl->groups.size();
    if (G == 1) {
        Exec& ex = pl->groups[0];
        sb_status st = fn(ex);
        if (st != SB_OK) pl->err = ex.err;
        return st;
    }
    SB_CK(pl, cudaEventRecord(pl->fork, pl->stream));
    for (Exec& ex : pl->groups) SB_CK(pl, cudaStreamWaitEvent(ex.s, pl->fork, 0));
    std::vector<sb_status> status(G, SB_OK);
    std::vector<std::thread> threads;
    for (int gi = 1; gi < G; ++gi)
        threads.emplace_back([&, gi]() {
            cudaSetDevice(pl->device);
            status[gi] = fn(pl->groups[gi]);
        });
    status[0] = fn(pl->groups[0]);
    for (auto& t : threads) t.join();
    for (Exec& ex : pl->groups) {
        SB_CK(pl, cudaEventRecord(ex.join, ex.s));
        SB_CK(pl, cudaStreamWaitEvent(pl->stream, ex.join, 0));
    }
    for (int gi = 0; gi < G; ++gi)
        if (status[gi] != SB_OK) {
            pl->err = pl->groups[gi].err;
            return status[gi];
        }
    return SB_OK;
}

// Algorithm 1 on one slice group.
sb_status sb_run(Exec& ex, const sb_sb_opts& o, const float2* y_full, float2* x_full, sb_pcg_result* h_last,
                 int* iters) {
    sb_plan pl = ex.pl;
    const Dims& d = ex.d;
    const size_t nb = d.nb, n = pl->n, ms = pl->ms;
    cudaStream_t s = ex.s;
    float2* x = at(x_full, ex, n);
    const float mu = (float)pl->d.mu, lam = (float)pl->d.lambda, gam = (float)pl->d.gamma;
    const float tau_tv = o.tau_tv > 0 ? (float)o.tau_tv : (lam > 0 ? 1.0f / lam : INFINITY);
    const float tau_w = o.tau_w > 0 ? (float)o.tau_w : (gam > 0 ? 1.0f / gam : INFINITY);
    const double tol2 = o.pcg.fixed_iters > 0 ? -1.0 : o.pcg.tol * o.pcg.tol;
    const int levels = pl->d.wavelet_levels;
    const int nsolve = o.n_outer * o.n_inner;
    const size_t yrow = (size_t)d.nc * ms * d.nx;  // yt elements per slice

    if (pl->general)  // whole k-space rows: the data themselves
        SB_XCK(ex, cudaMemcpyAsync(at(pl->yt1, ex, yrow), at(y_full, ex, (size_t)d.nc * n), sizeof(float2) * nb * yrow,
                                   cudaMemcpyDeviceToDevice, s));
    else
        SB_LAUNCH(ex, SB_KCLASS_OTHER, 1,
                  launch_ytilde(d, at(y_full, ex, (size_t)d.nc * n), at(pl->lines, ex, ms), (int)ms,
                                at(pl->yt1, ex, yrow), pl->tw_x, s));
    SB_XCK(ex, cudaMemcpyAsync(at(pl->yt, ex, yrow), at(pl->yt1, ex, yrow), sizeof(float2) * nb * yrow,
                               cudaMemcpyDeviceToDevice, s));
    int cur = 0;
    SB_XCK(ex, cudaMemsetAsync(at(pl->bx[0], ex, n), 0, sizeof(float2) * nb * n, s));
    SB_XCK(ex, cudaMemsetAsync(at(pl->by[0], ex, n), 0, sizeof(float2) * nb * n, s));
    const bool vol = pl->nz > 1;
    if (vol) SB_XCK(ex, cudaMemsetAsync(at(pl->bz[0], ex, n), 0, sizeof(float2) * nb * n, s));
    SB_XCK(ex, cudaMemsetAsync(at(pl->bw, ex, n), 0, sizeof(float2) * nb * n, s));
    SB_XCK(ex, cudaMemsetAsync(at(pl->g, ex, n), 0, sizeof(float2) * nb * n, s));
    auto fields = [&]() {
        SbFields f;
        f.sens = at(pl->sens, ex, (size_t)d.nc * n);
        f.maskw = at(pl->maskw, ex, (size_t)d.ny);
        f.slot = at(pl->slot, ex, (size_t)d.ny);
        f.lines = pl->lines ? at(pl->lines, ex, ms) : nullptr;
        f.yt = at(pl->yt, ex, yrow);
        f.yt1 = at(pl->yt1, ex, yrow);
        f.ms = (int)ms;
        f.bx = at(pl->bx[cur], ex, n);
        f.by = at(pl->by[cur], ex, n);
        f.bx_new = at(pl->bx[cur ^ 1], ex, n);
        f.by_new = at(pl->by[cur ^ 1], ex, n);
        f.bz = vol ? at(pl->bz[cur], ex, n) : nullptr;
        f.bz_new = vol ? at(pl->bz[cur ^ 1], ex, n) : nullptr;
        f.bw = at(pl->bw, ex, n);
        f.g = at(pl->g, ex, n);
        f.bd = at(pl->bd, ex, n);
        f.bd1 = at(pl->bd1, ex, n);
        return f;
    };
    const Dims dp = plane_dims(ex);
    float2* U = at(pl->spec, ex, (size_t)d.nc * n);
    const bool passes = pl->passes();
    if (passes) {
        SbFields f0 = fields();
        if (pl->general) {
            if (sb_status e = general_mid(ex, SB_KCLASS_OTHER, 2, 0, U, f0.yt, f0.yt1, nullptr)) return e;
        } else {
            SB_LAUNCH(ex, SB_KCLASS_OTHER, 1,
                      launch_g3_z(dp, pl->nz, 2, 0, U, f0.slot, f0.yt, f0.yt1, (int)ms, pl->tw_z, nullptr, s));
        }
        SB_LAUNCH(ex, SB_KCLASS_OTHER, 1,
                  launch_g3_inv_y(dp, pl->nz, 2, 0, U, f0, nullptr, x, o.init_rss ? 1 : 0, pl->tw_y, mu, lam, gam,
                                  ex.st, 0.0, ex.red, s));
    } else {
        SB_LAUNCH(ex, SB_KCLASS_OTHER, 1, launch_rss(d, fields(), x, o.init_rss ? 1 : 0, pl->tw_y, s));
    }

    sb_status first_err = SB_OK;
    int solve = 0;
    float2* r = at(pl->r, ex, n);
    for (int j = 0; j < o.n_outer; ++j) {
        for (int k = 0; k < o.n_inner; ++k, ++solve) {
            const int addback = (j > 0 && k == 0);
            if (passes && pl->general_cluster && pl->general_passes == 1) {  // one cluster launch
                SbFields f1 = fields();
                SB_LAUNCH(ex, SB_KCLASS_RHS, 1,
                          launch_rhs_general(dp, f1, addback, x, r, at(pl->mask8, ex, n), pl->tw_x, pl->tw_y, mu, lam,
                                             gam, ex.st, tol2, ex.red, s));
            } else if (passes) {
                SbFields f1 = fields();
                SB_LAUNCH(ex, SB_KCLASS_RHS, 1, launch_g3_fwd_y(dp, pl->nz, f1.sens, x, U, pl->tw_y, nullptr, s));
                if (pl->general) {
                    if (sb_status e = general_mid(ex, SB_KCLASS_RHS, 1, addback, U, f1.yt, f1.yt1, nullptr)) return e;
                } else
                    SB_LAUNCH(ex, SB_KCLASS_RHS, 1,
                              launch_g3_z(dp, pl->nz, 1, addback, U, f1.slot, f1.yt, f1.yt1, (int)ms, pl->tw_z, nullptr,
                                          s));
                SB_LAUNCH(ex, SB_KCLASS_RHS, 1,
                          launch_g3_inv_y(dp, pl->nz, 1, addback, U, f1, x, r, 0, pl->tw_y, mu, lam, gam, ex.st, tol2,
                                          ex.red, s));
            } else {
                const RhsMaps maps{&ex.smap, &ex.ymap, &ex.y1map, &ex.smap_sw64, &ex.ymap8, &ex.y1map8};
                SB_LAUNCH(ex, SB_KCLASS_RHS, 1,
                          launch_rhs(d, maps, fields(), addback, x, r, pl->tw_y, mu, lam, gam, ex.st, tol2, ex.red, s));
            }
            sb_status ps = pcg_run(ex, o.pcg, x_full, h_last, iters + solve, nsolve);
            if (ps == SB_ERR_TIMEOUT || ps == SB_ERR_CUDA) return ps;
            if (ps != SB_OK && first_err == SB_OK) first_err = ps;
            const bool last = (j == o.n_outer - 1) && (k == o.n_inner - 1);
            if (!last) {
                if (vol)
                    SB_LAUNCH(ex, SB_KCLASS_SB_UPDATE, 1,
                              launch_sb_update3(dp, pl->nz, fields(), x, levels, lam, gam, tau_tv, tau_w, s));
                else if (pl->d.wavelet == 1 && levels > 0 && gam != 0.f) {
                    // TV part here (g = lam D^H u), the Daubechies-4 part adds gam W^H u_w
                    SbFields f2 = fields();
                    SB_LAUNCH(ex, SB_KCLASS_SB_UPDATE, 1,
                              launch_sb_update(d, f2, x, levels, lam, 0.f, tau_tv, tau_w, s));
                    SB_LAUNCH(ex, SB_KCLASS_SB_UPDATE, d4_update_launches(levels),
                              launch_d4_update(d, x, at(pl->wb, ex, n), f2.bw, f2.g, levels, gam, tau_w, s));
                } else
                    SB_LAUNCH(ex, SB_KCLASS_SB_UPDATE, 1,
                              launch_sb_update(d, fields(), x, levels, lam, gam, tau_tv, tau_w, s));
                if (lam != 0.f) cur ^= 1;
            }
        }
    }
    SB_XCK(ex, cudaStreamSynchronize(s));
    timer_harvest(ex);
    return first_err;
}

}  // namespace

extern "C" {

const char* sb_status_string(sb_status s) {
    switch (s) {
        case SB_OK: return "SB_OK";
        case SB_ERR_INVALID_ARG: return "SB_ERR_INVALID_ARG";
        case SB_ERR_UNSUPPORTED: return "SB_ERR_UNSUPPORTED";
        case SB_ERR_CUDA: return "SB_ERR_CUDA";
        case SB_ERR_NOT_READY: return "SB_ERR_NOT_READY";
        case SB_ERR_NONFINITE: return "SB_ERR_NONFINITE";
        case SB_ERR_BREAKDOWN: return "SB_ERR_BREAKDOWN";
        case SB_ERR_NOT_CONVERGED: return "SB_ERR_NOT_CONVERGED";
        case SB_ERR_TIMEOUT: return "SB_ERR_TIMEOUT";
    }
    return "SB_ERR_UNKNOWN";
}

const char* sb_plan_last_error(sb_plan pl) { return pl ? pl->err.c_str() : "null plan"; }

uint64_t sb_kernel_launches(void) { return g_launches.load(); }

sb_status sb_plan_create(const sb_plan_desc* desc, void* cuda_stream, sb_plan* out) {
    if (!desc || !out) return SB_ERR_INVALID_ARG;
    *out = nullptr;
    const sb_plan_desc& d = *desc;
    const bool vol = d.ndim == 3;
    if ((d.ndim != 2 && d.ndim != 3) || (!vol && d.nz != 1 && d.nz != 0) || d.ncoils < 1 || d.nbatch < 1 ||
        !(d.mu > 0.0) ||
        !(d.lambda >= 0.0) || !(d.gamma >= 0.0) || d.wavelet_levels < 0 || d.groups < 0 ||
        (d.precond_passes != 0 && d.precond_passes != 1 && d.precond_passes != 3) ||
        (d.wavelet != 0 && d.wavelet != 1))
        return SB_ERR_INVALID_ARG;
    if (d.prec != SB_PREC_FP32 && d.prec != SB_PREC_SPLIT_BF16 && d.prec != SB_PREC_SPLIT_FP16)
        return SB_ERR_INVALID_ARG;
    if (!supported_n(d.nx) || !supported_n(d.ny) || d.wavelet_levels > (vol ? 4 : 5) ||
        (vol && (!supported_n(d.nz) || d.precond_passes == 1)))
        return SB_ERR_UNSUPPORTED;
    // the split-precision modes: tensor-core radix-16 stages of the 256-point column transform
    if (d.prec != SB_PREC_FP32 && (vol || !apply_A_tc_supported(Dims{d.nx, d.ny, d.ncoils, d.nbatch})))
        return SB_ERR_UNSUPPORTED;
    if (d.wavelet == 1 && d.wavelet_levels > 0 &&
        (vol || (d.nx >> (d.wavelet_levels - 1)) < 4 || (d.ny >> (d.wavelet_levels - 1)) < 4))
        return SB_ERR_UNSUPPORTED;
    const int nz = vol ? d.nz : 1;
    // the fused preconditioner (opt-in) needs a slice on one cluster that fits the device
    bool fused = false;
    if (d.precond_passes == 1) {
        fused = precond_fused_clusters(Dims{d.nx, d.ny, d.ncoils, d.nbatch}) > 0;
        if (!fused) return SB_ERR_UNSUPPORTED;
    }
    sb_plan pl = new (std::nothrow) sb_plan_s();
    if (!pl) return SB_ERR_INVALID_ARG;
    pl->d = d;
    pl->fused_precond = fused;
    pl->d.nz = nz;
    pl->nz = nz;
    pl->ny_plane = d.ny;
    pl->stream = static_cast<cudaStream_t>(cuda_stream);
    pl->dims = Dims{d.nx, d.ny * nz, d.ncoils, d.nbatch};
    pl->n = (size_t)d.nx * d.ny * nz;
    // CTAs per slice of the widest cross-CTA reduction: rows / 16, column tiles x planes, and
    // the z-columns of a volume (ny nx / 16)
    pl->maxparts = std::max<size_t>({(size_t)kMaxParts, (size_t)d.ny * nz / 16, (size_t)d.nx / 16 * nz,
                                     vol ? (size_t)d.ny * d.nx / 16 : (size_t)0});
    const size_t nb = d.nbatch, n = pl->n;
    cudaError_t e = cudaGetDevice(&pl->device);
    auto bail = [&](const char* what) {
        pl->err = cuda_msg(what, e);
        fprintf(stderr, "sb_plan_create: %s\n", pl->err.c_str());
        sb_plan_destroy(pl);
        return SB_ERR_CUDA;
    };
    if (e != cudaSuccess) return bail("cudaGetDevice");
#define ALLOC(ptr, count) \
    if ((e = dalloc(&(ptr), (count))) != cudaSuccess) return bail("cudaMalloc " #ptr);
    ALLOC(pl->tw_x, d.nx);
    ALLOC(pl->tw_y, d.ny);
    ALLOC(pl->tw_z, nz);
    if (d.prec != SB_PREC_FP32) {
        ALLOC(pl->tw_full, d.ny);
        if ((e = cudaMalloc(&pl->bmat, tc_bmat_bytes())) != cudaSuccess) return bail("cudaMalloc");
    }
    ALLOC(pl->maskw, nb * d.ny * nz);
    ALLOC(pl->slot, nb * d.ny * nz);
    ALLOC(pl->k, nb * n);
    ALLOC(pl->invk, nb * n);
    ALLOC(pl->kd, n);
    ALLOC(pl->r, nb * n);
    ALLOC(pl->p, nb * n);
    ALLOC(pl->q, nb * n);
    ALLOC(pl->tb, nb * n);
    ALLOC(pl->st, nb);
    ALLOC(pl->part, nb * pl->maxparts * 2);
    ALLOC(pl->counter, nb);
    ALLOC(pl->kmax, nb);
    ALLOC(pl->derr, 1);
#undef ALLOC
    if ((e = cudaMallocHost(reinterpret_cast<void**>(&pl->h_st), sizeof(SliceState) * nb)) != cudaSuccess)
        return bail("cudaMallocHost");
    const std::vector<float2> tx = twiddles(d.nx), ty = twiddles(d.ny), tz = twiddles(nz > 1 ? nz : 32);
    if ((e = cudaMemcpy(pl->tw_x, tx.data(), sizeof(float2) * d.nx, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail("cudaMemcpy twiddles");
    if ((e = cudaMemcpy(pl->tw_y, ty.data(), sizeof(float2) * d.ny, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail("cudaMemcpy twiddles");
    if ((e = cudaMemcpy(pl->tw_z, tz.data(), sizeof(float2) * nz, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail("cudaMemcpy twiddles");
    {  // k_d = 2 ndim - 2 cos(2 pi kx / nx) - 2 cos(2 pi ky / ny) (- 2 cos(2 pi kz / nz)), in double
        auto c2 = [](int len) {
            std::vector<double> c(len);
            for (int m = 0; m < len; ++m) c[m] = 2.0 * std::cos(2.0 * M_PI * m / len);
            return c;
        };
        const std::vector<double> cx = c2(d.nx), cy = c2(d.ny), cz = c2(nz);
        std::vector<float> hk(n);
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < d.ny; ++y)
                for (int x = 0; x < d.nx; ++x)
                    hk[((size_t)z * d.ny + y) * d.nx + x] = (float)(6.0 - cx[x] - cy[y] - cz[z]);
        if ((e = cudaMemcpy(pl->kd, hk.data(), sizeof(float) * n, cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail("cudaMemcpy k_d");
    }
    if (pl->tw_full) {
        std::vector<float2> tf(d.ny);
        for (int m = 0; m < d.ny; ++m) {
            const double a = -2.0 * M_PI * m / d.ny;
            tf[m] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        std::vector<uint16_t> bm(tc_bmat_bytes() / 2);
        build_tc_bmat(d.prec == SB_PREC_SPLIT_BF16, bm.data());
        if ((e = cudaMemcpy(pl->tw_full, tf.data(), sizeof(float2) * d.ny, cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(pl->bmat, bm.data(), tc_bmat_bytes(), cudaMemcpyHostToDevice)) != cudaSuccess)
            return bail("cudaMemcpy twiddles");
    }
    if ((e = cudaMemset(pl->counter, 0, sizeof(unsigned) * nb)) != cudaSuccess) return bail("cudaMemset");
    if ((e = cudaMemset(pl->derr, 0, sizeof(unsigned))) != cudaSuccess) return bail("cudaMemset");
    if ((e = cudaMemset(pl->st, 0, sizeof(SliceState) * nb)) != cudaSuccess) return bail("cudaMemset");

    // execution contexts
    bind_exec(pl, pl->whole, 0, (int)nb, pl->stream);
    int G = d.groups > 0 ? d.groups : std::max(1, std::min(4, (int)nb / 8));
    G = std::max(1, std::min(G, (int)nb));
    pl->groups.resize(G);
    for (int gi = 0; gi < G; ++gi) {
        const int b0 = (int)(nb * gi / G), b1 = (int)(nb * (gi + 1) / G);
        cudaStream_t s = pl->stream;
        if (G > 1) {
            if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess)
                return bail("cudaStreamCreateWithFlags");
            pl->groups[gi].own_stream = true;
            if ((e = cudaEventCreateWithFlags(&pl->groups[gi].join, cudaEventDisableTiming)) != cudaSuccess)
                return bail("cudaEventCreate");
        }
        bind_exec(pl, pl->groups[gi], b0, b1 - b0, s);
    }
    if (G > 1 && (e = cudaEventCreateWithFlags(&pl->fork, cudaEventDisableTiming)) != cudaSuccess)
        return bail("cudaEventCreate");
    *out = pl;
    return SB_OK;
}

sb_status sb_plan_destroy(sb_plan pl) {
    if (!pl) return SB_OK;
    if (pl->stream) cudaStreamSynchronize(pl->stream);
    else cudaDeviceSynchronize();
    for (void* p : {(void*)pl->tw_x, (void*)pl->tw_y, (void*)pl->maskw, (void*)pl->slot, (void*)pl->lines,
                    (void*)pl->k, (void*)pl->invk, (void*)pl->kd, (void*)pl->r, (void*)pl->p, (void*)pl->q, (void*)pl->tb,
                    (void*)pl->bx[0], (void*)pl->bx[1], (void*)pl->by[0], (void*)pl->by[1], (void*)pl->bw,
                    (void*)pl->g, (void*)pl->bd, (void*)pl->bd1, (void*)pl->yt, (void*)pl->yt1, (void*)pl->st,
                    (void*)pl->part, (void*)pl->counter, (void*)pl->kmax, (void*)pl->derr, (void*)pl->spec,
                    (void*)pl->gb, (void*)pl->rb, (void*)pl->line_val, (void*)pl->line_uni, (void*)pl->jw,
                    (void*)pl->tw_z, (void*)pl->bz[0], (void*)pl->bz[1], (void*)pl->mask8, (void*)pl->wb,
                    (void*)pl->tw_full, pl->bmat})
        dfree(p);
    if (pl->h_st) cudaFreeHost(pl->h_st);
    auto release = [](Exec& ex) {
        for (const auto& pe : ex.pending) {
            cudaEventDestroy(pe.a);
            cudaEventDestroy(pe.b);
        }
        for (cudaEvent_t e : ex.ev_pool) cudaEventDestroy(e);
        if (ex.join) cudaEventDestroy(ex.join);
        for (const auto& g : ex.graphs) cudaGraphExecDestroy(g.exec);
        if (ex.own_stream) {
            cudaStreamSynchronize(ex.s);
            cudaStreamDestroy(ex.s);
        }
    };
    release(pl->whole);
    for (Exec& ex : pl->groups) release(ex);
    if (pl->fork) cudaEventDestroy(pl->fork);
    delete pl;
    return SB_OK;
}

// retire every captured PCG graph of the plan (after the plan's work on them has finished)
void drop_graphs(sb_plan pl) {
    auto drop = [](Exec& ex) {
        if (ex.graphs.empty()) return;
        cudaStreamSynchronize(ex.s);
        for (const auto& g : ex.graphs) cudaGraphExecDestroy(g.exec);
        ex.graphs.clear();
    };
    drop(pl->whole);
    for (Exec& ex : pl->groups) drop(ex);
}

sb_status sb_set_coils(sb_plan pl, const void* d_sens) {
    if (!pl || !d_sens) return fail(pl, SB_ERR_INVALID_ARG, "null plan or sensitivities");
    if (reinterpret_cast<uintptr_t>(d_sens) % 16 != 0)
        return fail(pl, SB_ERR_INVALID_ARG, "sensitivities must be 16-byte aligned");
    const Dims& d = pl->dims;
    const size_t per = (size_t)d.nc * pl->n;
    auto enc = [&](Exec& ex) {
        const float2* base = static_cast<const float2*>(d_sens) + (size_t)ex.b0 * per;
        const size_t rows = (size_t)ex.d.nb * d.nc * d.ny;
        const int box = coil_box_rows(d.ny);  // a TMA box spans at most 256 rows
        return encode_rows(&ex.smap, base, d.nx, rows, box) && encode_rows(&ex.smap_sw, base, d.nx, rows, box, true) &&
               ((pl->d.prec == SB_PREC_FP32 && d.ny != 256 && d.ny != 512) ||
                encode_rows(&ex.smap_sw64, base, d.nx, rows, 256, true, 8, CU_TENSOR_MAP_SWIZZLE_64B));
    };
    bool ok = true;
    if (pl->nz == 1) {  // the TMA coil-tile maps serve the 2D kernels only
        ok = enc(pl->whole);
        for (Exec& ex : pl->groups) ok = ok && enc(ex);
    }
    if (!ok) return fail(pl, SB_ERR_CUDA, "cuTensorMapEncodeTiled failed for the sensitivities");
    pl->sens = static_cast<const float2*>(d_sens);
    pl->have_coils = true;
    pl->jw_ready = false;
    pl->have_mask = false;  // k depends on the coils: rebuilt by sb_set_mask
    return SB_OK;
}

sb_status sb_set_mask(sb_plan pl, const uint8_t* d_mask) {
    if (!pl || !d_mask) return fail(pl, SB_ERR_INVALID_ARG, "null plan or mask");
    if (!pl->have_coils) return fail(pl, SB_ERR_NOT_READY, "call sb_set_coils before sb_set_mask");
    Exec& ex = pl->whole;
    const Dims& d = pl->dims;
    const size_t nb = d.nb, n = pl->n;
    cudaStream_t s = pl->stream;
    // scratch of the k construction, allocated once per plan
    if (!pl->spec) {
        SB_CK(pl, dalloc(&pl->line_val, nb * d.ny));
        SB_CK(pl, dalloc(&pl->line_uni, nb * d.ny));
        SB_CK(pl, dalloc(&pl->spec, nb * d.nc * n));
        SB_CK(pl, dalloc(&pl->gb, nb * n));
        SB_CK(pl, dalloc(&pl->rb, nb * n));
        SB_CK(pl, dalloc(&pl->jw, nb * n));
    }
    // 1. line structure of the mask
    int *lv = pl->line_val, *lu = pl->line_uni;
    sb_status st = SB_OK;
    auto step = [&]() -> sb_status {
        SB_LAUNCH(ex, SB_KCLASS_OTHER, 1, launch_mask_lines(d, d_mask, lv, lu, s));
        return SB_OK;
    };
    if ((st = step()) != SB_OK) return fail(pl, st, ex.err);
    std::vector<int> hv(nb * d.ny), hu(nb * d.ny);
    SB_CK(pl, cudaMemcpyAsync(hv.data(), lv, sizeof(int) * hv.size(), cudaMemcpyDeviceToHost, s));
    SB_CK(pl, cudaMemcpyAsync(hu.data(), lu, sizeof(int) * hu.size(), cudaMemcpyDeviceToHost, s));
    SB_CK(pl, cudaStreamSynchronize(s));
    bool lines_only = true;
    for (size_t i = 0; i < hu.size(); ++i) lines_only = lines_only && hu[i];
    if (!lines_only && pl->d.prec != SB_PREC_FP32)
        return fail(pl, SB_ERR_UNSUPPORTED, "the split-precision modes need a mask constant along the readout (x) axis");
    pl->general = !lines_only;
    pl->general_cluster = pl->general && pl->nz == 1 && apply_A_general_ok(Dims{d.nx, d.ny, d.nc, 1});
    int ms = 1;
    std::vector<float> hw(nb * d.ny);
    std::vector<int> hs(nb * d.ny), hl;
    if (pl->general) {
        // every row is a k-space row of the data; hw = sampled fraction contributed by the row
        std::vector<uint8_t> hm(nb * n);
        SB_CK(pl, cudaMemcpy(hm.data(), d_mask, nb * n, cudaMemcpyDeviceToHost));
        ms = d.ny;
        hl.assign(nb * ms, 0);
        for (size_t b = 0; b < nb; ++b)
            for (int y = 0; y < d.ny; ++y) {
                int c = 0;
                for (int xx = 0; xx < d.nx; ++xx) c += hm[(b * d.ny + y) * d.nx + xx] != 0;
                hw[b * d.ny + y] = (float)c / (float)n;
                hs[b * d.ny + y] = y;
                hl[b * ms + y] = y;
            }
        if (!pl->mask8) SB_CK(pl, dalloc(&pl->mask8, nb * n));
        SB_CK(pl, cudaMemcpyAsync(pl->mask8, d_mask, nb * n, cudaMemcpyDeviceToDevice, s));
    } else {
        for (size_t b = 0; b < nb; ++b) {
            int c = 0;
            for (int y = 0; y < d.ny; ++y) c += hv[b * d.ny + y] != 0;
            ms = std::max(ms, c);
        }
        hl.assign(nb * ms, -1);
        for (size_t b = 0; b < nb; ++b) {
            int c = 0;
            for (int y = 0; y < d.ny; ++y) {
                const bool on = hv[b * d.ny + y] != 0;
                hw[b * d.ny + y] = on ? 1.0f / d.ny : 0.0f;
                hs[b * d.ny + y] = on ? c : -1;
                if (on) hl[b * ms + c++] = y;
            }
        }
    }
    if (ms != pl->ms) {
        dfree(pl->lines);
        pl->lines = nullptr;
        SB_CK(pl, dalloc(&pl->lines, nb * ms));
    }
    pl->ms = ms;
    SB_CK(pl, cudaMemcpyAsync(pl->maskw, hw.data(), sizeof(float) * hw.size(), cudaMemcpyHostToDevice, s));
    SB_CK(pl, cudaMemcpyAsync(pl->slot, hs.data(), sizeof(int) * hs.size(), cudaMemcpyHostToDevice, s));
    SB_CK(pl, cudaMemcpyAsync(pl->lines, hl.data(), sizeof(int) * hl.size(), cudaMemcpyHostToDevice, s));

    // 2. k = mu k_c + lam k_d + gam by FFTs (Eq. Kdiag, Eq. diagonalelements)
    float2 *spec = pl->spec, *gb = pl->gb, *rb = pl->rb;
    const int nimg_c = d.nb * d.nc;
    // unnormalised 2D / 3D DFT of nimg images: rows (x), per-plane columns (y), z columns
    const int nyp = pl->ny_plane, nz = pl->nz;
    const Dims dp{d.nx, nyp, d.nc, d.nb};  // plane dims
    auto fft_nd = [&](float2* data, int nimg, bool inv) -> sb_status {
        SB_LAUNCH(ex, SB_KCLASS_OTHER, 1, launch_fft_rows(d.nx, d.ny, nimg, data, pl->tw_x, inv, s));
        SB_LAUNCH(ex, SB_KCLASS_OTHER, 1, launch_fft_cols(d.nx, nyp, nimg * nz, data, pl->tw_y, inv, s));
        if (nz > 1) SB_LAUNCH(ex, SB_KCLASS_OTHER, 1, launch_fft_cols(d.nx * nyp, nz, nimg, data, pl->tw_z, inv, s));
        return SB_OK;
    };
    auto build_k = [&]() -> sb_status {
        if (nz == 1) {  // rows out of place from the sensitivities, then columns + coil sum in one pass
            SB_LAUNCH(ex, SB_KCLASS_OTHER, 1,
                      launch_fft_rows_from(d.nx, d.ny, nimg_c, pl->sens, spec, pl->tw_x, false, s));
            SB_LAUNCH(ex, SB_KCLASS_OTHER, 1, launch_coil_power_cols(d, spec, gb, pl->tw_y, s));
        } else {
            SB_CK(pl, cudaMemcpyAsync(spec, pl->sens, sizeof(float2) * nb * d.nc * n, cudaMemcpyDeviceToDevice, s));
            if (sb_status e2 = fft_nd(spec, nimg_c, false)) return e2;
            SB_LAUNCH(ex, SB_KCLASS_OTHER, 1, launch_coil_power(d, spec, gb, s));
        }
        SB_LAUNCH(ex, SB_KCLASS_OTHER, 1, launch_mask_to_complex(d, d_mask, rb, s));
        if (sb_status e2 = fft_nd(gb, d.nb, false)) return e2;
        if (sb_status e2 = fft_nd(rb, d.nb, false)) return e2;
        SB_LAUNCH(ex, SB_KCLASS_OTHER, 1, launch_mul_conj(d, rb, gb, s));
        if (sb_status e2 = fft_nd(rb, d.nb, true)) return e2;
        SB_LAUNCH(ex, SB_KCLASS_OTHER, 2,
                  launch_finish_k(dp, nz, rb, pl->kd, (float)pl->d.mu, (float)pl->d.lambda, (float)pl->d.gamma, pl->k,
                                  pl->invk, pl->kmax, s));
        pl->jw_ready = false;  // the Jacobi weights are built by the first solve that uses them
        return SB_OK;
    };
    if ((st = build_k()) != SB_OK) return fail(pl, st, ex.err);
    SB_CK(pl, cudaStreamSynchronize(s));
    timer_harvest(ex);

    // 3. Split Bregman workspace sized by the number of sampled lines
    const size_t yt_elems = nb * d.nc * (size_t)ms * d.nx;
    if (yt_elems != pl->yt_elems) {
        dfree(pl->yt);
        dfree(pl->yt1);
        pl->yt = pl->yt1 = nullptr;
        SB_CK(pl, dalloc(&pl->yt, yt_elems));
        SB_CK(pl, dalloc(&pl->yt1, yt_elems));
        pl->yt_elems = yt_elems;
    }
    const size_t yrow = (size_t)d.nc * ms * d.nx;
    auto enc = [&](Exec& e2) {
        const size_t rows = (size_t)e2.d.nb * d.nc * ms;
        if (ms > 256 || pl->passes()) return true;  // no compact-row maps (2D line RHS kernel only)
        return encode_rows(&e2.ymap, pl->yt + e2.b0 * yrow, d.nx, rows, ms) &&
               encode_rows(&e2.y1map, pl->yt1 + e2.b0 * yrow, d.nx, rows, ms) &&
               ((d.ny != 256 && d.ny != 512) ||
                (encode_rows(&e2.ymap8, pl->yt + e2.b0 * yrow, d.nx, rows, ms, true, 8, CU_TENSOR_MAP_SWIZZLE_64B) &&
                 encode_rows(&e2.y1map8, pl->yt1 + e2.b0 * yrow, d.nx, rows, ms, true, 8, CU_TENSOR_MAP_SWIZZLE_64B)));
    };
    bool ok = enc(pl->whole);
    for (Exec& e2 : pl->groups) ok = ok && enc(e2);
    if (!ok) return fail(pl, SB_ERR_CUDA, "cuTensorMapEncodeTiled failed for the k-space rows");
    if (pl->d.wavelet == 1 && !pl->wb) SB_CK(pl, dalloc(&pl->wb, nb * n));
    if (pl->nz > 1 && !pl->bz[0]) {
        SB_CK(pl, dalloc(&pl->bz[0], nb * n));
        SB_CK(pl, dalloc(&pl->bz[1], nb * n));
    }
    if (!pl->g) {
        SB_CK(pl, dalloc(&pl->bx[0], nb * n));
        SB_CK(pl, dalloc(&pl->bx[1], nb * n));
        SB_CK(pl, dalloc(&pl->by[0], nb * n));
        SB_CK(pl, dalloc(&pl->by[1], nb * n));
        SB_CK(pl, dalloc(&pl->bw, nb * n));
        SB_CK(pl, dalloc(&pl->bd, nb * n));
        SB_CK(pl, dalloc(&pl->bd1, nb * n));
        SB_CK(pl, dalloc(&pl->g, nb * n));
    }
    pl->have_mask = true;
    return SB_OK;
}

sb_status sb_get_k(sb_plan pl, float* d_k) {
    if (sb_status s = check_ready(pl)) return s;
    if (!d_k) return fail(pl, SB_ERR_INVALID_ARG, "null output");
    SB_CK(pl, cudaMemcpyAsync(d_k, pl->k, sizeof(float) * pl->n * pl->dims.nb, cudaMemcpyDeviceToDevice, pl->stream));
    return SB_OK;
}

sb_status sb_apply_A(sb_plan pl, const void* d_x, void* d_y) {
    if (sb_status s = check_ready(pl)) return s;
    if (!d_x || !d_y || d_x == d_y) return fail(pl, SB_ERR_INVALID_ARG, "need distinct non-null x and y");
    Exec& ex = pl->whole;
    auto go = [&]() -> sb_status {
        if (pl->passes()) return vol_apply_A(ex, static_cast<const float2*>(d_x), static_cast<float2*>(d_y), false);
        SB_LAUNCH(ex, SB_KCLASS_APPLY_A, 1,
                  apply_A_2d(pl, ex, pl->dims, static_cast<const float2*>(d_x), static_cast<float2*>(d_y),
                             pl->maskw, nullptr, ex.red, pl->stream));
        return SB_OK;
    };
    sb_status st = go();
    return st == SB_OK ? st : fail(pl, st, ex.err);
}

sb_status sb_apply_precond(sb_plan pl, const void* d_r, void* d_z) {
    if (sb_status s = check_ready(pl)) return s;
    if (!d_r || !d_z) return fail(pl, SB_ERR_INVALID_ARG, "null vector");
    Exec& ex = pl->whole;
    const Dims& d = pl->dims;
    auto go = [&]() -> sb_status {
        if (pl->nz > 1)
            return vol_precond(ex, 0, const_cast<float2*>(static_cast<const float2*>(d_r)), nullptr, nullptr, nullptr,
                               static_cast<float2*>(d_z), 0.0);
        SB_LAUNCH(ex, SB_KCLASS_PRECOND_ROW_FWD, 1,
                  launch_row_fwd(d, 0, const_cast<float2*>(static_cast<const float2*>(d_r)), nullptr, pl->tb, pl->tw_x,
                                 nullptr, 0.0, ex.red, pl->stream));
        SB_LAUNCH(ex, SB_KCLASS_PRECOND_COL, 1,
                  launch_col_precond(d, pl->tb, pl->invk, pl->tw_y, nullptr, 0, ex.red, pl->stream,
                                     pl->col_tile));
        SB_LAUNCH(ex, SB_KCLASS_PRECOND_ROW_INV, 1,
                  launch_row_inv(d, 0, pl->tb, static_cast<float2*>(d_z), nullptr, nullptr, pl->tw_x, nullptr, ex.red,
                                 pl->stream));
        return SB_OK;
    };
    sb_status st = go();
    return st == SB_OK ? st : fail(pl, st, ex.err);
}

// the Jacobi weights 1 / diag(A) for the current coils and mask, on the plan stream before the
// solve's work (only solves that ask for the Jacobi preconditioner need them)
sb_status ensure_jacobi(sb_plan pl, int precond) {
    if (precond != SB_PRECOND_JACOBI || pl->jw_ready) return SB_OK;
    Exec& ex = pl->whole;
    const Dims dp{pl->dims.nx, pl->ny_plane, pl->dims.nc, pl->dims.nb};
    SB_LAUNCH(ex, SB_KCLASS_OTHER, 1,
              launch_jacobi_diag(dp, pl->nz, pl->sens, pl->maskw, (float)pl->d.mu, (float)pl->d.lambda,
                                 (float)pl->d.gamma, pl->jw, ex.s));
    pl->jw_ready = true;
    return SB_OK;
}

sb_status sb_pcg_solve(sb_plan pl, const void* d_b, void* d_x, const sb_pcg_opts* o, sb_pcg_result* h_results) {
    if (sb_status s = check_ready(pl)) return s;
    if (sb_status s = check_opts(pl, o)) return s;
    if (sb_status s = ensure_jacobi(pl, o->precond)) return s;
    if (!d_b || !d_x || d_b == d_x) return fail(pl, SB_ERR_INVALID_ARG, "need distinct non-null b and x");
    float2* x_full = static_cast<float2*>(d_x);
    const float2* b_full = static_cast<const float2*>(d_b);
    const double tol2 = o->fixed_iters > 0 ? -1.0 : o->tol * o->tol;
    return run_groups(pl, [&](Exec& ex) -> sb_status {
        const size_t n = pl->n;
        float2* x = at(x_full, ex, n);
        float2* q = at(pl->q, ex, n);
        if (pl->passes()) {
            if (sb_status e = vol_apply_A(ex, x, q, false)) return e;
        } else {
            SB_LAUNCH(ex, SB_KCLASS_APPLY_A, 1,
                      apply_A_2d(pl, ex, ex.d, x, q, at(pl->maskw, ex, (size_t)ex.d.ny), nullptr, ex.red, ex.s));
        }
        SB_LAUNCH(ex, SB_KCLASS_VEC, 1,
                  launch_resid_init(ex.d, at(b_full, ex, n), q, at(pl->r, ex, n), ex.st, tol2, ex.red, ex.s));
        return pcg_run(ex, *o, x_full, h_results, nullptr, 0);
    });
}

sb_status sb_split_bregman(sb_plan pl, const void* d_y, void* d_x, const sb_sb_opts* o, sb_pcg_result* h_last) {
    if (sb_status s = check_ready(pl)) return s;
    if (!o || !d_y || !d_x) return fail(pl, SB_ERR_INVALID_ARG, "null argument");
    if (reinterpret_cast<uintptr_t>(d_x) % 16 != 0)
        return fail(pl, SB_ERR_INVALID_ARG, "the image buffer must be 16-byte aligned");
    if (o->n_outer < 1 || o->n_inner < 1) return fail(pl, SB_ERR_INVALID_ARG, "n_outer and n_inner must be >= 1");
    if (sb_status s = check_opts(pl, &o->pcg)) return s;
    if (sb_status s = ensure_jacobi(pl, o->pcg.precond)) return s;
    if (!pl->passes() && (pl->ms > 256 || rhs_smem_bytes(pl->dims.ny, pl->ms) > 227 * 1024))
        return fail(pl, SB_ERR_UNSUPPORTED, "too many sampled lines for the shared-memory pipeline of this size");
    const int nsolve = o->n_outer * o->n_inner;
    std::vector<int> iters((size_t)pl->dims.nb * nsolve, 0);
    const float2* y = static_cast<const float2*>(d_y);
    float2* x = static_cast<float2*>(d_x);
    sb_status st = run_groups(pl, [&](Exec& ex) { return sb_run(ex, *o, y, x, h_last, iters.data()); });
    if (st != SB_ERR_CUDA && st != SB_ERR_TIMEOUT) {
        SB_CK(pl, cudaStreamSynchronize(pl->stream));
        if (o->h_iters) std::memcpy(o->h_iters, iters.data(), sizeof(int) * iters.size());
    }
    return st;
}

sb_status sb_split_bregman_many(const sb_plan* plans, int nplans, const void* const* d_y, void* const* d_x,
                                const sb_sb_opts* opts, sb_pcg_result* const* h_last) {
    if (!plans || nplans < 1 || !d_y || !d_x || !opts) return SB_ERR_INVALID_ARG;
    for (int i = 0; i < nplans; ++i) {
        if (!plans[i]) return SB_ERR_INVALID_ARG;
        for (int k = 0; k < i; ++k)
            if (plans[k] == plans[i]) return fail(plans[i], SB_ERR_INVALID_ARG, "a plan appears twice");
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SB_ERR_CUDA;
    std::vector<sb_status> st(nplans, SB_OK);
    auto run = [&](int i) {
        st[i] = sb_split_bregman(plans[i], d_y[i], d_x[i], &opts[i], h_last ? h_last[i] : nullptr);
    };
    std::vector<std::thread> th;
    th.reserve(nplans - 1);
    for (int i = 1; i < nplans; ++i)
        th.emplace_back([&, i] {
            if (cudaSetDevice(dev) != cudaSuccess) {
                st[i] = fail(plans[i], SB_ERR_CUDA, "cudaSetDevice in a worker thread");
                return;
            }
            run(i);
        });
    run(0);
    for (auto& t : th) t.join();
    for (int i = 0; i < nplans; ++i)
        if (st[i] != SB_OK) return st[i];
    return SB_OK;
}

sb_status sb_set_tuning(sb_plan pl, const sb_tuning* t) {
    if (!pl || !t) return SB_ERR_INVALID_ARG;
    if (t->col_tile != 0 && !col_tile_ok(pl->ny_plane, pl->dims.nx, t->col_tile))
        return fail(pl, SB_ERR_UNSUPPORTED, "col_tile must be 8, 16 or 32, divide nx and fit the column pass");
    if (t->poll_every < 0 || t->poll_every > 64) return fail(pl, SB_ERR_INVALID_ARG, "poll_every must be 0..64");
    if (t->apply_tile != 0 && t->apply_tile != 8 && t->apply_tile != 16)
        return fail(pl, SB_ERR_INVALID_ARG, "apply_tile must be 0, 8 or 16");
    if (t->general_passes != 0 && t->general_passes != 1 && t->general_passes != 3)
        return fail(pl, SB_ERR_INVALID_ARG, "general_passes must be 0, 1 or 3");
    SB_CK(pl, pl->stream ? cudaStreamSynchronize(pl->stream) : cudaDeviceSynchronize());
    if (t->col_tile) pl->col_tile = t->col_tile;
    if (t->poll_every) pl->poll_every = t->poll_every;
    if (t->apply_tile) pl->apply_tile = t->apply_tile;
    if (t->general_passes) pl->general_passes = t->general_passes;
    drop_graphs(pl);
    return SB_OK;
}

sb_status sb_get_tuning(sb_plan pl, sb_tuning* t) {
    if (!pl || !t) return SB_ERR_INVALID_ARG;
    t->col_tile = pl->col_tile;
    t->poll_every = pl->poll_every;
    t->apply_tile = pl->apply_tile;
    t->general_passes = pl->general_passes;
    return SB_OK;
}

sb_status sb_set_graphs(sb_plan pl, int enable) {
    if (!pl) return SB_ERR_INVALID_ARG;
    SB_CK(pl, pl->stream ? cudaStreamSynchronize(pl->stream) : cudaDeviceSynchronize());
    pl->graphs = enable != 0;
    drop_graphs(pl);
    return SB_OK;
}

sb_status sb_set_wait_check(sb_plan pl, unsigned wait_polls, int withhold_coil_tiles) {
    if (!pl) return SB_ERR_INVALID_ARG;
    if (wait_polls > kWaitLimit) return fail(pl, SB_ERR_INVALID_ARG, "wait_polls above the default limit");
    SB_CK(pl, pl->stream ? cudaStreamSynchronize(pl->stream) : cudaDeviceSynchronize());
    for (Exec& ex : pl->groups) SB_CK(pl, cudaStreamSynchronize(ex.s));
    pl->wait_limit = wait_polls ? wait_polls : kWaitLimit;
    pl->red_flags = withhold_coil_tiles ? kRedWithholdCoilTiles : 0u;
    auto rebind = [pl](Exec& ex) {
        ex.red.wait_limit = pl->wait_limit;
        ex.red.flags = pl->red_flags;
    };
    rebind(pl->whole);
    for (Exec& ex : pl->groups) rebind(ex);
    drop_graphs(pl);  // captured launches hold the old Red by value
    SB_CK(pl, cudaMemset(pl->derr, 0, sizeof(unsigned)));
    SB_CK(pl, cudaDeviceSynchronize());
    return SB_OK;
}

sb_status sb_plan_set_timing(sb_plan pl, unsigned class_mask) {
    if (!pl) return SB_ERR_INVALID_ARG;
    SB_CK(pl, pl->stream ? cudaStreamSynchronize(pl->stream) : cudaDeviceSynchronize());
    timer_harvest(pl->whole);
    for (Exec& ex : pl->groups) timer_harvest(ex);
    std::lock_guard<std::mutex> lock(pl->tmu);
    pl->tmask = class_mask;
    for (int c = 0; c < SB_KCLASS_COUNT; ++c) {
        pl->tcount[c] = 0;
        pl->tms[c] = 0.0;
    }
    return SB_OK;
}

sb_status sb_plan_get_timing(sb_plan pl, int kernel_class, uint64_t* launches, double* total_ms) {
    if (!pl || kernel_class < 0 || kernel_class >= SB_KCLASS_COUNT || !launches || !total_ms)
        return fail(pl, SB_ERR_INVALID_ARG, "bad timing query");
    SB_CK(pl, pl->stream ? cudaStreamSynchronize(pl->stream) : cudaDeviceSynchronize());
    timer_harvest(pl->whole);
    for (Exec& ex : pl->groups) timer_harvest(ex);
    std::lock_guard<std::mutex> lock(pl->tmu);
    *launches = pl->tcount[kernel_class];
    *total_ms = pl->tms[kernel_class];
    return SB_OK;
}

}  // extern "C"
