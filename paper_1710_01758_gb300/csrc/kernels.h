// Internal interface between the C-ABI layer (sb_api.cu) and the CUDA kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sb {

// Columns per CTA of the column kernels; the TMA box of a coil tile is kColTile x ny.
constexpr int kColTile = 16;

// Per-slice CG state; lives in device memory, one entry per slice of the batch.
enum : int {
    ST_ACTIVE = 0,     // iterating
    ST_FINISHING = 1,  // tolerance met by the residual update of this iteration: apply x += a p
    ST_DONE = 2,       // converged
    ST_BREAKDOWN = 3,  // Re(p^H A p) <= 0
    ST_NONFINITE = 4,  // NaN / Inf in a CG scalar
    ST_ZERO = 5,       // ||b|| = 0: the solution is x = 0
};

struct SliceState {
    double rho;     // r^H z of the current iterate
    double alpha;   // step length of the current iteration
    double beta;    // direction update of the current iteration
    double bnorm2;  // ||b||^2
    double rnorm2;  // ||r||^2 after the latest residual update
    double pq;      // Re(p^H A p) of the current iteration
    int state;
    int iters;      // A applications since the initial residual
};

// rows of one TMA box of a coil tile (boxes span at most 256 rows and must tile ny)
__host__ __device__ constexpr int coil_box_rows(int ny) { return ny <= 256 ? ny : (ny % 256 == 0 ? 256 : ny / 2); }

// Raise a kernel's dynamic shared-memory limit to `bytes`, once per (kernel, device): the
// attribute is one setting shared by all host threads, and a driver call before every launch
// costs more than the launch itself when several host threads drive slice groups.
cudaError_t set_smem_limit(const void* kernel, int bytes);
template <class F>
cudaError_t set_smem_limit(F* kernel, int bytes) {
    return set_smem_limit(reinterpret_cast<const void*>(kernel), bytes);
}

struct Dims {
    int nx, ny, nc, nb;
};

// polls of a bounded mbarrier wait before it gives up (about half a second with the back-off)
constexpr uint32_t kWaitLimit = 1u << 22;
// Red::flags bit: the coil-tile kernels of the line path (q = A p, the right-hand side) issue
// no TMA load, so their waits for a tile run out (a check of the bounded waits; results are
// meaningless while it is set)
constexpr uint32_t kRedWithholdCoilTiles = 1u;

// Workspace of the cross-CTA reductions: part[nb][maxparts][K] doubles, counter[nb]; err is
// the device error word (bit kErrTmaTimeout: a bounded TMA wait gave up); wait_limit: polls of
// each bounded wait; flags: kRedWithholdCoilTiles or 0.
struct Red {
    double* part;
    unsigned* counter;
    unsigned* err;
    uint32_t wait_limit = kWaitLimit;
    uint32_t flags = 0;
};

// minimum per-slice capacity of Red::part (plans raise it to their widest launch: rows / 16,
// column tiles x planes, z columns of a volume)
constexpr int kMaxParts = 1024;
constexpr int kVecThreads = 256;
constexpr int kVecPerThread = 8;

// ------------------------------------------------------------------ PCG kernels (k_pcg.cu)
// q = A p (readout-axis shortcut of the data term); st == nullptr: plain application;
// otherwise PCG mode: skips inactive slices, accumulates Re(p^H q) and sets alpha = rho/pq.
// smap: TMA map of the sensitivities viewed as float32 [nb*nc*ny][2*nx], box [ny][2*kColTile]
// with the 128-byte swizzle; smap8: the same rows as 8-column boxes of 256 rows with the 64-byte
// swizzle (read at ny = 256 and 512).  tile: columns per CTA there, 8 (tensor-memory kernel) or 16.
cudaError_t launch_apply_A(const Dims& d, const CUtensorMap& smap, const CUtensorMap& smap8, const float2* p,
                           float2* q, const float* maskw, const float2* tw_y, float mu, float lam, float gam,
                           SliceState* st, Red red, cudaStream_t s, int tile = 8);

// q = A p on 2D slices with an arbitrary mask (mask: u8 [nb][ny][nx]) in one launch: a thread-block
// cluster per slice keeps every coil's 2D spectrum in distributed shared memory (k_general.cu).
// st == nullptr: plain application; otherwise PCG mode as launch_apply_A.  nx, ny in {64, 128,
// 256}; apply_A_general_ok tells whether the device can run the shape.
bool apply_A_general_ok(const Dims& d);
cudaError_t launch_apply_A_general(const Dims& d, const float2* sens, const float2* p, float2* q, const uint8_t* mask,
                                   const float2* tw_x, const float2* tw_y, float mu, float lam, float gam,
                                   SliceState* st, Red red, cudaStream_t s);

// q = A p with the radix-16 DFT stages on the tensor cores, operands split in two bf16 or fp16
// terms with FP32 accumulation (the split-precision modes; ny = 256 or 512, nx a multiple of 8).
// smap8: the coil maps as 8-column x 256-row boxes with the 64-byte swizzle; tw: W_256^m, m < 256;
// bmat: tc_bmat_bytes() of DFT-matrix operands from build_tc_bmat (same bf16 flag).
struct TcOperands {
    const CUtensorMap* smap8;
    const float2* tw;
    const void* bmat;
    bool bf16;
};
bool apply_A_tc_supported(const Dims& d);
cudaError_t launch_apply_A_tc(const Dims& d, const TcOperands& tc, const float2* p, float2* q, const float* maskw,
                              float mu, float lam, float gam, SliceState* st, Red red, cudaStream_t s);
size_t tc_bmat_bytes();
void build_tc_bmat(bool bf16, uint16_t* img);  // img: tc_bmat_bytes() / 2 entries

// Row pass of M^{-1}: mode 0 = t = F_x(in) (no CG work); mode 1 = PCG update r -= alpha q,
// ||r||^2, convergence test, t = F_x(r).
cudaError_t launch_row_fwd(const Dims& d, int mode, float2* r, const float2* q, float2* t,
                           const float2* tw_x, SliceState* st, double tol2, Red red, cudaStream_t s);

// Column pass of M^{-1}: t <- F_y^H diag(invk) F_y t (in place); with st != nullptr also
// rho_new = sum |F t|^2 invk and (init = 0) beta = rho_new / rho, rho = rho_new or
// (init = 1) rho = rho_new.
// ct: columns per CTA of the column pass (8, 16 or 32; a tuning choice, see col_tile_ok)
cudaError_t launch_col_precond(const Dims& d, float2* t, const float* invk, const float2* tw_y,
                               SliceState* st, int init, Red red, cudaStream_t s, int ct = kColTile);
// whether `ct` columns per CTA fit the column pass at (ny, nx): 8 | 16 | 32 dividing nx, at most
// 1024 threads and 160 KB of exchange buffers
bool col_tile_ok(int ny, int nx, int ct);

// Row pass back: z = F_x^H t; mode 0: out = z; mode 1 (PCG init): p = z;
// mode 2 (PCG step): x += alpha p, p = z + beta p (FINISHING slices: x += alpha p, -> DONE).
cudaError_t launch_row_inv(const Dims& d, int mode, const float2* t, float2* out, float2* x,
                           float2* p, const float2* tw_x, SliceState* st, Red red, cudaStream_t s);

// CG with a diagonal preconditioner z = w r (w == nullptr: w = 1, plain CG; else w = 1 / diag(A),
// Jacobi): mode 0 (init): p = z, rho = r^H z; mode 1 (step, after q = A p): r -= alpha q,
// ||r||^2 test, beta = r^H z / rho; mode 2 (step): x += alpha p, p = z + beta p.
// The whole circulant M^{-1} step of PCG in one cluster launch per slice (k_precond_fused.cu):
// mode 0 (init): p = z = M^{-1} r, rho = r^H z; mode 1 (step, after q = A p): r -= alpha q,
// ||r||^2 test (converged: x += alpha p, done), z = M^{-1} r, beta, x += alpha p, p = z + beta p.
// nx, ny in {32, 64, 128, 256}.
bool precond_fused_shape_ok(const Dims& d);
// clusters of the fused kernel that fit on the device at once (0: cannot run)
int precond_fused_clusters(const Dims& d);
cudaError_t launch_precond_fused(const Dims& d, int mode, float2* x, float2* r, float2* p, const float2* q,
                                 const float* invk, const float2* tw_x, const float2* tw_y, SliceState* st,
                                 double tol2, cudaStream_t s);

cudaError_t launch_vec_plain(const Dims& d, int mode, float2* x, float2* r, float2* p,
                             const float2* q, const float* w, SliceState* st, double tol2, Red red,
                             cudaStream_t s);
// w = 1 / (mu nnz(r)/N sum_c |S_c|^2 + 4 lambda + gamma): the inverse diagonal of A (Jacobi).
cudaError_t launch_jacobi_diag(const Dims& d, int nz, const float2* sens, const float* maskw, float mu, float lam,
                               float gam, float* w, cudaStream_t s);

// r = b - q, ||b||^2, ||r||^2, initial convergence test and state.
cudaError_t launch_resid_init(const Dims& d, const float2* b, const float2* q, float2* r,
                              SliceState* st, double tol2, Red red, cudaStream_t s);

// x = 0 on slices whose ||b|| = 0, state -> DONE.
cudaError_t launch_zero_rhs_slices(const Dims& d, float2* x, SliceState* st, cudaStream_t s);

// ------------------------------------------------------------------ set-up kernels (k_setup.cu)
// Per slice and phase-encode line: flag whether the mask is constant along x and its value.
cudaError_t launch_mask_lines(const Dims& d, const uint8_t* mask, int* line_val, int* line_uniform,
                              cudaStream_t s);
// Generic batched unnormalised FFT of complex rows (along x) or columns (along y) of
// [nbatch_images][ny][nx] arrays, in place; inv selects the sign.
cudaError_t launch_fft_rows(int nx, int ny, int nimg, float2* data, const float2* tw_x, bool inv,
                            cudaStream_t s);
// the same row transform from src into dst (src == dst: in place)
cudaError_t launch_fft_rows_from(int nx, int ny, int nimg, const float2* src, float2* dst, const float2* tw_x,
                                 bool inv, cudaStream_t s);
cudaError_t launch_fft_cols(int nx, int ny, int nimg, float2* data, const float2* tw_y, bool inv,
                            cudaStream_t s);
// g[b] = sum_c |data[b][c]|^2 / N^2 (data: [nb][nc][N], the DFTs of the sensitivities);
// out as complex (imaginary part 0) for the next FFT.
cudaError_t launch_coil_power(const Dims& d, const float2* data, float2* g, cudaStream_t s);
// 2D planes: g[b] = sum_c |DFT_y(spec[b][c])|^2 / N^2 with spec the row-transformed sensitivities
// (the column transforms and the coil sum in one pass; spec is read only).
cudaError_t launch_coil_power_cols(const Dims& d, const float2* spec, float2* g, const float2* tw_y, cudaStream_t s);
// Pack the mask as complex: out[b][i] = (mask != 0, 0).
cudaError_t launch_mask_to_complex(const Dims& d, const uint8_t* mask, float2* out, cudaStream_t s);
// prod[b][i] = R[b][i] * conj(G[b][i])  (the spectra of r and g), in place in R.
cudaError_t launch_mul_conj(const Dims& d, float2* R, const float2* G, cudaStream_t s);
// k = mu Re(kc)/N + lam k_d + gam, clamped; invk = 1 / (k N).  kd: [N] k_d of the geometry
// (shared by the slices); kmax: nb words of scratch.
cudaError_t launch_finish_k(const Dims& d, int nz, const float2* kc_unscaled, const float* kd, float mu, float lam,
                            float gam, float* k, float* invk, unsigned* kmax, cudaStream_t s);

// ------------------------------------------------------------------ Split Bregman (k_sb.cu)
struct SbFields {
    const float2* sens;
    const float* maskw;   // [nb][ny]: 1/ny on sampled lines, 0 elsewhere
    const int* slot;      // [nb][ny]: compact index of a sampled line, -1 elsewhere
    const int* lines;     // [nb][ms]: the line of each compact index (2D line path)
    float2* yt;           // [nb][nc][ms][nx]: F_x^H y^[j] on sampled lines
    const float2* yt1;    // [nb][nc][ms][nx]: F_x^H y^[1]
    int ms;               // slots per slice
    const float2* bx;     // Bregman variables b_x, b_y before this update (read)
    const float2* by;
    float2* bx_new;       // ... after it (written; the caller swaps the two buffers)
    float2* by_new;
    const float2* bz;     // volumes: b_z before / after (nullptr in 2D)
    float2* bz_new;
    float2* bw;           // wavelet Bregman variable, tile-local Mallat layout, in place
    float2* g;            // lam Dx^H(dx-bx) + lam Dy^H(dy-by) + gam W^H(dw-bw)
    float2* bd;           // [nb][N]: data term of b for the current y^[j]: sum_c S_c^H F^H R y_c^[j]
    float2* bd1;          // [nb][N]: the same for y^[1]
};

// The right-hand side and initial residual of launch_rhs for 2D slices with an arbitrary mask
// (mask: u8 [nb][ny][nx]; f.yt, f.yt1: the whole k-space [nb][nc][ny][nx]) in one launch of the
// thread-block clusters of launch_apply_A_general (k_general.cu); the same shapes.
cudaError_t launch_rhs_general(const Dims& d, const SbFields& f, int addback, const float2* x, float2* r,
                               const uint8_t* mask, const float2* tw_x, const float2* tw_y, float mu, float lam,
                               float gam, SliceState* st, double tol2, Red red, cudaStream_t s);

// yt1[b][c][s][:] = F_x^H y[b][c][line(s)][:] (unitary).
cudaError_t launch_ytilde(const Dims& d, const float2* y, const int* lines, int ms, float2* yt1,
                          const float2* tw_x, cudaStream_t s);
// Start of Algorithm 1 from yt1: bd1 = bd = sum_c S_c^H F^H y_c and, if write_x,
// x = sqrt(sum_c |F^H y_c|^2).
cudaError_t launch_rss(const Dims& d, const SbFields& f, float2* x, int write_x, const float2* tw_y,
                       cudaStream_t s);
// Right-hand side and initial residual: optional outer data update yt += yt1 - R F S x,
// b = mu bd + g with bd advanced by linearity, r = b - A x; ||b||^2, ||r||^2, state.
// smap: as for launch_apply_A; ymap / y1map: TMA maps of yt / yt1 viewed as float32
// [nb*nc*ms][2*nx] with box [ms][2*kColTile]; at ny = 256 the 8-column maps with the 64-byte
// swizzle are read instead (smap8 as for launch_apply_A, ymap8 / y1map8 with box [ms][16]).
struct RhsMaps {
    const CUtensorMap *smap, *ymap, *y1map;
    const CUtensorMap *smap8, *ymap8, *y1map8;
};
cudaError_t launch_rhs(const Dims& d, const RhsMaps& maps, const SbFields& f, int addback, const float2* x,
                       float2* r, const float2* tw_y, float mu, float lam, float gam, SliceState* st,
                       double tol2, Red red, cudaStream_t s);
// Shared memory the right-hand-side kernel needs for ny and ms (bytes).
size_t rhs_smem_bytes(int ny, int ms);
// Shrink + Bregman updates (steps 6-11) and the next g.
cudaError_t launch_sb_update(const Dims& d, const SbFields& f, const float2* x, int levels,
                             float lam, float gam, float tau_tv, float tau_w, cudaStream_t s);

// ---- volumes (k_vol.cu): Dims are per plane (nx, ny, nc, nb volumes), nz planes each
// DFT along y of every plane (nplanes = nb * nz); st (optional) filters by volume.
cudaError_t launch_col_dft(int nx, int ny, int nplanes, int nz, float2* data, const float2* tw_y, bool inv,
                           const SliceState* st, cudaStream_t s);
// U[b][c] = DFT_y(S_c v) per plane.
cudaError_t launch_g3_fwd_y(const Dims& d, int nz, const float2* sens, const float2* v, float2* U, const float2* tw_y,
                            const SliceState* st, cudaStream_t s);
// DFT_z, mask operation (mode 0: A; 1: right-hand side with the outer update if addback;
// 2: back-projection of yt1), IDFT_z.
cudaError_t launch_g3_z(const Dims& d, int nz, int mode, int addback, float2* U, const int* slot, float2* yt,
                        const float2* yt1, int ms, const float2* tw_z, const SliceState* st, cudaStream_t s);
// 2D slices with an arbitrary mask (the x pass between the y passes, nz = 1): DFT_x, the
// per-point mask operation of `mode` (as launch_g3_z, on whole k-space rows), IDFT_x.
cudaError_t launch_g2_x(const Dims& d, int mode, int addback, float2* U, const uint8_t* mask, float2* yt,
                        const float2* yt1, const float2* tw_x, const SliceState* st, cudaStream_t s);
// IDFT_y, coil combine and the epilogue of the mode (0: q = A p, flag = PCG; 1: right-hand side,
// flag = addback; 2: bd1, bd and the RSS start if write_x).
cudaError_t launch_g3_inv_y(const Dims& d, int nz, int mode, int flag, const float2* U, const SbFields& f,
                            const float2* vin, float2* out, int write_x, const float2* tw_y, float mu, float lam,
                            float gam, SliceState* st, double tol2, Red red, cudaStream_t s);
// Daubechies-4 steps 8 and 11 (k_wave.cu): w = W x (levels >= 1, Mallat layout), shrink and
// Bregman update of bw, w = W^H (d_w - b_w), g += gam w.  w: [nb][ny][nx] scratch.
cudaError_t launch_d4_update(const Dims& d, const float2* x, float2* w, float2* bw, float2* g, int levels, float gam,
                             float tau_w, cudaStream_t s);
int d4_update_launches(int levels);
// Steps 6-11 of Algorithm 1 on 16^3 tiles (levels <= 4).
cudaError_t launch_sb_update3(const Dims& d, int nz, const SbFields& f, const float2* x, int levels, float lam,
                              float gam, float tau_tv, float tau_w, cudaStream_t s);


}  // namespace sb
