/*
 * sb.h — C ABI of a GB300 (sm_103a) library for the circulant-preconditioned conjugate-gradient
 * solve inside Split Bregman for parallel imaging + compressed sensing MRI
 * (Koolstra, van Gemert et al., arXiv 1710.01758).
 *
 * Problem (Theory, Eq. original and Eq. system):
 *   A = mu * sum_i (R F S_i)^H (R F S_i) + lambda (D_x^H D_x + D_y^H D_y) + gamma W^H W,
 * F the unitary 2D DFT, S_i diagonal coil sensitivities, R = diag(r) a binary k-space mask,
 * D_x, D_y periodic first-order differences, W an orthonormal (Haar) wavelet, so W^H W = I.
 * Preconditioner (Eq. precon, Eq. Kdiag): M^{-1} = F^H diag(k)^{-1} F with
 * k = mu k_c + lambda k_d + gamma, k_c the diagonal of F (sum_i S_i^H F^H R F S_i) F^H.
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are DEVICE pointers on the device that was current at sb_plan_create;
 *    h_* are host pointers.  The caller owns all of them.
 *  - Complex data is interleaved complex64 (float re, float im), C order, x fastest:
 *    an image is [nbatch][ny][nx]; coil data are [nbatch][ncoils][ny][nx].
 *  - k-space arrays are in DFT (unshifted) order; the DFT is unitary, forward sign negative.
 *  - All device work is enqueued on the plan's stream.  sb_apply_A and sb_apply_precond are
 *    asynchronous; sb_set_mask, sb_pcg_solve and sb_split_bregman synchronise the stream before
 *    they return (they report iteration counts to the host).
 *  - Errors are returned as sb_status, never by abort; sb_plan_last_error() gives a message.
 *    A CUDA error leaves the plan in an undefined numerical state (destroy it).
 *  - Masks (sb_set_mask): a 2D mask constant along the readout (x) axis (Cartesian
 *    phase-encode lines, the paper's first scheme in Methods, "Undersampling") takes the fast
 *    path, DFTs along y only; any other 2D mask (the paper's random 2D sampling) takes the
 *    general path, a per-point mask between DFTs along y and x.  On volumes (ndim = 3) a mask
 *    constant along x (sampled (k_y, k_z) lines) takes three passes per data-term operation and
 *    any other mask the general path's five (DFTs along y and z, the per-point mask between DFTs
 *    along x, inverse DFTs along z and y).  Split-precision plans need 2D line masks
 *    (SB_ERR_UNSUPPORTED otherwise).
 *  - Supported sizes: ndim = 2 (slices) or 3 (volumes of nz planes); nx, ny (and nz for
 *    volumes) in {32, 64, 128, 192, 224, 256, 320, 384, 512} (powers of two and
 *    16 x {12, 14, 20, 24}, mixed-radix transforms); ncoils >= 1; nbatch >= 1; wavelet_levels in
 *    [0, 5] for slices (Haar blocks stay inside the 32 x 32 update tiles) and [0, 4] for volumes
 *    (16^3 tiles).  Further limits of a precision mode or schedule are stated at its field.
 */
#ifndef SB_H
#define SB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SB_OK = 0,
    SB_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad option */
    SB_ERR_UNSUPPORTED = 2,   /* valid but not implemented (size, mask kind, precision) */
    SB_ERR_CUDA = 3,          /* a CUDA runtime call failed; message in sb_plan_last_error */
    SB_ERR_NOT_READY = 4,     /* coils / mask not set yet */
    SB_ERR_NONFINITE = 5,     /* NaN or Inf met in a CG scalar (rho, p^H A p, ||r||) */
    SB_ERR_BREAKDOWN = 6,     /* Re(p^H A p) <= 0: A not positive definite on the data */
    SB_ERR_NOT_CONVERGED = 7, /* maxit reached before the tolerance */
    SB_ERR_TIMEOUT = 8        /* a bounded device-side wait gave up (a TMA tile never arrived) */
} sb_status;

typedef enum { SB_PREC_FP32 = 0, SB_PREC_SPLIT_BF16 = 1, SB_PREC_SPLIT_FP16 = 2 } sb_precision;
typedef enum { SB_PRECOND_NONE = 0, SB_PRECOND_CIRCULANT = 1, SB_PRECOND_JACOBI = 2 } sb_precond;

typedef struct {
    int ndim;               /* 2: slices; 3: volumes of nz planes (x the readout; 3D k, 7-point
                               TV, 3D Haar on 16^3 tiles) */
    int nx, ny, nz;         /* image size, x fastest; each a supported transform length
                               (32, 64, 128, 192, 224, 256, 320, 384, 512); nz = 1 (or 0) in 2D */
    int ncoils;             /* N_c */
    int nbatch;             /* independent slices (volumes) of this geometry solved together (>= 1) */
    double mu, lambda, gamma;  /* weights of Eq. system; mu > 0, lambda >= 0, gamma >= 0 */
    int wavelet_levels;     /* Haar levels of W used by sb_split_bregman; 0 = identity W */
    sb_precision prec;      /* arithmetic of q = A p (Eq. system): SB_PREC_FP32 (FP32 DFTs), or
                               SB_PREC_SPLIT_BF16 / SB_PREC_SPLIT_FP16: the DFT stages along y
                               (256 = 16 x 16 or 512 = 16 x 32) run as tensor-core products on
                               operands split in two bf16 or fp16 terms, FP32 accumulation; 2D
                               line masks (a mask varying along x gives SB_ERR_UNSUPPORTED at
                               sb_set_mask), ny = 256 or 512, nx a multiple of 8, else
                               SB_ERR_UNSUPPORTED at create.  CG scalars stay FP64 in every mode. */
    int groups;             /* sb_pcg_solve / sb_split_bregman run the batch as this many
                               contiguous slice groups, each on its own stream driven by its own
                               host thread, so that one group's work fills the GPU while another
                               waits on its convergence test; 0 = automatic (nbatch / 8, at most
                               4, at least 1); clamped to [1, nbatch] */
    int precond_passes;     /* schedule of the circulant M^{-1} inside PCG: 1 = one launch per
                               iteration, each slice on one thread-block cluster that exchanges
                               the 2D spectrum through distributed shared memory (needs
                               nx * ny <= 65536 and nx, ny <= 256, else SB_ERR_UNSUPPORTED at
                               create); 3 = three launches (DFT along x, DFT along y with k^{-1}
                               and its inverse, inverse DFT along x) through an HBM buffer;
                               0 = automatic (3: on a 64-slice 256 x 256 batch the cluster
                               launch took 151 us against 92 us for the three passes).  Both
                               give the same iterates up to rounding order. */
    int wavelet;            /* W of steps 4, 8 and 11: 0 = orthonormal Haar (in place, 32 x 32
                               tiles), 1 = periodic Daubechies-4, the wavelet of the paper's
                               experiments (Methods, "Reconstruction"); 2D only, nx, ny <= 512,
                               and the coarsest band at least 4 wide, else SB_ERR_UNSUPPORTED.
                               A and k do not depend on W (W^H W = I). */
} sb_plan_desc;

typedef struct sb_plan_s* sb_plan;

/* Create a plan: validates the descriptor and allocates the plan's device workspace
 * (PCG vectors, Split Bregman fields, k^{-1}, FFT twiddles, CG scalars) on the current
 * device.  cuda_stream: a cudaStream_t (NULL = legacy default stream).  *out receives the plan.
 * No allocation happens after sb_set_mask. */
sb_status sb_plan_create(const sb_plan_desc* desc, void* cuda_stream, sb_plan* out);

/* Destroy a plan and free its workspace (synchronises its stream).  NULL is accepted. */
sb_status sb_plan_destroy(sb_plan plan);

/* Set the coil sensitivities S_i (Eq. ill0), complex64 [nbatch][ncoils][ny][nx].
 * BORROWED: d_sens is read by every later operator call and must stay alive and unchanged
 * until sb_plan_destroy or the next sb_set_coils.  Invalidates k: call sb_set_mask next. */
sb_status sb_set_coils(sb_plan plan, const void* d_sens);

/* Set the sampling mask r (R = diag(r), Eq. ill0), uint8 [nbatch][ny][nx], nonzero = sampled,
 * DFT order, and build k of Eq. Kdiag by FFTs (Eq. diagonalelements and the k_d paragraph of
 * "Efficient Implementation of the Preconditioner").  Requires sb_set_coils.  d_mask is read
 * during this call only.  Synchronises the stream.  A 2D mask that varies along x (the paper's
 * random sampling, Methods, "Undersampling") switches the plan to the general path: q = A p in
 * one cluster launch (nx, ny in {64, 128, 256}) or three passes with a per-point mask, the
 * right-hand side in three passes; a volume mask that varies along x does too (five passes).
 * Returns SB_ERR_UNSUPPORTED for such a mask on a split-precision plan. */
sb_status sb_set_mask(sb_plan plan, const uint8_t* d_mask);

/* Copy k (float32 [nbatch][ny][nx], DFT order, before inversion) into d_k. */
sb_status sb_get_k(sb_plan plan, float* d_k);

/* d_y = A d_x for every slice (Eq. system).  complex64 [nbatch][ny][nx] each; d_x and d_y
 * must not overlap.  Asynchronous. */
sb_status sb_apply_A(sb_plan plan, const void* d_x, void* d_y);

/* d_z = M^{-1} d_r = F^H diag(k)^{-1} F d_r (Eq. precon).  complex64 [nbatch][ny][nx];
 * d_r and d_z may be equal (in place).  Asynchronous. */
sb_status sb_apply_precond(sb_plan plan, const void* d_r, void* d_z);

typedef struct {
    double tol;          /* stop when ||b - A x|| <= tol ||b|| (recurrence residual) */
    int maxit;           /* iteration cap (>= 1) */
    int fixed_iters;     /* > 0: run exactly this many iterations, no tolerance test */
    sb_precond precond;  /* SB_PRECOND_CIRCULANT (Eq. precon), SB_PRECOND_NONE (plain CG) or
                            SB_PRECOND_JACOBI (diag(A)^{-1}, the comparison of the Results; its
                            weights are built on the plan stream by the first Jacobi solve after
                            sb_set_coils / sb_set_mask) */
} sb_pcg_opts;

typedef struct {
    int iters;           /* A applications after the initial residual */
    double rel_resid;    /* final ||r|| / ||b|| */
    int converged;       /* 1 if the tolerance was met (or fixed_iters ran) */
} sb_pcg_result;

/* Solve A x = b for every slice by preconditioned CG (Complexity section; standard PCG with
 * the HPD preconditioner), warm-started from d_x.  d_b, d_x complex64 [nbatch][ny][nx];
 * d_x is overwritten with the solution.  h_results (host, may be NULL) receives nbatch
 * entries.  FP64 CG scalars.  Synchronises.  Returns SB_ERR_NOT_CONVERGED if any slice missed
 * the tolerance within maxit, SB_ERR_BREAKDOWN / SB_ERR_NONFINITE on a CG breakdown. */
sb_status sb_pcg_solve(sb_plan plan, const void* d_b, void* d_x, const sb_pcg_opts* opts,
                       sb_pcg_result* h_results);

typedef struct {
    int n_outer;            /* Algorithm 1 outer iterations (j loop) */
    int n_inner;            /* Algorithm 1 inner iterations (k loop) */
    sb_pcg_opts pcg;        /* the solve of step 5 */
    double tau_tv, tau_w;   /* shrink thresholds; <= 0 selects 1/lambda and 1/gamma */
    int init_rss;           /* 1: x starts as the root-sum-of-squares coil combination of
                               F^H y_i (step 1); 0: d_x holds the caller's start */
    int* h_iters;           /* host, may be NULL: receives nbatch * n_outer * n_inner PCG
                               iteration counts, slice-major */
} sb_sb_opts;

/* Split Bregman reconstruction (Algorithm 1) of every slice from undersampled k-space
 * d_y (complex64 [nbatch][ncoils][ny][nx], DFT order; entries off the mask are ignored),
 * result in d_x (complex64 [nbatch][ny][nx]).  Each inner iteration forms b (step 4), solves
 * A x = b by PCG warm-started from x (step 5), shrinks and updates the Bregman variables
 * (steps 6-11); each outer iteration adds the data residual back (steps 12-14).
 * h_last (host, may be NULL) receives the last solve's result per slice.  Synchronises.
 * d_x must be 16-byte aligned (SB_ERR_INVALID_ARG otherwise; the update kernels move pixel
 * pairs as 16-byte words).  Returns the first non-OK PCG status met (the reconstruction still
 * completes). */
sb_status sb_split_bregman(sb_plan plan, const void* d_y, void* d_x, const sb_sb_opts* opts,
                           sb_pcg_result* h_last);

/* sb_split_bregman on several plans at once: a batch of slices that differ in size, coil count
 * or weights is split by the caller into one plan per geometry, and this call reconstructs all
 * of them concurrently (plan i from its own host thread on its own stream, so plans whose
 * streams differ overlap on the GPU).  For plan i: d_y[i], d_x[i], opts[i] and h_last[i] (may be
 * NULL) mean what they mean for sb_split_bregman.  The same plan may not appear twice
 * (SB_ERR_INVALID_ARG).  Synchronises every plan's stream; returns the first non-OK status in
 * plan order (every plan still runs to completion).  No counterpart in the paper: it batches the
 * independent slice reconstructions of the Methods. */
sb_status sb_split_bregman_many(const sb_plan* plans, int nplans, const void* const* d_y, void* const* d_x,
                                const sb_sb_opts* opts, sb_pcg_result* const* h_last);

/* d_z = F^H diag(d_k)^{-1} F d_r, like sb_apply_precond, but without a plan and without any
 * device allocation, for callers that cannot call cudaMalloc when they apply the
 * preconditioner (fixed memory budgets after start-up, plugins handed only pre-allocated
 * buffers, hosts whose framework owns the memory pool).  The paper has no counterpart; this is
 * a deployment variant of the same operation.
 *   d_r, d_z: complex64 [nbatch][ny][nx] (may be equal); d_k: float32 [nbatch][ny][nx], the
 *   diagonal k, every entry positive and finite, e.g. as returned by sb_get_k (whose entries
 *   are already floored at 1e-12 max k); d_k is divided by as given, so a zero entry gives a
 *   non-finite z there.  cuda_stream: a cudaStream_t (NULL = legacy stream).
 *   nx, ny in {32, 64, 128, 256}, else SB_ERR_UNSUPPORTED; nbatch >= 1 and
 *   nbatch * ny * nx <= 1048576 (the fixed scratch), else SB_ERR_INVALID_ARG.
 * The intermediate lives in one fixed 8 MiB device array that this library defines and every
 * GPU using it keeps until the process exits.  The first call on a device sets that array up
 * (resolves its address, writes the DFT twiddle tables and synchronises the device), so make it
 * before any stream capture.  The set-up is kept per device: the entry point serves the
 * device's primary context (the CUDA runtime's) and is not valid after cudaDeviceReset.  All
 * calls share the array: calls whose kernels overlap on the GPU race with each other and must
 * be ordered by the caller.  Asynchronous after set-up. */
sb_status sb_apply_precond_noalloc(const void* d_r, const float* d_k, void* d_z, int nx, int ny,
                                   int nbatch, void* cuda_stream);

/* Coil compression (Methods, "Coil Compression"): for every slice of a batch, the nv x nc
 * compression matrix A from the principal components of its coil data, then the virtual coil
 * data d_y_out = A d_y and maps d_sens_out = A d_sens (the paper drops the least dominant virtual
 * coils to shorten the reconstruction; the preconditioner's effect is unchanged).
 *   d_y, d_sens:          complex64 [nbatch][nc][npix] on the device (npix = nx ny (nz)).
 *   d_y_out, d_sens_out:  complex64 [nbatch][nv][npix] on the device, distinct from the inputs.
 *   h_matrix (optional):  host complex64 [nbatch][nv][nc], the matrices used (row v = the
 *                         conjugate of the v-th eigenvector of C = sum y y^H, eigenvalues
 *                         descending; a row is defined up to a unit phase).
 *   h_eig (optional):     host double [nbatch][nc], the eigenvalues of C, descending.
 *   1 <= nv <= nc <= 32.  C is summed in FP32 over 128-sample chunks and in FP64 across them;
 * the eigen-decomposition is a cyclic complex Jacobi in FP64 on the host.  Keeps one device
 * scratch block per device, grown on demand and kept until the process exits (calls on one
 * device are serialised on it); synchronises cuda_stream; SB_ERR_INVALID_ARG / SB_ERR_CUDA on
 * failure. */
sb_status sb_coil_compress(const void* d_y, const void* d_sens, size_t npix, int nc, int nbatch, int nv,
                           void* d_y_out, void* d_sens_out, void* h_matrix, double* h_eig, void* cuda_stream);

/* The host step of sb_coil_compress alone (no device work): the compression matrix of one
 * Hermitian covariance.  cov: interleaved complex double [nc][nc] row-major; mat_out:
 * interleaved complex double [nv][nc]; eig_out (may be NULL): double [nc], descending. */
sb_status sb_coil_compression_matrix(const double* cov, int nc, int nv, double* mat_out, double* eig_out);

/* Human-readable name of a status code (static string). */
const char* sb_status_string(sb_status status);

/* Message of the last error raised on this plan ("" if none).  Valid until the next call. */
const char* sb_plan_last_error(sb_plan plan);

/* Number of kernels this library has launched in this process (graph replays count every
 * kernel node they run).  Instrumentation for benchmarks. */
uint64_t sb_kernel_launches(void);

/* Tuning of a plan's launch configuration (results are unchanged up to the summation order of
 * the FP64 partial sums).  col_tile: columns per CTA of the preconditioner's column pass (the
 * length-ny DFTs of M^{-1} = F^H diag(k)^{-1} F, Eq. precon): 8, 16 (default) or 32.  poll_every:
 * PCG iterations between two polls of the slices' convergence state, which is also the length
 * of a captured graph block (default 4, 1..64).  apply_tile: columns per CTA of q = A p (Eq.
 * system) on 2D line-mask plans in FP32 with ny = 256 or 512: 8 (default; p and the coil
 * accumulator in tensor memory) or 16 (both in registers, a two-stage coil-tile ring); other
 * geometries ignore it.  general_passes: how q = A p and the Split Bregman right-hand side run
 * on 2D plans whose mask varies along x (the general path): 1 (default) = one launch per batch
 * each, a thread-block cluster per slice keeping every coil's 2D spectrum in distributed shared
 * memory (nx, ny in {64, 128, 256}; other sizes use three passes), 3 = three passes through a
 * coil scratch in device memory.  A zero field keeps the current value.  The
 * library's autotuner (paper_1710_01758_gb300.autotune) times the choices per geometry and
 * caches the fastest.  SB_ERR_UNSUPPORTED when col_tile does not divide nx or does not fit the
 * column pass (at most 1024 threads, 160 KB of exchange buffers); SB_ERR_INVALID_ARG for other
 * out-of-range values.  Synchronises the plan's stream. */
typedef struct {
    int col_tile;
    int poll_every;
    int apply_tile;
    int general_passes;
} sb_tuning;
sb_status sb_set_tuning(sb_plan plan, const sb_tuning* tuning);
sb_status sb_get_tuning(sb_plan plan, sb_tuning* tuning);

/* CUDA graphs for the PCG loop (default on).  PCG polls the slices' convergence state every
 * few iterations; with graphs enabled, each such block of iterations (q = A p and the
 * preconditioner step, Algorithm 1 step 5 / the Complexity section's PCG) is captured once per
 * execution context (slice group) on the context's stream and replayed while its parameters
 * (the x buffer, tolerance, preconditioner, schedule and block length) repeat.  Capture starts
 * with the context's second block and is skipped while the event timer below is on and on the
 * legacy or per-thread default stream (which cannot be captured).  Results
 * are bitwise identical either way.  enable: 0 = direct launches, 1 = graphs.  Synchronises the
 * plan's stream; SB_ERR_INVALID_ARG for a null plan. */
sb_status sb_set_graphs(sb_plan plan, int enable);

/* Check of the bounded device waits (no counterpart in the paper).  Every wait of a kernel for
 * a TMA tile polls an mbarrier at most a fixed number of times (about half a second by
 * default), then records a timeout in the plan's device error word and lets the kernel finish;
 * sb_pcg_solve and sb_split_bregman read that word at each convergence poll and return
 * SB_ERR_TIMEOUT.  wait_polls: the poll limit (1 .. 4194304; 0 restores the default).
 * withhold_coil_tiles != 0: the coil-tile kernels of the 2D line path in FP32 (q = A p and the
 * Split Bregman right-hand side) request no tile at all, so nothing is in flight and every wait
 * for a tile runs out after wait_polls polls; what the plan computes while it is set is
 * meaningless (switch it off and start the solve again, or destroy the plan).  Clears the error
 * word, drops captured graphs, synchronises the device.  SB_ERR_INVALID_ARG for a null plan or wait_polls above the default. */
sb_status sb_set_wait_check(sb_plan plan, unsigned wait_polls, int withhold_coil_tiles);

/* Kernel classes for the event timer below. */
typedef enum {
    SB_KCLASS_APPLY_A = 0,       /* q = A p (data term by DFTs along y, TV stencil, gamma p) */
    SB_KCLASS_PRECOND_ROW_FWD = 1,  /* r -= alpha q, ||r||^2, DFT along x */
    SB_KCLASS_PRECOND_COL = 2,   /* DFT along y, k^{-1}, inverse DFT along y, r^H z */
    SB_KCLASS_PRECOND_ROW_INV = 3,  /* inverse DFT along x, x and p updates */
    SB_KCLASS_RHS = 4,           /* Split Bregman right-hand side + initial residual */
    SB_KCLASS_SB_UPDATE = 5,     /* shrink, Bregman updates, Haar analysis / synthesis */
    SB_KCLASS_VEC = 6,           /* preconditioner-free CG vector updates */
    SB_KCLASS_OTHER = 7,         /* set-up: k construction, mask analysis, y transform, RSS */
    SB_KCLASS_PRECOND_FUSED = 8, /* whole M^{-1} step in one cluster launch per slice: r, x, p
                                    updates, 2D DFT, k^{-1}, inverse 2D DFT, r^H z */
    SB_KCLASS_COUNT = 9
} sb_kernel_class;

/* Event timer (instrumentation).  With bit c of class_mask set, the plan records a CUDA event
 * pair on its stream around every launch of kernel class c, and accumulates the elapsed times
 * whenever it synchronises.  sb_plan_get_timing synchronises the stream and returns the number
 * of timed launches and their summed duration (ms) since the last sb_plan_set_timing. */
sb_status sb_plan_set_timing(sb_plan plan, unsigned class_mask);
sb_status sb_plan_get_timing(sb_plan plan, int kernel_class, uint64_t* launches, double* total_ms);

#ifdef __cplusplus
}
#endif

#endif /* SB_H */
