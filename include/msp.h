/*
 * msp.h -- C ABI of the GB300 random-sampling multiscale solver.
 *
 * Method: K. Chen, Q. Li, J. Lu, S. J. Wright, "Random sampling and efficient
 * algorithms for multiscale PDEs" (arXiv:1807.08848).  The library runs the
 * data-parallel hot path of Algorithm alg:summary on one GPU:
 *
 *   msp_build_medium    domain decomposition of [0,1]^2 into patches K_m with
 *                       buffered patches K~_m; fine-grid face coefficients
 *                       a(x, x/eps) (Sec. 5, Eq. Elliptic).
 *   msp_sample_patches  offline stage, RanLocalSolu: for every patch and every
 *                       sample, Gaussian data on the ring of K~_m, local solve of
 *                       div(a grad u) = 0 on K~_m, restriction to K_m
 *                       (Sec. 3.3, Sec. 5.2, Eq. elliptic_random).
 *   msp_extract_basis   orthonormal basis of the snapshot range, truncated at
 *                       sigma_i > tau sigma_1 (Sec. 3.2, Eq. svd; the QR remark
 *                       of Sec. 3.3), plus the value/flux edge operators and the
 *                       patch blocks of the least-squares system.
 *   msp_online_solve    online stage: c = argmin |P c - d| (Eq.
 *                       elliptic_cond_reduced) by CGLS preconditioned with a
 *                       block-tridiagonal Cholesky factor of the normal matrix
 *                       over rows of patches (or, on request, the patch blocks
 *                       alone: one-level additive Schwarz), then
 *                       u = sum_m chi_m G_m c_m with a partition of unity.
 *   msp_online_solve_constrained, msp_ras_setup / msp_online_solve_ras
 *                       online variants: the boundary data imposed exactly
 *                       (the remark after Eq. elliptic_cond_reduced), and
 *                       restricted additive Schwarz on the buffered patches
 *                       reduced to the bases (the online step as a standard
 *                       domain-decomposition step, Sec. 3).
 *   msp_kinetic_*       the slab radiative-transfer example of Sec. 4 with
 *                       discrete ordinates (Eq. RTE, Eq. rte_random, Eq.
 *                       rte_cond_reduced).
 *
 * Conventions
 *  - Every call returns an msp_status: MSP_OK (0) or a negative MSP_ERR_* code;
 *    msp_last_error() returns the message of the calling thread's last error.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are stream-ordered; a call returns once its work is enqueued unless
 *    it says it synchronises.
 *  - Pointers named *_dev are device pointers, *_host host pointers.  Caller
 *    buffers are borrowed for the duration of the call only.
 *  - Handles (msp_medium, msp_basis, msp_kmedium, msp_kbasis, msp_server) are
 *    opaque and own device memory allocated by the library (stream-ordered);
 *    free them with the matching *_destroy.
 *  - Fine grid: N cells per side, n = N+1 nodes, h = 1/N, node (i, j) at
 *    (ih, jh), grids row-major with i fastest.  Face coefficients:
 *    aE[j][i] = a((i+1/2)h, jh), (N+1) x N;  aN[j][i] = a(ih, (j+1/2)h),
 *    N x (N+1).  5-point operator
 *      (A u)_ij = sum over faces f of (i,j) of a_f (u_ij - u_nbr(f)).
 *  - Ring of a node box [X0,X1]x[Y0,Y1]: counter-clockwise from (X0,Y0),
 *    every node once (bottom i=X0..X1-1, right j=Y0..Y1-1, top i=X1..X0+1,
 *    left j=Y1..Y0+1).  The global boundary ring has 4N nodes.
 *  - No CPU fallback: without a usable CUDA device every compute call fails
 *    with MSP_ERR_CUDA.
 */
#ifndef MSP_H
#define MSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int msp_status;
#define MSP_OK                 0
#define MSP_ERR_INVALID_ARG   -1   /* bad pointer, size or option; nothing was launched   */
#define MSP_ERR_OOM           -2   /* device allocation failed                             */
#define MSP_ERR_NOT_CONVERGED -3   /* an iteration hit max_iter; results are the last iterate */
#define MSP_ERR_BREAKDOWN     -4   /* a factorisation broke down (non-positive pivot after all shifts, singular coarse matrix) */
#define MSP_ERR_TIMEOUT       -5   /* a bounded wait gave up                               */
#define MSP_ERR_CUDA          -6   /* a CUDA runtime call failed (message has the CUDA text) */
#define MSP_ERR_STATE         -7   /* call out of order (e.g. extract before sample)       */

/* Opaque handles. */
typedef struct msp_medium_s* msp_medium;   /* medium, patches and snapshot storage  */
typedef struct msp_basis_s* msp_basis;     /* reduced bases and online operators    */
typedef struct msp_kmedium_s* msp_kmedium; /* kinetic slab: patches and snapshots   */
typedef struct msp_kbasis_s* msp_kbasis;   /* kinetic reduced bases and online factor */

typedef enum { MSP_FP64 = 0, MSP_MIXED = 1 } msp_precision;

typedef enum {
    MSP_MEDIUM_PERIODIC_SIN = 0,  /* a = 2 + sin(2 pi x/eps) sin(2 pi y/eps)                      */
    MSP_MEDIUM_LOGNORMAL    = 1,  /* a = exp(amp * norm * sum_q [A cos(2 pi k.x) + B sin(2 pi k.x)]) */
    MSP_MEDIUM_CHANNELS     = 2,  /* contrast inside strips of width `width`, 1 elsewhere         */
    MSP_MEDIUM_HOU_WU       = 3,  /* the two-scale medium of the elliptic test, Sec. 5.3          */
    MSP_MEDIUM_USER         = 4   /* explicit face coefficients                                   */
} msp_medium_kind;

/* Coefficient field description.  Host pointers; the library copies them. */
typedef struct {
    int kind;                 /* msp_medium_kind                                  */
    int n_cells;              /* N >= 2                                           */
    double eps;               /* oscillation scale (PERIODIC_SIN, HOU_WU)         */
    int n_modes;              /* LOGNORMAL: number of rows of `modes`             */
    const double* modes_host; /* LOGNORMAL: [n_modes][4] = kx, ky, A, B           */
    double amp, norm;         /* LOGNORMAL: exponent scale and per-mode factor    */
    int n_channels;           /* CHANNELS: number of rows of `channels`           */
    const double* channels_host; /* CHANNELS: [n][3] = px, py, theta (line through (px,py) at angle theta) */
    double width, contrast;   /* CHANNELS                                         */
    const double* user_aE_host; /* USER: (N+1) x N                               */
    const double* user_aN_host; /* USER: N x (N+1)                               */
} msp_medium_desc;

/* Tensor partition into patches, patch m = p + q * nx_patches (p fastest).
 * Patch (p,q) covers cells [x_breaks[p], x_breaks[p+1]] x [y_breaks[q], y_breaks[q+1]];
 * its buffered patch extends it by buffers[m] cells on every side, clipped to
 * the domain.  Every patch draws samples[m] Gaussian samples; patches whose
 * buffered ring touches the domain boundary also solve one delta datum per
 * ring node on the domain boundary (the full basis there, as the boundary
 * patches of Sec. 4.2 do), so patch m has cols_m = samples[m] + n_b(m)
 * snapshot columns. */
typedef struct {
    int nx_patches, ny_patches;
    const int* x_breaks_host;   /* nx_patches+1, increasing, 0 .. N */
    const int* y_breaks_host;   /* ny_patches+1, increasing, 0 .. N */
    const int* buffers_host;    /* per patch, >= 0                  */
    const int* samples_host;    /* per patch, >= 1                  */
} msp_patch_desc;

/* Geometry of one patch (closed node boxes). */
typedef struct {
    int x0, x1, y0, y1;   /* K_m                          */
    int X0, X1, Y0, Y1;   /* K~_m (buffered, clipped)     */
    int n_k;              /* (x1-x0+1)(y1-y0+1) nodes of K_m */
    int n_ring;           /* ring nodes of K~_m           */
    int samples;          /* Gaussian columns             */
    int n_b;              /* delta columns (ring nodes on the domain boundary) */
    int cols;             /* samples + n_b                */
    int64_t snap_offset;  /* first element of this patch's snapshot block */
} msp_patch_info;

/* Iteration statistics of a batch of local solves. */
typedef struct {
    int64_t n_solves;
    int64_t total_iters;      /* sum over solves of inner (PCG) iterations   */
    int max_iters;            /* largest inner iteration count of one solve  */
    int max_refinements;      /* largest number of FP64 refinement steps     */
    int n_not_converged;      /* solves that stopped at max_iter              */
    int64_t unknown_iters;    /* sum over solves of (CG iterations x interior unknowns) */
} msp_solve_stats;

/* Last error message of the calling thread ("" if none). */
const char* msp_last_error(void);

/* Library version string. */
const char* msp_version(void);

/* Number of CUDA kernels the library has launched in this process so far
 * (all threads, all devices); for launch accounting in benchmarks. */
int64_t msp_kernel_launches(void);

/* Bound on the polls of a device-side grid barrier (the cooperative sweeps of the
 * online factor): a CTA that has polled the barrier this many times without the
 * rest of the grid arriving gives up, raises the barrier's error word and every
 * CTA of the launch returns at its next barrier; the call that launched it then
 * returns MSP_ERR_TIMEOUT and the context stays usable.  Process-wide, read at
 * every launch.  polls = 0 restores the default (2^24 polls, tens of seconds);
 * INVALID_ARG if polls < 0.  Small values are for tests of the timeout path. */
msp_status msp_set_wait_limit(int64_t polls);

/* Engine of the FP64 matrix products inside msp_extract_basis (the Gram and
 * triangular products of Cholesky-QR, the projection onto the singular vectors)
 * and of the large products of the online factorisation:
 *   MSP_GEMM_TENSOR_CORES (default): FP64-accurate products on the tensor cores --
 *     each FP64 row / column cut by truncation into 8 BF16 slices of 7 bits under
 *     a power-of-two scale (error-free splitting, Ozaki et al. 2012), the slice
 *     products with t + u <= 9 accumulated exactly by tcgen05 kind::f16 MMAs in
 *     K chunks of 128 and in int32 registers across the chunks, the sum formed in
 *     FP64; the error of a product is of the order of 2^-56 |a_i|_inf |b_j|_inf per
 *     term, below the rounding of an FP64 product;
 *   MSP_GEMM_CUDA_CORES: the FP64 FMA kernels.
 * Process-wide, read by every extraction; products with K > 16256 use the CUDA
 * cores.  INVALID_ARG on an unknown engine. */
#define MSP_GEMM_TENSOR_CORES 0
#define MSP_GEMM_CUDA_CORES   1
msp_status msp_set_gemm_engine(int engine);

/* The SVD of the triangular Cholesky-QR factor T in the extraction (Sec. 3.2,
 * Eq. svd), one-sided Jacobi on the columns of T^T either way:
 *   MSP_SVD_FP64: FP64 sweeps from V = I;
 *   MSP_SVD_FP32_PRECONDITIONED: sweeps in FP32 first (V32 orthogonal to about
 *     1e-6), V re-orthogonalised in FP64 by two Newton-Schulz steps
 *     V (3 I - V^T V) / 2, then FP64 sweeps on T^T V to the FP64 convergence
 *     level.  The FP32 sweeps resolve only the directions of singular values
 *     above about 1e-7 sigma_1, and the snapshot blocks of the elliptic
 *     workloads keep most of their columns below that, so the FP64 sweeps still
 *     need nearly as many sweeps (measured at 2049^2: 283 ms of FP64 sweeps after
 *     71 ms of FP32 start, against 371 ms from V = I);
 *   MSP_SVD_QR_PRECONDITIONED (default): Householder QR with column pivoting
 *     T P = Q R in FP64 first (Drmac and Veselic 2008), then FP64 sweeps on the
 *     columns of R^T with V started at Q: the rows of R decay with the pivots,
 *     so the sweeps start from graded, nearly orthogonal columns (measured at
 *     2049^2: 37 ms of QR and 228 ms of sweeps, at most 10 and 6.3 on average,
 *     against 370 ms and 20 / 8.1 sweeps from V = I).
 * Both end at the same FP64 stopping test; process-wide, read by every
 * extraction.  INVALID_ARG on an unknown mode. */
#define MSP_SVD_FP64                0
#define MSP_SVD_FP32_PRECONDITIONED 1
#define MSP_SVD_QR_PRECONDITIONED   2
msp_status msp_set_svd_mode(int mode);

/* --------------------------------------------------------------------- medium */

/* Build the patch tables and evaluate the face coefficients on the device
 * (Sec. 5: a(x, x/eps) on the fine mesh).  Allocates the snapshot storage
 * (sum over patches of n_k * cols_m doubles).  INVALID_ARG on malformed
 * descriptions (breaks not covering [0,N], non-positive sizes, NULL tables). */
msp_status msp_build_medium(const msp_medium_desc* medium, const msp_patch_desc* patches,
                            void* stream, msp_medium* out);
/* The full-basis medium of DetLocalSolu (Algorithm alg:summary, Sec. 3.3): as
 * msp_build_medium, but every patch m has one delta column per ring node of its
 * buffered patch and no Gaussian columns (samples_host is ignored and may be
 * NULL): samples = 0, n_b = cols = n_ring, column t the unit datum at ring
 * position t.  msp_sample_patches then computes the restricted Green's matrix
 * G~_m (n_k x n_ring) of the buffered patch -- of K_m itself with buffer 0 --
 * and msp_extract_basis its singular values and basis as for sampled media. */
msp_status msp_build_medium_full(const msp_medium_desc* medium, const msp_patch_desc* patches,
                                 void* stream, msp_medium* out);
void msp_medium_destroy(msp_medium m);

/* Counts: patches, total snapshot elements, N. */
msp_status msp_medium_counts(msp_medium m, int* n_patches, int64_t* snapshot_elems, int* n_cells);
msp_status msp_medium_patch(msp_medium m, int patch, msp_patch_info* out);

/* Copy the FP64 face coefficients to device buffers of (N+1)*N (aE) and
 * N*(N+1) (aN) doubles. */
msp_status msp_get_coefficients(msp_medium m, double* aE_dev, double* aN_dev, void* stream);

/* --------------------------------------------------------------------- offline */

/* RanLocalSolu on every patch (Algorithm alg:summary; Eq. elliptic_random):
 * for each patch m and column s < cols_m, ring data of K~_m -- i.i.d. N(0,1)
 * from Philox4x32-10 (key = seed, counter = (node pair, s, m, tag)) with
 * Box-Muller for s < samples[m], a unit delta at the (s - samples[m])-th ring
 * node on the domain boundary otherwise -- then the local solve on K~_m by
 * Jacobi-preconditioned CG and the restriction to K_m, stored as the patch's
 * snapshot block (n_k x cols_m, column-major).
 *   precision MSP_FP64: CG in FP64 to |r| <= tol |b|.
 *   precision MSP_MIXED: CG in FP32 inside FP64 iterative refinement (FP64
 *     residual r = b - A x, FP32 correction), to |r| <= tol |b|.
 * max_iter bounds the CG iterations of each inner solve.  If stats_host is
 * not NULL the call synchronises the stream and fills it; it then returns
 * MSP_ERR_NOT_CONVERGED if any solve stopped at max_iter. */
msp_status msp_sample_patches(msp_medium m, uint64_t seed, int precision, double tol, int max_iter,
                              void* stream, msp_solve_stats* stats_host);

/* Copy patch `patch`'s snapshot block (n_k x cols, column-major) to dst_dev. */
msp_status msp_get_snapshots(msp_medium m, int patch, double* dst_dev, void* stream);

/* The local solves of the listed patches only (the offline loop of Algorithm
 * alg:summary restricted to a set of patches: a share of the patches when the
 * offline stage is split across GPUs).  Every column of each listed patch is
 * solved as msp_sample_patches solves it (same random data, same launch: the
 * split or fused CG launch of the medium's setting; a medium set to the direct
 * solver uses the split launch here); the other patches' snapshot blocks are
 * left as they are.  Synchronises; stats_host (optional) covers the listed
 * patches; NOT_CONVERGED as for msp_sample_patches; INVALID_ARG on an index
 * outside the medium. */
msp_status msp_sample_patch_list(msp_medium m, const int* patches_host, int n_patches, uint64_t seed, int precision,
                                 double tol, int max_iter, void* stream, msp_solve_stats* stats_host);
/* Write patch `patch`'s snapshot block (n_k x cols, column-major) from src_dev,
 * e.g. a block another GPU computed; the medium then counts as sampled. */
msp_status msp_set_snapshots(msp_medium m, int patch, const double* src_dev, void* stream);

/* Ring data of patch `patch` as the sampler draws it, (n_ring x cols)
 * column-major, to dst_dev (for checking the generator). */
msp_status msp_get_samples(msp_medium m, int patch, uint64_t seed, double* dst_dev, void* stream);

/* Local solves of ONE patch without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device
 * memory while it runs -- code working inside a memory pool it does not own, a
 * framework that forbids allocation on its hot path, or a process whose
 * allocator is already at its limit.  The caller passes every input and output:
 *   aE_dev, aN_dev  face coefficients of the medium ((N+1) x N and N x (N+1),
 *                   e.g. from msp_get_coefficients);
 *   boxes_host      x0, x1, y0, y1 of K_m then X0, X1, Y0, Y1 of the buffered
 *                   box (closed node boxes, 0 <= X0 <= x0 < x1 <= X1 <= N);
 *   patch_index     the patch's index m in the Philox counter (same samples as
 *                   msp_sample_patches draws for patch m);
 *   samples         Gaussian columns, 1..4096 (no boundary-delta columns);
 *   snap_dev        output, n_k x samples doubles, column-major;
 *   n_not_converged_host  optional: if not NULL the call synchronises the
 *                   stream, stores the number of columns whose solve stopped at
 *                   max_iter and returns MSP_ERR_NOT_CONVERGED if it is not 0
 *                   (read back from the static array's statistics through a
 *                   stack buffer); if NULL that count is not reported and the
 *                   call returns once the launch is enqueued.
 * Its scratch lives in one file-scope device array of 32 MiB that every GPU
 * loading the library holds until the process exits; a buffered patch whose
 * interior exceeds the on-chip tile (98 columns, 12 rows per thread segment)
 * or whose per-block scratch does not fit is rejected with INVALID_ARG.  The
 * first call on a device looks up the array's device address (with that device
 * current); make that first call before any stream capture.  Every call shares
 * the array and leaves its contents behind: calls that overlap on the GPU
 * (concurrent streams, several threads) race and must be serialised by the
 * caller.  No cudaMalloc, cudaFree or allocating library routine is called. */
msp_status msp_sample_patch_static(const double* aE_dev, const double* aN_dev, int n_cells, const int* boxes_host,
                                   int patch_index, int samples, uint64_t seed, int precision, double tol,
                                   int max_iter, double* snap_dev, void* stream, int* n_not_converged_host);

/* Orthonormal basis of every patch's snapshot range (Sec. 3.2, Eq. svd):
 * shifted Cholesky-QR3 of the snapshot block, SVD of its triangular factor by
 * one-sided Jacobi, truncation k_m = #{sigma_i > tau sigma_1}; basis
 * Q_m = left singular vectors 1..k_m (n_k x k_m).  Then the edge operators
 * (value and flux rows on the ring of K_m, Eq. elliptic_cond_tilde), the row
 * tables of P~ and the Cholesky factors of the patch blocks of P~^T P~.
 * Synchronises the stream (the k_m decide the online layout).
 * BREAKDOWN if a Cholesky factorisation fails after its shift retries. */
msp_status msp_extract_basis(msp_medium m, double tau, int precision, void* stream, msp_basis* out);
void msp_basis_destroy(msp_basis b);

/* Number of kept vectors k_m and (if sigma_host != NULL, length cols_m) all
 * singular values of patch `patch`'s snapshot block, descending. */
msp_status msp_basis_info(msp_basis b, int patch, int* k, double* sigma_host);
/* Copy Q_m (n_k x k_m, column-major) to dst_dev. */
msp_status msp_get_basis(msp_basis b, int patch, double* dst_dev, void* stream);
/* Diagnostics of the extraction. */
typedef struct {
    int max_jacobi_sweeps;     /* largest sweep count of the one-sided Jacobi SVDs          */
    int max_cholqr_tries;      /* largest number of shift attempts in Cholesky-QR           */
    float online_shift;        /* diagonal shift the online factorisation needed (0 = none) */
    int online_blocks;         /* rows of patches = diagonal blocks of the online factor    */
    int online_factor_bits;    /* 32 or 64: precision the online factor was built in; 0 if the
                                  patch-block preconditioner is in use                         */
    float mean_jacobi_sweeps;  /* mean sweep count of the one-sided Jacobi SVDs over patches   */
    int online_apply_bits;     /* 32 or 64: precision the factor sweeps run in; 0 if it depends
                                  on the batch size (FP64 below 4 data sets) or as above       */
} msp_basis_stats;
msp_status msp_basis_get_stats(msp_basis b, msp_basis_stats* out);

/* Phase timing of msp_extract_basis (CUDA events on the caller's stream at the
 * phase boundaries; off by default, process-wide switch): after an extraction made
 * with timing on, msp_basis_extract_timing waits for its events and returns the
 * milliseconds of ms_host[6] = Cholesky-QR, the start of the Jacobi SVD (FP32
 * sweeps, re-orthogonalisation and T^T V in MSP_SVD_FP32_PRECONDITIONED mode, the
 * copy T^T otherwise), the FP64 Jacobi sweeps, truncation and projection, online
 * operators, online factorisation (zeros if the basis was extracted with timing
 * off or loaded from a file), and optionally the algorithmic FP64 work of the
 * FP64 Jacobi sweeps (22 c flop per column pair and sweep, summed over the
 * patches). */
msp_status msp_set_extract_timing(int enable);
msp_status msp_basis_extract_timing(msp_basis b, double* ms_host, double* jacobi_flop_host);

/* Preconditioner of the online least-squares iteration (the iteration itself,
 * its residuals and iterates are FP64 in every case):
 *   MSP_PRECOND_BLOCK_ROWS (default): block-tridiagonal Cholesky of the scaled
 *     normal matrix over rows of patches.  Factorised in FP32 when that succeeds,
 *     else in FP64.  An FP64 factor is applied in FP64 for batches of fewer than
 *     4 data sets and through an FP32 rounded copy for larger batches (a few more
 *     iterations, each sweep at the FP32 rate);
 *   MSP_PRECOND_PATCH_BLOCKS: the inverse patch blocks (P~^T P~)_mm^{-1} only
 *     (one-level additive Schwarz);
 *   MSP_PRECOND_BLOCK_ROWS_FP64: as BLOCK_ROWS, an FP64 factor always applied in FP64;
 *   MSP_PRECOND_BLOCK_ROWS_FP32: as BLOCK_ROWS, an FP64 factor always applied
 *     through its FP32 copy. */
#define MSP_PRECOND_BLOCK_ROWS      0
#define MSP_PRECOND_PATCH_BLOCKS    1
#define MSP_PRECOND_BLOCK_ROWS_FP64 2
#define MSP_PRECOND_BLOCK_ROWS_FP32 3
msp_status msp_basis_set_preconditioner(msp_basis b, int kind);

/* Total unknowns N_p = sum k_m and rows of P~. */
msp_status msp_online_counts(msp_basis b, int* n_unknowns, int* n_rows);

/* Matrix-free 5-point operator of the local problems (Sec. 5; the finite-
 * difference reading: (A u)_ij = sum over the faces f of node (i, j) of
 * a_f (u_ij - u_nbr(f))) applied to a stack of tiles: for every patch m and sample
 * s < samples, y = A x on the interior nodes of the buffered box K~_m, with the
 * ring values taken from x; y = 0 on the ring and in the padding.
 *   x_dev, y_dev: [patch][sample][rows][pitch] device arrays of float
 *     (precision MSP_MIXED) or double (MSP_FP64); node (i, j) of patch m at row
 *     j - Y0, column i - X0; x_dev 16-byte aligned;
 *   pitch: multiple of 4, >= the widest buffered box; rows >= the tallest
 *     (msp_operator_tile_shape gives both maxima);
 *   ms_out: optional device time of the launch (CUDA events), synchronising.
 * This is the streaming form of the operator (each tile read and written once);
 * the local solves use a tile-resident form inside their kernels.  INVALID_ARG
 * on a bad shape, TIMEOUT if a tile copy does not complete. */
msp_status msp_operator_tile_shape(msp_medium m, int* rows, int* cols);
msp_status msp_apply_operator(msp_medium m, int samples, int precision, const void* x_dev, void* y_dev, int pitch,
                              int rows, double* ms_out, void* stream);

/* Launch of the local solves of msp_sample_patches, per precision.
 *   MSP_LAUNCH_SPLIT (default): the tile-resident kernel for the buffered patches
 *     whose tile fits on chip, then the global-scratch kernel for the rest;
 *   MSP_LAUNCH_FUSED: one persistent launch for every (patch, column): the CTAs
 *     take the large tiles first (global-scratch path), then the on-chip tiles.
 *   MSP_LAUNCH_DIRECT (precision MSP_MIXED only; buffered patches of at most 160
 *     interior nodes per row): the direct local solver -- per patch, a block LDL^T
 *     factorisation of the Jacobi-scaled operator over the grid rows with FP32
 *     inverses W_j of the Schur complements (computed once per medium, on the
 *     first call), applied to chunks of 32 columns by a forward and a backward
 *     sweep of dense W_j products, inside FP64 iterative refinement (FP64
 *     residual, FP32 correction) until |r| <= tol |b| per column, at most 8
 *     passes; the statistics count passes as iterations.  Device memory: the
 *     inverses (ny ld^2 floats per patch, ld = interior row length rounded up to
 *     4) and the FP64 iterate, the residual and the forward sweep's blocks of
 *     every column (about 25 GB at 2049^2 with 32 x 32 patches).
 *   rows: rows per thread segment of the tile kernel, 4, 8 or 12 (0: the smallest
 *     that every eligible tile fits); INVALID_ARG if below that.
 * Results do not depend on the launch beyond the solver tolerance: the split and
 * fused launches run each column's arithmetic identically; the direct solver
 * reaches the same tolerance by another route. */
#define MSP_LAUNCH_SPLIT 0
#define MSP_LAUNCH_FUSED 1
#define MSP_LAUNCH_DIRECT 2
msp_status msp_medium_set_launch(msp_medium m, int precision, int mode, int rows);

/* Phase timing of the direct solver (CUDA events on the caller's stream around
 * each of its launches; off by default).  After a msp_sample_patches call with the
 * direct launch and timing on, msp_medium_direct_timing waits for the events and
 * returns, per phase -- 0 factorisation (first call only), 1 iterate set-up,
 * 2 FP64 residuals, 3 sweeps (the dense W_j products), 4 restriction -- the summed
 * milliseconds (ms_host[5]) and launch counts (launches_host[5], optional). */
msp_status msp_medium_set_timing(msp_medium m, int enable);
msp_status msp_medium_direct_timing(msp_medium m, double* ms_host, int* launches_host);

/* Autotuner of that launch: every CG candidate (split or fused, each rows instance
 * the eligible tiles fit) runs an even-strided subset of at most max_probe_items
 * of the medium's columns, once to warm up and once timed (CUDA events).  With
 * precision MSP_MIXED and a medium the direct solver fits, MSP_LAUNCH_DIRECT is a
 * candidate too (rows 0): it runs the whole medium once untimed (factorising every
 * patch; the factor is kept) and once timed, and its ms is that time scaled to the
 * probe's share of the columns.  The fastest is kept for msp_sample_patches of that
 * precision and reported.  The CG probes write the subset's snapshot columns with
 * the values a full run writes; the direct candidate writes every column (its own
 * values, replaced by the next msp_sample_patches).  Synchronises. */
#define MSP_TUNE_MAX_CANDIDATES 8
typedef struct {
    int mode, rows;    /* mode: MSP_LAUNCH_SPLIT, MSP_LAUNCH_FUSED or MSP_LAUNCH_DIRECT */
    float ms;          /* device time of the probe; -1 if the configuration does not fit */
} msp_tune_candidate;
typedef struct {
    int probe_items, n_candidates;
    msp_tune_candidate candidates[MSP_TUNE_MAX_CANDIDATES];
    int best_mode, best_rows;
    float best_ms;
} msp_tune_report;
msp_status msp_medium_autotune(msp_medium m, int precision, uint64_t seed, double tol, int max_iter,
                               int max_probe_items, void* stream, msp_tune_report* out);

/* enable != 0: msp_sample_patches replays its launches from a CUDA graph, captured
 * on the first call of each configuration (precision, seed, tolerances, launch);
 * the stream must not be capturing when that first call is made. */
msp_status msp_medium_set_graph(msp_medium m, int enable);

/* --------------------------------------------------------------------- online */

/* Online stage for `batch` Dirichlet data sets (Eq. elliptic_cond_reduced):
 *   phi_dev: [batch][4N] values on the global boundary ring;
 *   u_dev:   [batch][N+1][N+1] reconstructed fields (output);
 *   c_dev:   optional [batch][N_p] coefficients (output) or NULL.
 * CGLS on the normal equations, preconditioned as msp_basis_set_preconditioner
 * selects (default: the block-tridiagonal Cholesky factor of the scaled normal
 * matrix over rows of patches), stopped per data set at
 * |P~^T r| <= tol |P~^T d| or max_iter; every data set's iteration is
 * independent of the others in the batch (fixed-order reductions).
 * The stop test is read on the host every 2 iterations (every 16 with the
 * patch-block preconditioner), so the call synchronises the stream while it
 * iterates; the reconstruction after the last test is enqueued without a
 * further synchronisation unless iters_host is given.  iters_host (optional,
 * [batch]) receives the iteration counts; NOT_CONVERGED if any data set hit
 * max_iter or its residual became NaN or Inf (non-finite phi: that data set
 * stops at once, the others finish); TIMEOUT if the factor sweeps' grid barrier gave up (see
 * msp_set_wait_limit).  u_dev may be NULL when c_dev is given (coefficients
 * only, no reconstruction). */
msp_status msp_online_solve(msp_basis b, const double* phi_dev, int batch, double tol, int max_iter,
                            double* u_dev, double* c_dev, int* iters_host, void* stream);

/* The constrained least-squares variant of the online stage (the remark after
 * Eq. elliptic_cond_reduced): the boundary rows u_m(x) = phi(x) on the domain
 * boundary hold exactly, the continuity rows are solved in the least-squares
 * sense.  The boundary rows of a patch involve only its own coefficients, so
 * they are eliminated patch by patch (null-space method: pivoted Householder QR
 * of B_m^T, c_m = Z_m phi_m + N_m z_m with the minimum-norm particular part) and
 * the reduced unknowns z go through the same preconditioned FP64 CGLS on a
 * derived basis (bases Q_m N_m, continuity rows only), built on the first call
 * and kept with the basis (synchronises; its factorisation costs about as much
 * as the extraction's).  Arguments, layouts, stopping rule and return codes as
 * msp_online_solve; c_dev receives the full coefficients c.  BREAKDOWN when a
 * boundary patch keeps fewer basis vectors than it has domain-boundary nodes, or
 * their boundary rows are not independent to working accuracy (|R_jj| <= 1e-12
 * |R_00| in the pivoted QR): the data cannot be imposed exactly there. */
msp_status msp_online_solve_constrained(msp_basis b, const double* phi_dev, int batch, double tol, int max_iter,
                                        double* u_dev, double* c_dev, int* iters_host, void* stream);

/* The overlapping Schwarz variant of the online stage.  The paper leaves the
 * online step to a standard domain-decomposition step (Sec. 3, before Algorithm
 * alg:summary); this one is restricted additive Schwarz on the buffered patches
 * K~_m (Cai and Sarkis 1999), reduced to the bases: each step sets
 *     c_m <- B_m g_m(c),   B_m = Q_m^T G~_m  (k_m x n_ring_m),
 * with G~_m the restricted Green's matrix of DetLocalSolu (Algorithm alg:summary)
 * and g_m(c) the values on the ring of K~_m of the reconstruction
 * u = sum_n chi_n Q_n c_n (chi_n = 1/#patches holding the node), phi on the
 * domain boundary.  Its fixed point solves (I - T) c = F phi.
 *
 * msp_ras_setup(b, full, coarse, stream): `full` is a medium built by
 * msp_build_medium_full on the same medium description and partition as the
 * basis's medium and sampled by msp_sample_patches (its snapshot blocks are the
 * G~_m); it is only read and may be destroyed afterwards.  Computes every B_m
 * (FP64 products on the engine msp_set_gemm_engine selects), gathers the ring
 * rows chi_n Q_n[node, :], and with coarse != 0 the two-level coarse space of
 * Nicolaides (one vector z_m = Q_m^T 1 / |Q_m^T 1| per patch) with the coarse
 * matrix E = Z^T (I - T) Z (M x M, FP64) inverted by Gauss-Jordan elimination with
 * partial pivoting on the device.  Owns about (sum_m k_m n_ring_m + sum of ring
 * entries x k) doubles plus 2 M^2 for the coarse space until the basis is
 * destroyed; a second call replaces the first.  Synchronises.  INVALID_ARG when
 * `full` is not a sampled full-basis medium of the basis's grid and partition;
 * BREAKDOWN when E is singular to working precision (call again with coarse = 0).
 *
 * msp_online_solve_ras: restarted GMRES (restart 30) on (I - T) c = F phi, right-
 * preconditioned by the coarse space in the A-DEF2 form M^{-1} = I + Z E^{-1} Z^T T
 * (Tang, Nabben, Vuik, Erlangga 2009) when it was built, stopped per data set at
 * |F phi - (I - T) c| <= tol |F phi| or max_iter GMRES iterations; FP64
 * throughout; data sets in passes of 16, each data set's arithmetic independent of
 * the others (fixed-order reductions).  Arguments and layouts as msp_online_solve
 * (phi_dev [batch][4N], u_dev [batch][N+1][N+1] or NULL, c_dev [batch][N_p] or
 * NULL, iters_host [batch] or NULL: GMRES iterations).  The call reads the stop
 * test on the host after every iteration, so it synchronises the stream while it
 * iterates.  NOT_CONVERGED if a data set hit max_iter or its residual is not
 * finite; INVALID_ARG before msp_ras_setup. */
msp_status msp_ras_setup(msp_basis b, msp_medium full, int coarse, void* stream);
msp_status msp_online_solve_ras(msp_basis b, const double* phi_dev, int batch, double tol, int max_iter,
                                double* u_dev, double* c_dev, int* iters_host, void* stream);

/* Boundary-to-coefficient map.  The data of Eq. elliptic_cond_reduced enter only
 * through the boundary rows, linearly, so c = G phi with G = P~^+ S (N_p x 4N; S
 * places the ring values phi into the boundary rows).  msp_basis_build_map
 * computes G column by column (online solves of the 4N unit ring vectors, to
 * tolerance tol, in batches) and keeps it on the device in FP32 together with an
 * FP32 copy of the bases; it synchronises and owns the memory until the basis
 * is destroyed.  NOT_CONVERGED if a column stopped at max_iter.
 * msp_online_solve_map then gives u for `batch` data sets phi_dev [batch][4N]
 * (FP64) as u_dev [batch][N+1][N+1] (FP64): one FP32 GEMM c = G phi, the FP32
 * reconstruction inside the patches and the FP64 skeleton average; stream
 * ordered, and each data set's result does not depend on the rest of the batch.
 * INVALID_ARG if the map has not been built.  The paper has no counterpart of
 * the map; it is the serving form of the same least-squares solution. */
msp_status msp_basis_build_map(msp_basis b, double tol, int max_iter, void* stream);
/* Engine of the map GEMM c = G phi: MSP_MAP_TENSOR_CORES (default) uses the fifth-
 * generation tensor cores (tcgen05, TF32 inputs with the three-term split G_hi phi_hi
 * + G_hi phi_lo + G_lo phi_hi, FP32 accumulation per 128 terms, FP64 across them);
 * MSP_MAP_CUDA_CORES the FP32 FMA kernel with the same accumulation scheme. */
#define MSP_MAP_TENSOR_CORES 0
#define MSP_MAP_CUDA_CORES   1
msp_status msp_basis_set_map_engine(msp_basis b, int engine);
msp_status msp_online_solve_map(msp_basis b, const double* phi_dev, int batch, double* u_dev, void* stream);

/* Persistence: msp_save_basis writes the geometry, the bases Q_m, their singular
 * values and the medium's face coefficients to a file (host I/O, synchronises);
 * msp_load_basis reads such a file on the current device and rebuilds the online
 * operators with the extraction's own code, so the loaded basis gives the same online
 * results.  The map of msp_basis_build_map is not saved.  INVALID_ARG on an unreadable,
 * foreign or truncated file (checked before any device work). */
msp_status msp_save_basis(msp_basis b, const char* path);
/* Geometry of a basis (also of a loaded one): the number of cells and patches, and
 * patch `patch`'s boxes as msp_medium_patch gives them (out may be NULL). */
msp_status msp_basis_patch(msp_basis b, int patch, int* n_cells, int* n_patches, msp_patch_info* out);
msp_status msp_load_basis(const char* path, msp_basis* out);

/* The online system of Eq. elliptic_cond_reduced for inspection of small cases:
 * P~ (rows x N_p, see msp_online_counts) as COO triplets and d for the ring data
 * phi_host ([4N], host).  *nnz receives the entry count; with rows = NULL only the
 * count (and d if d_host is given) is returned; otherwise rows, cols, vals (host,
 * capacity entries) receive the entries.  Synchronises. */
msp_status msp_get_online_system(msp_basis b, const double* phi_host, int64_t capacity, int64_t* nnz, int* rows,
                                 int* cols, double* vals, double* d_host);

/* -------------------------------------------------------------------- serving */

/* A request loop over several prebuilt media (bases with their maps built):
 * requests (a medium and its boundary data phi, host FP64 [4N]) are queued on
 * submit; worker threads, each on its own CUDA stream, admit queued requests
 * into batches of one medium, oldest request first, as long as the slot count
 * (requests admitted and not yet released) stays within max_slots and the
 * device memory they hold (phi and u of each request) within mem_budget_bytes;
 * each batch is one msp_online_solve_map call.  Batches of different workers run
 * on the device at the same time, and a request that arrives while others are on
 * the device is admitted as soon as slots and memory allow.  A result stays on
 * the device until it is fetched or released.  Latency = submit to the host
 * seeing the batch complete.  n_workers = 0: no threads; msp_server_step runs
 * one admit + solve + retire cycle on the caller's stream.
 * The server borrows the bases: they must outlive it.  With the map engine
 * (the default, msp_server_set_engine) every medium needs its map
 * (msp_basis_build_map); a batch of a medium without one fails with STATE. */
typedef struct msp_server_s* msp_server;
typedef struct {
    long long submitted, completed, released, failed, batches;
    int queued, in_flight, held, max_batch_seen;
    long long mem_in_use, mem_peak;
} msp_server_stats;
msp_status msp_server_create(const msp_basis* media, int n_media, long long mem_budget_bytes, int max_slots,
                             int max_batch, int n_workers, msp_server* out);
/* Non-blocking: copies phi_host (4N values of the medium's ring). INVALID_ARG on a
 * bad medium index; OOM if one request alone exceeds the memory budget. */
msp_status msp_server_submit(msp_server s, int medium, const double* phi_host, uint64_t* req_id);
/* Never blocks: done = 1 when the result is on the device (latency_ms optional),
 * done = -1 if its batch failed (the status is returned). */
msp_status msp_server_poll(msp_server s, uint64_t req_id, int* done, double* latency_ms);
/* Copies a finished result to u_host ([N+1][N+1], host) and releases it. */
msp_status msp_server_fetch(msp_server s, uint64_t req_id, double* u_host);
/* Releases a finished result without copying it. */
msp_status msp_server_release(msp_server s, uint64_t req_id);
/* Manual mode (n_workers = 0): one admit + solve + retire cycle; *n_done (optional)
 * receives the number of requests it completed. */
msp_status msp_server_step(msp_server s, void* stream, int* n_done);
msp_status msp_server_get_stats(msp_server s, msp_server_stats* out);
/* Engine of the batch solves, read when a batch is admitted (so it may change
 * between requests):
 *   MSP_SERVE_MAP (default): one msp_online_solve_map per batch (the FP32 map
 *     on the tensor cores, FP64 skeleton); INVALID_ARG unless every medium has
 *     its map;
 *   MSP_SERVE_ITERATIVE_FP64: the plain FP64 path, the CGLS iteration of
 *     msp_online_solve to |P~^T r| <= tol |P~^T d| (at most max_iter
 *     iterations) with an FP64 block-row factor applied in FP64 (the
 *     preconditioner only sets the pace: residuals and iterates are FP64 with
 *     either factor precision).  That iteration
 *     works in the basis's own buffers, so the batches of one medium run one at
 *     a time (a lock per medium) and the caller must not run msp_online_solve on
 *     a served basis meanwhile; a batch whose data sets stop at max_iter fails
 *     with NOT_CONVERGED.
 * tol and max_iter are ignored by the map engine. */
#define MSP_SERVE_MAP            0
#define MSP_SERVE_ITERATIVE_FP64 1
msp_status msp_server_set_engine(msp_server s, int engine, double tol, int max_iter);
void msp_server_destroy(msp_server s);

/* --------------------------------------------------------------------- kinetic */

/* Slab radiative transfer with isotropic scattering (Sec. 4; Eq. RTE with the
 * Henyey-Greenstein kernel of Eq. HG at g = 0):
 *     v d_x f = (1/eps)(rho - f),  rho = (1/2) sum_l w_l f_l,  x in [0, 1],
 * on nodes x_i = i/N with n_v Gauss-Legendre velocities (ascending) and implicit
 * upwind differences; incoming data f(0, v>0) and f(1, v<0).  n_patches equal
 * patches K_m = [m W, (m+1) W] cells (W = N/n_patches), buffered by `buffer`
 * cells (clipped); `samples` random incoming data sets per patch.  Snapshot
 * rows are node-major with the velocity fastest ((W+1) n_v rows).
 * INVALID_ARG unless N is a multiple of n_patches, n_v is even in 2..256,
 * eps > 0.  Same as msp_kinetic_build_hg with g = 0. */
msp_status msp_kinetic_build(int n_cells, double eps, int n_v, int n_patches, int buffer, int samples,
                             void* stream, msp_kmedium* out);

/* The slab with the Henyey-Greenstein collision of Eq. HG (Sec. 4):
 *     v d_x f = (1/eps) [ int k(v, v') f(v') dv' - (int k(v', v) dv') f(v) ],
 *     k(v, v') = (1/2) (1 - g^2) / (1 + g^2 + 2 g v v'),
 * both integrals by the Gauss-Legendre rule.  g in (-1, 1) (INVALID_ARG
 * otherwise); g != 0 needs n_v <= 128 and selects the direct solver
 * (msp_kinetic_set_solver).  Everything else as msp_kinetic_build. */
msp_status msp_kinetic_build_hg(int n_cells, double eps, double g, int n_v, int n_patches, int buffer, int samples,
                                void* stream, msp_kmedium* out);

/* Local solver of msp_kinetic_sample.
 * MSP_KINETIC_SOURCE_ITERATION (default at g = 0; g = 0 only): transport sweeps
 *   with the lagged density, as described at msp_kinetic_sample.
 * MSP_KINETIC_DIRECT (default at g != 0; n_v <= 128): block LU of the upwind
 *   operator over the nodes of each buffered patch (the inverse of every
 *   n_v x n_v Schur complement kept; factorised at the first sample call of
 *   each precision and reused), FP64 residual refinement: precision MSP_FP64
 *   factors in FP64, MSP_MIXED in FP32; stops when max_l |r_l| / D_ll <=
 *   tol max |f| (r the FP64 residual, D the operator's diagonal) after at most
 *   min(max_iter, 16) corrections; iterations in the stats count corrections.
 * INVALID_ARG for another value or a solver the medium cannot take. */
#define MSP_KINETIC_SOURCE_ITERATION 0
#define MSP_KINETIC_DIRECT 1
msp_status msp_kinetic_set_solver(msp_kmedium k, int solver);
void msp_kinetic_destroy(msp_kmedium k);
/* Gauss-Legendre velocities and weights (host arrays of n_v, either may be NULL). */
msp_status msp_kinetic_velocities(msp_kmedium k, double* v_host, double* w_host);

/* RanLocalSolu for the slab (Eq. rte_random): per patch and sample, i.i.d.
 * N(0,1) incoming data on the buffered patch (Philox4x32-10, counter = (datum
 * pair, sample, patch, kinetic tag); data 0..n_v/2-1 are the positive velocities
 * at the left end, the rest the negative velocities at the right end, each
 * ascending in v), restricted to K_m.  precision MSP_FP64: source iteration
 * (FP64 transport sweeps with the lagged density) until max|rho_new - rho| <=
 * tol max|rho|.  MSP_MIXED: FP64 residuals of the density with FP32 source-
 * iteration corrections (each to a relative 1e-6, at most max_iter sweeps),
 * stopped on the same criterion; iterations in the stats count FP32 and FP64
 * sweeps.  stats as for msp_sample_patches (synchronises when given). */
msp_status msp_kinetic_sample(msp_kmedium k, uint64_t seed, int precision, double tol, int max_iter, void* stream,
                              msp_solve_stats* stats_host);
/* Copy patch `patch`'s snapshot block ((W+1) n_v x samples, column-major). */
msp_status msp_kinetic_get_snapshots(msp_kmedium k, int patch, double* dst_dev, void* stream);

/* Truncated SVD bases of the snapshots (as msp_extract_basis) and the FP64
 * block-tridiagonal factor of the normal equations of Eq. rte_cond_reduced
 * (continuity of all velocities at every interface, incoming data at x = 0, 1).
 * Synchronises.  BREAKDOWN if the normal matrix is not positive definite. */
msp_status msp_kinetic_extract(msp_kmedium k, double tau, void* stream, msp_kbasis* out);
void msp_kinetic_basis_destroy(msp_kbasis b);
msp_status msp_kinetic_basis_info(msp_kbasis b, int patch, int* k, double* sigma_host);

/* Online stage for `batch` data sets: inflow_dev [batch][2][n_v] holds, per data
 * set, the n_v values at x = 0 (only v > 0 used) then the n_v values at x = 1
 * (only v < 0 used).  c = argmin |P c - d| by the factorised normal equations
 * with two corrected-semi-normal-equation steps; f_dev [batch][N+1][n_v]
 * receives the reconstruction (patch values inside, interface averages, the
 * incoming data at the ends); c_dev [batch][N_p] optional.  Synchronises. */
msp_status msp_kinetic_online_solve(msp_kbasis b, const double* inflow_dev, int batch, double* f_dev, double* c_dev,
                                    void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MSP_H */
