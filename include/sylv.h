/*
 * sylv.h -- C ABI of the GB300 (sm_103a) solver for the N-dimensional
 * Sylvester tensor equation
 *
 *     sum_{j=1..N} A_j (x)_j X = B,
 *     [A (x)_j X]_{i_1..i_j..i_N} = sum_k a_{i_j k} x_{i_1..k..i_N}
 *
 * (Cuesta & de la Hoz, arXiv 2412.15840, Section 1, Eq. (sylvesterND)), by the
 * non-recursive Bartels-Stewart method of Section 2 / Algorithm 3:
 *   setup    A_j = U_j T_j U_j^*  (complex Schur, host FP64, once per plan);
 *   forward  C = U_N^* (x)_N ( ... (U_1^* (x)_1 B))        Eq. (CUNU2U1B);
 *   sweep    sum_j T_j (x)_j Y = C solved entrywise         Eq. (yi1i2iN);
 *   back     X = U_N (x)_N ( ... (U_1 (x)_1 Y))           Eq. (XUNU2U1Y).
 *
 * Conventions shared by every entry point
 *  - Complex numbers are interleaved (re, im) pairs: complex128 = 2 doubles,
 *    complex64 = 2 floats.
 *  - Matrices (A_j, U_j, T_j) are column-major n_j x n_j complex128 in HOST
 *    memory: entry (a, b) is at [2*(a + b*n_j)].  The real-arithmetic
 *    variant (sylv_plan_create_real) takes float64 A_j, entry (a, b) at
 *    [a + b*n_j], and float64 / float32 tensors.
 *  - Tensors are column-major with i_1 fastest (Section 2.2, Eq. (index)) and
 *    live in DEVICE memory; a tensor with nrhs right-hand sides has one extra
 *    trailing index of extent nrhs (the right-hand sides are independent).
 *  - Modes with n_j = 1 ("singletons", Section 4) carry a scalar A_j; they are
 *    not transformed and add a_j to every diagonal sum.
 *  - All device work is stream-ordered on the caller's `stream` (a
 *    cudaStream_t passed as void*; NULL = legacy default stream) and
 *    asynchronous unless stated.  No entry point throws; every failure is a
 *    sylv_status.  CUDA errors map to SYLV_ERR_CUDA.
 *  - The library allocates device memory only inside sylv_plan_create (and
 *    sylv_plan_create_real, sylv_plan_autotune for its candidate tables): the
 *    factors and tiling tables, and, when prod_j n_j * 16 bytes <= 1 GiB, a
 *    table of the sweep's FP64 reciprocals (one per multi-index; without it
 *    the sweep forms them on the fly).  Tensor-sized scratch memory
 *    is the caller's: query sylv_workspace_size and pass a device buffer of at
 *    least that many bytes, 256-byte aligned.
 *  - A plan may be used by one stream at a time: calls that overlap on the
 *    GPU and share a workspace race.
 */
#ifndef SYLV_H
#define SYLV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sylv_plan_s *sylv_plan_t;

typedef enum {
    SYLV_OK = 0,
    SYLV_ERR_INVALID_ARG = 1,   /* NULL pointer, bad precision, misaligned buffer, ... */
    SYLV_ERR_SHAPE = 2,         /* N < 1, n_j < 1, nrhs < 1, overflow, too many modes  */
    SYLV_ERR_SINGULAR = 3,      /* some t_{1,i1i1}+...+t_{N,iNiN} is 0 or not finite   */
    SYLV_ERR_NOT_CONVERGED = 4, /* mixed path: refinement did not reach rtol           */
    SYLV_ERR_TIMEOUT = 5,       /* a device-side dependency wait hit its time limit    */
    SYLV_ERR_OOM = 6,           /* plan-time device allocation failed                  */
    SYLV_ERR_CUDA = 7,          /* any other CUDA runtime error                        */
    SYLV_ERR_SCHUR = 8,         /* the host Schur iteration did not converge           */
    SYLV_ERR_WORKSPACE = 9      /* workspace NULL or smaller than required             */
} sylv_status;

typedef enum {
    SYLV_FP64 = 0,        /* every phase in FP64 (complex128)                          */
    SYLV_MIXED_FP32 = 1,  /* forward / sweep / back in FP32 (complex64) with the FP64
                             diagonal division, FP64 residual and FP64 update:
                             iterative refinement to relative error rtol            */
    SYLV_MIXED_FP32_EMU = 2 /* as SYLV_MIXED_FP32, but the residual's mode products run
                             on the bf16 tensor cores, exactly on 6 base-256 digits of
                             X / 2^eX and A_j / 2^eA (Ozaki-style splitting), summed in
                             FP32 pairs: the residual is accurate to ~2^-45 of
                             sum_j ||A_j|| ||X|| instead of FP64 rounding.  Used when
                             every non-singleton mode has 8 <= n_j <= 64 and either
                             prod_{m<j} n_m >= 8 or (first mode) at least 64 columns
                             (prod_{m>1} n_m times nrhs), and when the ratio of the
                             largest to the smallest |diagonal sum| (a lower bound of
                             the condition number kappa) times 2^-44 is <= rtol: the
                             refined error is about kappa 2^-45.  Otherwise the
                             residual stays FP64 (sylv_info.path bit 1 tells which
                             ran).  For strongly non-normal operators, whose kappa can
                             far exceed that ratio, SYLV_MIXED_FP32 is the safe
                             choice.  Entries of B and of the scaled products must lie
                             in the FP32 range. */
} sylv_prec;

/* Per-solve report, filled (after a stream synchronisation) only when the
 * caller passes a non-NULL pointer. */
typedef struct {
    int32_t status;           /* sylv_status of the device-side checks              */
    int32_t refine_iters;     /* refinement steps taken (0 for SYLV_FP64)             */
    int32_t launches;         /* kernels this call enqueued                           */
    int32_t path;             /* bit 0: the sweep ran as the entrywise division of
                                 Remark 1 (every A_j normal, see sylv_tuning);
                                 bit 1: the residual ran on the tensor cores
                                 (SYLV_MIXED_FP32_EMU);
                                 bit 2: real-arithmetic plan (sylv_plan_create_real) */
    double last_corr_rel;     /* ||D_k|| / ||X_k|| of the last refinement step        */
    double est_rel_err;       /* contraction-based estimate of the final error        */
    double min_abs_den;       /* min |sum_j t_{j,i_j i_j}| over all multi-indices      */
    double max_abs_den;       /* max of the same                                       */
} sylv_info;

/* Phase timing accumulated by CUDA events when enabled with sylv_plan_set_timing. */
typedef struct {
    double ms[8];             /* forward, sweep, back, residual, update, total,
                                 evolve (the right-hand side of Theorem 1), unused    */
    int64_t launches[8];      /* kernel launches per phase                             */
    int64_t solves;           /* solves accumulated                                    */
} sylv_timing;

enum { SYLV_PH_FORWARD = 0, SYLV_PH_SWEEP = 1, SYLV_PH_BACK = 2, SYLV_PH_RESIDUAL = 3,
       SYLV_PH_UPDATE = 4, SYLV_PH_TOTAL = 5, SYLV_PH_EVOLVE = 6 };

/* Optional tuning (NULL = defaults).  block[j] = sweep tile extent along input
 * mode j (0 = automatic); group_max = largest product of adjacent mode sizes
 * fused into one transform pass (0 = automatic). */
typedef struct {
    int32_t block[64];
    int32_t group_max;
    int32_t sweep_threads;    /* 0 = automatic */
    int32_t no_tensor_cores;  /* 1 = FP32 transforms on CUDA cores only */
    int32_t timeout_ms;       /* limit of each device-side dependency wait (0 = 2000) */
    int32_t fault_tile;       /* test hook: k > 0 makes the sweep never release the
                                 predecessors of its (k-1)-th tile, so that their waits
                                 run out and the solve reports SYLV_ERR_TIMEOUT */
    int32_t general_sweep;    /* 0 = automatic: when every T_j is diagonal to rounding,
                                 ||strict upper part of T_j||_F <= 4 n_j 2^-53 ||T_j||_F
                                 (A_j normal, Section 2, Remark 1), the sweep is the
                                 entrywise division y = c / (sum_j t_{j,i_j i_j}) of
                                 Eq. (yi1i2iNdiag), computed in FP64 and ignoring the
                                 rounding-level off-diagonal entries; 1 = always run
                                 the triangular sweep of Eq. (yi1i2iN) */
    int32_t sweep_ctas_per_sm;  /* 0 = as many sweep CTAs per SM as fit; k > 0 caps it
                                 (fewer CTAs shorten each tile's latency) */
    int32_t tc_plain;         /* 1 = tensor-core transform passes without the TMA-fed
                                 warp-specialised pipeline (0 = use it where it applies:
                                 modes after the first with a stride that is a multiple
                                 of 64 and n_j <= 64) */
} sylv_tuning;

/*
 * sylv_plan_create -- setup for one equation shape (Section 2 and Algorithm 3,
 * first loop: the Schur factors; Section 2.1 puts its cost at ~25 n_j^3).
 *   N        number of modes, 1 <= N <= 256.
 *   n        host int64[N], n_j >= 1.  At most 40 modes may have n_j > 1.
 *   nrhs     right-hand sides per solve, >= 1.
 *   A        host array of N pointers to n_j x n_j complex128 matrices, or NULL.
 *   Q, T     host arrays of N pointers to precomputed Schur factors
 *            (A_j = Q_j T_j Q_j^*, T_j upper triangular; entries below the
 *            diagonal are ignored), or NULL.  Exactly one of A or (Q and T)
 *            must be non-NULL.  For a singleton mode Q_j is ignored and T_j
 *            holds the scalar.  All matrices are copied; the caller keeps them.
 *   prec     sylv_prec.
 *   rtol     mixed path: target relative error (e.g. 1e-10); ignored for FP64.
 *   max_refine  mixed path: maximum refinement steps (>= 1).
 *   device   CUDA device ordinal that owns the plan.
 *   tuning   optional, may be NULL.
 * Returns SYLV_OK and *out, or an error and *out = NULL.  SYLV_ERR_SINGULAR if
 * some diagonal sum is zero or not finite (Eq. (yi1i2iN) needs it nonzero).
 * Synchronises the device once (the tables are uploaded and checked).
 */
sylv_status sylv_plan_create(sylv_plan_t *out, int N, const int64_t *n, int64_t nrhs,
                             const double *const *A, const double *const *Q,
                             const double *const *T, int prec, double rtol,
                             int max_refine, int device, const sylv_tuning *tuning);

/*
 * sylv_plan_create_real -- the real-arithmetic variant for real A_j and real
 * right-hand sides: A_j = Q_j T_j Q_j^T with Q_j orthogonal and T_j
 * quasi-upper-triangular (real Schur form, 2 x 2 diagonal blocks for
 * complex-conjugate eigenvalue pairs; sylv_schur_real), so the transforms of
 * Eqs. (CUNU2U1B) and (XUNU2U1Y) run on real tensors with real Q_j (half the
 * bytes and a quarter of the flops of the complex path).  The sweep of
 * Eq. (yi1i2iN) keeps real C and Y in memory; inside a tile the entries coupled
 * by 2 x 2 blocks are rotated by the blocks' unitary Schur vectors V_j to the
 * complex triangular V_j^* T_j V_j, solved, and rotated back.
 *   A        host array of N pointers to n_j x n_j float64 matrices (column-major).
 *   prec     SYLV_FP64 (float64 tensors) or SYLV_MIXED_FP32 (float32 working
 *            tensor, FP64 residual); SYLV_MIXED_FP32_EMU is not offered.
 *   Other arguments as sylv_plan_create.
 * A plan made here takes float64 B and X in sylv_solve / sylv_solve_batched,
 * and its working-precision tensors (sylv_forward / sylv_sweep / sylv_back) are
 * float64 (SYLV_FP64) or float32 (SYLV_MIXED_FP32); sylv_residual reads and
 * writes float64.  sylv_plan_factors returns the real Q_j and T_j with zero
 * imaginary parts.  sylv_evolve is not offered (SYLV_ERR_INVALID_ARG).
 * SYLV_ERR_SHAPE if a sweep tile cannot hold every coupled pair: each mode with
 * a 2 x 2 block needs a tile extent of at least 2, and a tile holds at most
 * 8192 entries (at most 13 such modes).
 */
sylv_status sylv_plan_create_real(sylv_plan_t *out, int N, const int64_t *n, int64_t nrhs,
                                  const double *const *A, int prec, double rtol, int max_refine,
                                  int device, const sylv_tuning *tuning);

sylv_status sylv_plan_destroy(sylv_plan_t plan);

/* Bytes of device workspace a solve with this plan needs (0 is possible). */
sylv_status sylv_workspace_size(sylv_plan_t plan, size_t *bytes);

/*
 * sylv_solve -- Algorithm 3 on the device: forward transform, triangular
 * sweep, back transform; for SYLV_MIXED_FP32 followed by the FP64 residual
 * R = B - sum_j A_j (x)_j X, a low-precision solve of R and the FP64 update
 * X += D, repeated until the estimated relative error is below rtol.
 *   B_dev  device complex128 tensor n_1 x ... x n_N x nrhs (read only).
 *   X_dev  device complex128 tensor of the same shape (written).  X_dev ==
 *          B_dev (in place, as Section 4 does) is allowed for SYLV_FP64 only.
 *   workspace, workspace_bytes  device scratch (see sylv_workspace_size).
 *   info   optional; when non-NULL the call synchronises `stream` and fills it.
 * Stream-ordered and asynchronous when info == NULL.
 */
sylv_status sylv_solve(sylv_plan_t plan, const void *B_dev, void *X_dev, void *workspace,
                       size_t workspace_bytes, void *stream, sylv_info *info);

/*
 * sylv_solve_batched -- `count` independent equations (any shapes) in one
 * call.  The equations' launch sequences are recorded once per argument set
 * (plans, tensors, workspace) into a CUDA graph, spread over up to 8 forked
 * streams so that small equations run concurrently, and replayed by one
 * graph launch on `stream` on every later call with the same arguments.
 * plans[e], B_dev[e], X_dev[e] as for sylv_solve (one device for all plans);
 * the workspace must hold sylv_workspace_size_batched bytes.  infos may be
 * NULL, else an array of `count` reports (the call then synchronises).  A
 * plan with phase timing enabled makes the call launch directly, in order.
 * The first call with a new argument set must not happen during a stream
 * capture of the caller's own.
 */
sylv_status sylv_workspace_size_batched(int count, const sylv_plan_t *plans, size_t *bytes);
sylv_status sylv_solve_batched(int count, const sylv_plan_t *plans, const void *const *B_dev,
                               void *const *X_dev, void *workspace, size_t workspace_bytes,
                               void *stream, sylv_info *infos);

/*
 * sylv_evolve -- Theorem 1 (Section 3): the solution at time t of the linear
 * ODE system
 *     X_t = sum_j A_j (x)_j X + B,   X(0) = X0,
 * with the plan's A_j, as the solution of the Sylvester equation
 *     sum_j A_j (x)_j X(t) = F,
 *     F = exp(t A_N) (x)_N ( ... exp(t A_1) (x)_1 (sum_j A_j (x)_j X0 + B)) - B
 * (Eqs. (sylvesterNDC) and (C)).  A singleton mode contributes the scalar
 * factor exp(t a_j).  F is formed on the device in FP64 (one FP64 pass of the
 * products A_j (x)_j X0 and one of the exp(t A_j) products), then solved as by
 * sylv_solve in the plan's precision (with refinement for SYLV_MIXED_FP32).
 *   t        finite real time (t = 0 returns X0 up to rounding).
 *   B, X0    device complex128 tensors of the plan's shape (x nrhs), read only.
 *   X        device complex128 output; may be the same buffer as X0 or B.
 *   workspace  device buffer of sylv_evolve_workspace_size bytes (256-byte
 *            aligned): the plan's solve workspace plus one complex128 tensor.
 *   info     as for sylv_solve (the launches include the F passes).
 * The exponentials exp(t A_j) are computed on the host (sylv_expm) when t
 * differs from the previous call's and copied to the plan's device buffers in
 * stream order; calls with the same t enqueue device work only.
 * Errors: SYLV_ERR_INVALID_ARG (NULL or misaligned pointers, non-finite t,
 * non-finite exponentials), SYLV_ERR_WORKSPACE, SYLV_ERR_CUDA, and those of
 * sylv_solve.
 */
sylv_status sylv_evolve_workspace_size(sylv_plan_t plan, size_t *bytes);
sylv_status sylv_evolve(sylv_plan_t plan, double t, const void *B, const void *X0, void *X,
                        void *workspace, size_t workspace_bytes, void *stream,
                        sylv_info *info);

/*
 * Single phases (same tensors and workspace rules as sylv_solve), in the
 * plan's working precision: complex128 for SYLV_FP64, complex64 for
 * SYLV_MIXED_FP32.  They expose the steps of Algorithm 3 one by one so that
 * each can be checked against a reference that uses the plan's own factors.
 *   sylv_forward   C = U_N^* (x)_N ( ... (U_1^* (x)_1 B)),  in place on T_dev.
 *   sylv_sweep     Y with sum_j T_j (x)_j Y = C, Eq. (yi1i2iN), in place.
 *   sylv_back      X = U_N (x)_N ( ... (U_1 (x)_1 Y)),  in place.
 * sylv_residual computes, in FP64, R = B - sum_j A_j (x)_j X on complex128
 * tensors (R_dev must not alias B_dev or X_dev).
 */
sylv_status sylv_forward(sylv_plan_t plan, void *T_dev, void *workspace, size_t workspace_bytes,
                         void *stream);
sylv_status sylv_sweep(sylv_plan_t plan, void *T_dev, void *workspace, size_t workspace_bytes,
                       void *stream);
sylv_status sylv_back(sylv_plan_t plan, void *T_dev, void *workspace, size_t workspace_bytes,
                      void *stream);
sylv_status sylv_residual(sylv_plan_t plan, const void *B_dev, const void *X_dev, void *R_dev,
                          void *stream);

/*
 * sylv_sweep_static -- the same triangular sweep as sylv_sweep, for callers
 * that cannot allocate device memory at all: code that runs with a fixed
 * device-memory budget fully reserved up front (for instance by another
 * framework's caching allocator, so a cudaMalloc would fail), or code in a
 * latency-critical loop where a cudaMalloc/cudaFree would stall on an
 * implicit device synchronisation.  The paper has no counterpart; this is a
 * service of this library.
 *
 * The sweep's scratch (a 64-byte control block plus one int per tile) comes
 * from one array of SYLV_STATIC_SCRATCH_BYTES inside the library, which every
 * GPU that loads the library holds until the process exits; nothing is
 * allocated and no workspace is passed.  T_dev is as for sylv_sweep (plan's
 * working precision, in place).
 *  - The tiled sweep needs 256 bytes for the control block plus 4 bytes per
 *    tile rounded up to 256, i.e. at most 262,080 tiles in the 1 MiB array;
 *    plans with more tiles are rejected with SYLV_ERR_SHAPE.  A plan whose
 *    sweep is the entrywise division of Remark 1 (sylv_info.path bit 0)
 *    needs the control block only and is never refused for its size.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and keeps it for the
 *    life of the process; make that first call before any stream capture.
 *    Calls after a cudaDeviceReset of that device are not supported (the
 *    kept address belongs to the destroyed context).
 *  - Every call on a device shares the one array and leaves its contents
 *    behind; each call clears what must start at zero before it sweeps.
 *    Calls whose work overlaps on the GPU (other streams, other threads,
 *    other plans) race on the array and give wrong results: serialise them.
 */
#define SYLV_STATIC_SCRATCH_BYTES (1u << 20)
sylv_status sylv_sweep_static(sylv_plan_t plan, void *T_dev, void *stream);

/*
 * sylv_plan_autotune -- measure candidate tilings of the triangular sweep on
 * this device (tile extents from ~64 to ~2048 entries, 128 or 256 threads
 * per CTA, 1 or 4 lanes per entry in the in-tile wavefront, each number of
 * CTAs per SM) for the plan's own shape and keep the fastest; then the
 * transform passes: the plan's tensor-core passes with or without the TMA
 * pipeline, or CUDA-core passes only at several fusion widths of adjacent
 * modes (one forward and one back transform timed per candidate).  T_dev: scratch
 * tensor in the plan's working precision (complex128 for SYLV_FP64, complex64
 * for SYLV_MIXED_FP32), overwritten with zeros and sweep results; workspace as
 * for sylv_solve.  The workspace size of the plan does not change.  On
 * return block_out[j] (nullable, N entries) holds the chosen extent along
 * input mode j and *best_ms (nullable) the measured sweep time.
 * Synchronises `stream`.
 */
sylv_status sylv_plan_autotune(sylv_plan_t plan, void *T_dev, void *workspace,
                               size_t workspace_bytes, void *stream, int32_t *block_out,
                               float *best_ms);

/*
 * sylv_plan_describe -- the launch structure the plan chose (host-only, no
 * device work): how Algorithm 3's phases map onto passes and tiles on this
 * GPU.  Useful to relate a measured phase time to its pass-model traffic
 * and to report the settings that sylv_plan_autotune picked.
 */
typedef struct {
    int32_t transform_passes;   /* passes of one forward (= one back) transform in the
                                   working precision (fused groups of adjacent modes) */
    int32_t transform_tc_passes;/* of which on the tensor cores (tcgen05)              */
    int32_t residual_passes;    /* passes of one residual (mixed precisions)           */
    int32_t residual_tc;        /* 1: the residual runs on the tensor cores            */
    int32_t diag_sweep;         /* 1: the sweep is the entrywise division of Remark 1  */
    int32_t sweep_threads;      /* threads per CTA of the tiled sweep                  */
    int32_t sweep_ctas_per_sm;  /* resident CTAs per SM of its persistent grid         */
    int32_t sweep_grid;         /* CTAs of its persistent grid                         */
    int64_t sweep_tiles;        /* tiles (right-hand sides included)                   */
    int32_t sweep_tile_entries; /* entries of a full tile                              */
    int32_t sweep_tile_levels;  /* tile levels sum_j (blocks_j - 1) + 1                */
    int32_t sweep_inv_table;    /* 1: FP64 reciprocals read from the plan's table      */
    int32_t sweep_far_split;    /* 1: far strips applied ahead of the full wait        */
    int32_t sweep_block[64];    /* tile extent along each input mode (first N used)    */
    int32_t sweep_lanes;        /* lanes per entry in the sweep's in-tile wavefront    */
    int32_t transform_tma;      /* tensor-core passes fed by the TMA pipeline          */
    int32_t transform_group_max;/* fusion width of the CUDA-core passes (0: automatic) */
    int32_t sweep_3m;           /* 1: FP64 complex strips by three multiplications     */
    int32_t transform_fib_passes;/* of the transform passes: one thread per fibre      */
} sylv_plan_desc;
sylv_status sylv_plan_describe(sylv_plan_t plan, sylv_plan_desc *out);

/* The plan's Schur factors of input mode j (host copies; Q is the identity
 * 1x1 for a singleton).  Q_out and T_out hold n_j*n_j complex128 each. */
sylv_status sylv_plan_factors(sylv_plan_t plan, int j, double *Q_out, double *T_out);

/* Phase timing with CUDA events recorded on the solve's stream.  Enabling it
 * adds event records between phases; sylv_plan_timing synchronises those
 * events, writes the sums and, if reset != 0, clears them. */
sylv_status sylv_plan_set_timing(sylv_plan_t plan, int enable);
sylv_status sylv_plan_timing(sylv_plan_t plan, sylv_timing *out, int reset);

/*
 * Host-only helper (no GPU needed): complex Schur decomposition A = Q T Q^*
 * of one n x n complex128 matrix by Householder reduction to Hessenberg form
 * and shifted QR (Section 2 uses this factorisation; the algorithm is the
 * textbook one, e.g. Golub & Van Loan, ch. 7).  A, Q, T column-major.
 */
sylv_status sylv_schur(int64_t n, const double *A, double *Q, double *T);

/*
 * Host-only helper (no GPU needed): real Schur decomposition A = Q T Q^T of one
 * n x n real (float64) matrix, the factorisation the real-arithmetic variant
 * uses: Q orthogonal, T quasi-upper-triangular with 1 x 1 blocks for real
 * eigenvalues and 2 x 2 blocks for complex-conjugate pairs (Golub & Van Loan,
 * ch. 7: Hessenberg reduction, Francis double-shift QR).  Every 2 x 2 block
 * starts at an even index (T[k+1, k] != 0 only for even k), reached by direct
 * swaps of adjacent blocks (Bai & Demmel 1993).  A, Q, T column-major, n*n
 * doubles each.  SYLV_ERR_SCHUR if QR does not converge or a swap is
 * ill-conditioned; SYLV_ERR_INVALID_ARG for n < 1 or non-finite entries.
 */
sylv_status sylv_schur_real(int64_t n, const double *A, double *Q, double *T);

/*
 * sylv_expm -- host-only matrix exponential E = exp(M) of an n x n complex128
 * matrix (column-major, 1 <= n <= 1024), by scaling and squaring with the
 * [13/13] Pade approximant (Higham, SIAM J. Matrix Anal. Appl. 26(4), 2005).
 * sylv_evolve uses it for the exp(t A_j) of Eq. (C).  No device is touched.
 * SYLV_ERR_INVALID_ARG for non-finite input or result.
 */
sylv_status sylv_expm(int64_t n, const double *M, double *E);

/* Human-readable name of a status code (static storage). */
const char *sylv_status_string(sylv_status s);

/* Library version as major*10000 + minor*100 + patch. */
int sylv_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SYLV_H */
