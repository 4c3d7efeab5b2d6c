// Internal declarations shared by the host runtime (capi.cu, schur.cpp) and
// the sm_103a kernels (kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/sylv.h"

#ifdef __CUDACC__
#include <cuda_runtime.h>
#endif

namespace sylv {

constexpr int MAXM = 40;   // modes with n_j > 1 (after singleton removal)
constexpr int MAXG = 16;   // modes fused into one transform pass
constexpr int FIB_NMAX = 24;  // longest fibre of the one-thread-per-fibre FP32 pass (at
                              // n = 32 its 154 registers leave one CTA per SM, and the
                              // tensor-core pass is faster: 32^5 forward 1.07 vs 1.27 ms)
constexpr int MAX_N = 1024;
constexpr int SWEEP_KCH = 64;  // columns of T_j staged per chunk by the sweep
constexpr size_t INV_TABLE_MAX = (size_t)1 << 30;  // plan-resident reciprocal table budget
constexpr int SWEEP_BMAX = 64; // automatic tile extents stay <= 64 per mode, so the
                               // tile's diagonal T blocks fit in shared memory

sylv_status schur_host(int64_t n, const double *A, double *Q, double *T);
sylv_status expm_host(int64_t n, const double *M, double *E);
sylv_status schur_real_host(int64_t n, const double *A, double *Q, double *T);

// Device-side control block at the start of every workspace.
struct DevFlags {
    int done;        // refinement finished: later kernels of the solve return at once
    int err;         // bit set of sylv_status codes raised on the device
    int ticket;      // sweep: next tile ticket
    int iters;       // refinement steps taken
    unsigned dmax;   // float bits: max(|re|,|im|) of the last correction D
    unsigned xmax;   // float bits: max(|re|,|im|) of the updated X
    float dprev;     // ||D_{k-1}|| (||X_0|| before the first step)
    float est;       // estimated relative error after the last step
    float lastcorr;  // ||D_k|| / ||X_k||
    unsigned xlast;  // float bits: max(|re|,|im|) of the current X (scale of the residual)
    int pad[6];
};
static_assert(sizeof(DevFlags) == 64, "DevFlags layout");

enum { ERRBIT_TIMEOUT = 1, ERRBIT_NOTCONV = 2, ERRBIT_NAN = 4 };

enum Epi { EPI_STORE = 0, EPI_RESID = 1, EPI_ACCUM = 2, EPI_STORE_NORM = 3, EPI_SUB = 4 };
// element types of a tensor: complex64 / complex128, or float32 / float64 for
// the real-arithmetic variant
enum ElemKind { ELEM_C64 = 0, ELEM_C128 = 1, ELEM_R32 = 2, ELEM_R64 = 3 };

// One transform pass over the view (L, P, R) of a tensor, where P is the
// product of the sizes of `G` adjacent modes; tiles are Lt x P x Rt.
struct MPArgs {
    const void *in;
    void *out;
    const void *mats[MAXG];   // n x n column-major, compute precision
    int gn[MAXG];
    int G;
    int Lt, Rt;
    int64_t L, P, R;
    int64_t tilesL;
    // residual: R = (first ? B - sigma*X : R) - sum_m A_m (x)_m X;
    // EPI_SUB: out = sigma * (product) - B
    const void *B;
    double sig_re, sig_im;
    int first;
    int g3;                   // FP64 residual: three-multiplication products (re + im
                              // plane of X staged beside the tile); 0: classical
    int rows4;                // FP64 residual of one mode: four rows per thread (a pass
                              // with enough tiles to fill the GPU several times)
    // norms (float bits, max(|re|,|im|))
    DevFlags *flags;
    const int *done;          // early exit when *done != 0 (nullable)
};

struct SweepArgs {
    void *Y;
    int Nm;
    int nin;                  // modes with block > 1 (inside a tile)
    int Lin;                  // in-tile levels
    int Pt;                   // entries of a full tile
    int bmax;                 // largest in-tile block extent
    int fast;                 // packed coordinates available (their widths fit 64 bits)
    int cshift[MAXM];         // bit offset of in-tile mode q in a packed coordinate
    unsigned cmask[MAXM];     // its mask (ceil(log2 b) bits)
    double den_scale;         // power of two keeping |scale * diagonal sum|^2 in range
    int64_t n[MAXM];
    int64_t S[MAXM];          // element strides
    int64_t TS[MAXM];         // tile-index strides
    int b[MAXM];              // block extents
    int Bc[MAXM];             // blocks per mode
    int inmode[MAXM];         // indices of in-tile modes
    int BS[MAXM];             // box strides of in-tile modes (by position in inmode)
    int tdoff[MAXM];          // offset of each in-tile mode's b x b diagonal block of T
    int tdsize;               // entries of all diagonal blocks
    int qpos[MAXM];           // position of mode j in inmode, or -1
    const void *T[MAXM];      // T_j, compute precision, column-major
    const double *d[MAXM];    // diag(T_j) as interleaved FP64 pairs
    double sig_re, sig_im;
    int64_t ntiles1, ntiles, ntot;
    const int *order;         // tile ids by level
    int *cnt;                 // per-tile count of unfinished immediate successors
    DevFlags *flags;
    const int *sched;         // in-tile schedule (a'-linear offsets by level)
    const int *sched_e;       // the same schedule as box offsets, for full tiles
    const unsigned long long *coord;  // per box offset: in-tile coordinates, 8 bits each
    const int *offs;          // per box offset: element offset sum_q t_q S_q from the tile's
                              // first entry (full tiles; when use_offs)
    int use_offs;
    const int *lev_start;     // Lin + 1 entries
    long long timeout_cycles;
    int fault_tile;           // test hook: this tile never releases its predecessors (-1: none)
    const void *inv_tab;      // per multi-index reciprocals in the sweep's format, or null
    // real-arithmetic variant (real = 1): C and Y are real; T holds the complex
    // triangular T~_j = V_j^* T_j V_j (in-tile blocks and diagonal), Tr the real
    // quasi-triangular T_j (strips of solved tiles), Vp the unitary 2 x 2 Schur
    // vectors V of the diagonal blocks, 4 complex entries (column-major) per
    // pair of indices (2u, 2u + 1), identity where both are 1 x 1 blocks; null
    // for a mode without 2 x 2 blocks
    int far_split;            // strips beyond the successor block before the full wait
    int sub;                  // lanes per entry in the in-tile wavefront (1, 2 or 4)
    int g3;                   // FP64 complex strips by three multiplications (re + im plane
                              // of the staged T block in shared memory)
    int real;
    const void *Tr[MAXM];
    const void *Vp[MAXM];
};

// Batched sweep over many equations in one persistent launch: each
// equation's full sweep arguments (device copy owned by its plan) and the
// call's tensor, tile counters and control block; cum[e] = tiles of the
// equations before e.  Passed by value as the kernel parameter.
constexpr int SWB_MAX = 512;
struct SweepBatch {
    int neq;
    int far_split;
    const SweepArgs *sa[SWB_MAX];
    void *Y[SWB_MAX];
    int *cnt[SWB_MAX];
    DevFlags *flags[SWB_MAX];
    long long cum[SWB_MAX + 1];
};

// Sweep of a plan whose T_j are all diagonal (every A_j normal, Remark 1):
// y = c / (sigma + sum_j t_{j,i_j i_j}), Eq. (yi1i2iNdiag).  The leading
// modes whose size product P1 is at most DIAG_HEAD_MAX share one table of
// partial diagonal sums; the remaining ("tail") modes are decoded per column
// of P1 consecutive entries.
constexpr int64_t DIAG_HEAD_MAX = 4096;
struct DiagArgs {
    void *Y;
    int64_t total;            // ntot * nrhs entries
    int64_t P1;               // product of the head modes' sizes
    int64_t Qt;               // ntot / P1 (tail index range without the right-hand sides)
    const double *dhead;      // P1 complex FP64: sigma + sum over the head modes
    int Nt;                   // tail modes
    int64_t tn[MAXM];
    const double *td[MAXM];   // diag(T_j) of the tail modes, interleaved FP64
    double den_scale;
    DevFlags *flags;
};

// dynamic shared memory of the tensor-core pass (below the 227 KB opt-in limit,
// leaving room for its static shared memory)
constexpr int TC_SMEM_MAX = 220 * 1024;

// Tensor-core (tcgen05, 3xTF32) transform pass over one mode, complex64 in.
// mode1 = 0: modes with L >= 64, a tile is 64 consecutive l of one r;
// mode1 = 1: the first mode (L = 1), a tile is 64 consecutive columns r.
struct TCArgs {
    const void *in;               // complex64 tensor (complex128 allowed when mode1)
    void *out;                    // complex64, or complex128 for the last back pass
    const unsigned char *bimg;    // B_hi image followed by B_lo image (shared-memory layout)
    int n, Kp, Np;                // mode size, K padded to 8, N = 2n padded to 16
    int mode1;                    // 1: first-mode pass (L = 1)
    int in_c128;                  // mode1 only: the input is complex128
    int lboA, sboA, sboB;         // A: K-adjacent and 8-row-group strides; B: 8-row stride
    int abytes;                   // bytes of one A image (hi or lo)
    int bimg_bytes;               // bytes of one B image
    int tmem_cols;                // TMEM columns of one accumulator (power of two >= 32)
    int nbuf;                     // A operand / accumulator buffers (1 or 2)
    int64_t L, R, tilesL;         // view (L, n, R); tiles of 64 along L (or R when mode1)
    DevFlags *flags;
    const int *done;
};

// Residual pass on the bf16 tensor cores (digit splitting, see resid_oz.cu).
struct OzArgs {
    const void *X;                // complex128
    const void *B;                // complex128 (first pass)
    const void *Rin;              // R as FP32 pairs (re hi, im hi, re lo, im lo)
    void *Rout;                   // output as FP32 pairs (out_mode OZ_OUT_PAIRS)
    void *Rc64;                   // output as complex64 or complex128 (OZ_OUT_C64 / _C128)
    int in_mode;                  // base of the update: OZ_IN_B (bsign * B), OZ_IN_PAIRS, OZ_IN_ZERO
    int out_mode;                 // OZ_OUT_PAIRS, OZ_OUT_C64, OZ_OUT_C128
    int neg;                      // 0: out = base - A (x)_j X; 1: out = base + A (x)_j X
    float bsign;                  // +1 or -1
    const unsigned char *aimg;    // 6 digit images of [Re A^T | Im A^T] (B operand layout)
    int n, Kp, Np;                // mode size, K padded to 16, N = 2n padded to 16
    int mode1;                    // 1: first mode (tiles of 64 columns)
    int lboX, sboX;               // X digit images: K-adjacent / 8-row-group strides (bytes)
    int sboAd;                    // A digit images: 8-row-group stride (bytes)
    int ximg_bytes, aimg_bytes;   // bytes of one digit image
    int rstage_off;               // shared-memory offset of the epilogue's operand slots
    int tmem_cols;                // 4 accumulators of Np columns, power of two
    int eA;                       // |A entries| < 2^(eA - 1)
    int64_t L, R, tilesL;
    DevFlags *flags;
    const int *done;
};

enum { OZ_IN_PAIRS = 0, OZ_IN_B = 1, OZ_IN_ZERO = 2 };
enum { OZ_OUT_PAIRS = 0, OZ_OUT_C64 = 1, OZ_OUT_C128 = 2 };

#ifdef __CUDACC__
cudaError_t launch_resid_oz(const OzArgs &a, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_maxabs(const void *x, int64_t count, DevFlags *flags, int num_sms,
                          cudaStream_t st);
cudaError_t resid_oz_init_attrs();
cudaError_t launch_modeprod_tc(int epi, const TCArgs &a, int grid, size_t smem, cudaStream_t st);
cudaError_t modeprod_tc_init_attrs();
// warp-specialised TMA-fed variant (modeprod_tcw.cu); cudaErrorNotSupported
// when the pass does not qualify
cudaError_t launch_modeprod_tcw(int epi, const TCArgs &a, int num_sms, cudaStream_t st);
// FP32 pass over one mode with n <= FIB_NMAX, one thread per fibre (modeprod_fib.cu)
int fib_nx(int n);
cudaError_t launch_modeprod_fib(int in_kind, int out_kind, int epi, const MPArgs &a, int num_sms,
                                cudaStream_t st);
cudaError_t modeprod_tcw_init_attrs();
cudaError_t launch_modeprod(int fp64, int in_kind, int out_kind, int epi, const MPArgs &a,
                            size_t smem, cudaStream_t st);
cudaError_t launch_sweep(int fp64, const SweepArgs &a, int grid, int threads, size_t smem,
                         cudaStream_t st);
cudaError_t launch_sweep_init(const SweepArgs &a, cudaStream_t st);
cudaError_t launch_sweep_batch(int fp64, int real, const SweepBatch &b, int grid, int threads,
                               size_t smem, cudaStream_t st);
int sweep_batch_blocks_per_sm(int fp64, int threads, size_t smem, int real);
cudaError_t launch_inv_table(int fp64, const SweepArgs &a, void *tab, int num_sms,
                             cudaStream_t st);
cudaError_t launch_sweep_diag(int fp64, const DiagArgs &a, int num_sms, cudaStream_t st);
cudaError_t launch_solve_init(DevFlags *f, cudaStream_t st);
cudaError_t launch_refine_decide(DevFlags *f, float rtol, int step, int max_refine,
                                 cudaStream_t st);
cudaError_t launch_den_minmax(int Nm, const int64_t *n, const double *const *d, double sig_re,
                              double sig_im, int64_t ntot, unsigned long long *out3,
                              cudaStream_t st);
cudaError_t kernels_init(int device);
cudaError_t sweep_init_attrs();
int sweep_blocks_per_sm(int fp64, int threads, size_t smem, int real = 0);
// real-arithmetic mode products (float32 / float64 tensors, real matrices)
cudaError_t launch_modeprod_real(int fp64, int in_kind, int out_kind, int epi, const MPArgs &a,
                                 size_t smem, cudaStream_t st);
cudaError_t modeprod_real_init_attrs();
#endif

}  // namespace sylv
