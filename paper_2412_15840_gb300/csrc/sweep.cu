// Triangular sweep of the transformed system sum_j T_j (x)_j Y = C
// (Eq. (yi1i2iN), the second phase of Algorithm 3) on sm_103a.
//
// The entries are grouped in tiles: a box of b_j consecutive indices along
// every mode.  Eq. (yi1i2iN) makes entry i depend on the entries that differ
// from it in one mode and have a larger index there; at tile granularity,
// tile I therefore needs the tiles I + m e_j (m >= 1) along every mode, and
// waiting for the immediate successors I + e_j suffices (each of them waited
// for its own successors).  A persistent grid takes tiles in the order of
// their level sum_j (B_j - 1 - I_j) through an atomic ticket; before solving,
// a tile waits (bounded) until a per-tile counter of unfinished immediate
// successors reaches zero.  A CTA only ever waits on tiles with smaller
// tickets, which running CTAs hold, so no co-residency is needed.
//
// One tile, three stages:
//  1. load C, form the FP64 reciprocal of sigma + sum_j t_{j,i_j i_j} for
//     every entry (or read it from the plan's table) and the diagonal T blocks
//     -- the tile's own data, loaded before the dependency wait; subtract,
//     entry by entry, the strips of the modes outside the tile; then subtract
//     the contributions of the solved tiles along the in-tile modes, mode by
//     mode, as a small GEMM: T_j[rows of the block, later columns] times the
//     strip of solved values.  A fiber of the tile along mode j belongs to one
//     thread (or a few adjacent lanes), which loads every strip value once and
//     applies all b_j rows of the T block (staged in shared memory) to it.
//     Where the sweep is latency-bound, the columns beyond the immediate
//     successor block are applied first, as soon as each successor I + e_j is
//     ready to run (its own counter is zero, so every I + m e_j with m >= 2 is
//     solved), and the successor block after the full wait.
//  2. solve the tile in place, level by level of the in-tile index sum
//     measured from the tile's end: the in-tile part of Eq. (yi1i2iN), then
//     y = num * (1/den) with the reciprocal formed in FP64 in stage 1.
//  3. store Y (L2), fence, release the counters of the predecessor tiles.
// The real-arithmetic variant (RL) keeps C, Y and the strips real and rotates
// the tile's 2 x 2 blocks to complex triangular form around stage 2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "cplx.cuh"
#include "sweep_common.cuh"
#include "sylv_internal.h"

namespace sylv {

constexpr int SW_KCH = SWEEP_KCH;
constexpr int SW_RG = 8;     // fiber rows kept in registers at once
constexpr int SW_OUT = 128;  // strip entries of the modes outside the tile applied in stage 1a

// Real-arithmetic variant (RL): C, Y and the strips are real (YT = real), the
// tile itself is complex.  After the strips are subtracted, the tile's
// right-hand side is rotated into the basis of the complex triangular
// T~_j = V_j^* T_j V_j along every in-tile mode with 2 x 2 blocks (V_j unitary,
// block diagonal, one 2 x 2 factor per pair of indices), the in-tile wavefront
// runs with T~_j, and the result is rotated back by V_j; its real part is Y.
// This is exact for the quasi-triangular T_j because tiles never split a 2 x 2
// block (its indices 2u, 2u + 1 and even tile offsets).
__device__ __forceinline__ void cmsub(float &acc, float t, float y) { acc = fmaf(-t, y, acc); }
__device__ __forceinline__ void cmsub(double &acc, double t, double y) { acc = fma(-t, y, acc); }
__device__ __forceinline__ void shfl_add(float2 &v, int o) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
}
__device__ __forceinline__ void shfl_add(double2 &v, int o) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
}
__device__ __forceinline__ void shfl_add(float &v, int o) { v += __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ void shfl_add(double &v, int o) { v += __shfl_xor_sync(0xffffffffu, v, o); }
template <typename C2> __device__ __forceinline__ void add_to(C2 &v, C2 a) { v.x += a.x; v.y += a.y; }
__device__ __forceinline__ void add_to(float2 &v, float a) { v.x += a; }
__device__ __forceinline__ void add_to(double2 &v, double a) { v.x += a; }
template <typename C2> __device__ __forceinline__ C2 as_tile(C2 v) { return v; }
__device__ __forceinline__ float2 as_tile(float v) { return make_float2(v, 0.f); }
__device__ __forceinline__ double2 as_tile(double v) { return make_double2(v, 0.0); }
template <typename YT, typename C2> __device__ __forceinline__ YT from_tile(C2 v) {
    if constexpr (std::is_same<YT, C2>::value) return v;
    else return v.x;
}

// [x0; x1] <- V^* [x0; x1] (adj) or V [x0; x1] on the pairs (t, t + 1), t even,
// of every in-tile mode that has 2 x 2 blocks; V is column-major (v00, v10,
// v01, v11).  Entries outside a partial tile hold zeros and stay zero.
template <typename C2>
__device__ __forceinline__ void rotate_pairs(const SweepArgs &a, C2 *tile_s, const int *be,
                                             const int64_t *o, bool adj) {
    for (int q = 0; q < a.nin; ++q) {
        const int j = a.inmode[q];
        if (!a.Vp[j]) continue;
        const C2 *V = reinterpret_cast<const C2 *>(a.Vp[j]);
        const int bq = a.b[j], sq = a.BS[q], half = (bq + 1) / 2;
        const int npair = a.Pt / bq * half;
        const int64_t u0 = o[j] / 2;
        for (int idx = threadIdx.x; idx < npair; idx += blockDim.x) {
            const int lo = idx % sq;
            const int rest = idx / sq;
            const int u = rest % half;
            const int hi = rest / half;
            if (2 * u + 1 >= be[j]) continue;
            const int e0 = lo + sq * (2 * u) + hi * sq * bq;
            const C2 x0 = tile_s[e0], x1 = tile_s[e0 + sq];
            const C2 *v = V + 4 * (u0 + u);
            const C2 v00 = v[0], v10 = v[1], v01 = v[2], v11 = v[3];
            C2 y0, y1;
            if (adj) {      // conj(v00) x0 + conj(v10) x1, conj(v01) x0 + conj(v11) x1
                y0.x = v00.x * x0.x + v00.y * x0.y + v10.x * x1.x + v10.y * x1.y;
                y0.y = v00.x * x0.y - v00.y * x0.x + v10.x * x1.y - v10.y * x1.x;
                y1.x = v01.x * x0.x + v01.y * x0.y + v11.x * x1.x + v11.y * x1.y;
                y1.y = v01.x * x0.y - v01.y * x0.x + v11.x * x1.y - v11.y * x1.x;
            } else {        // v00 x0 + v01 x1, v10 x0 + v11 x1
                y0.x = v00.x * x0.x - v00.y * x0.y + v01.x * x1.x - v01.y * x1.y;
                y0.y = v00.x * x0.y + v00.y * x0.x + v01.x * x1.y + v01.y * x1.x;
                y1.x = v10.x * x0.x - v10.y * x0.y + v11.x * x1.x - v11.y * x1.y;
                y1.y = v10.x * x0.y + v10.y * x0.x + v11.x * x1.y + v11.y * x1.x;
            }
            tile_s[e0] = y0;
            tile_s[e0 + sq] = y1;
        }
        __syncthreads();
    }
}

// One group of RB rows of a fiber's strip update: acc[r] = -sum_c T[rg + r, c] y_c
// over `ncol` columns (y in L2 at yp + c*Sj, T staged in shared memory with row
// stride 1 and column stride bj), the H lanes of the fiber combined by
// shuffles, and lane 0 of them adding the first `rows` accumulators to the
// tile (rows <= RB; rows beyond `rows` read staged T entries of the next rows
// of the block or zero padding and are not written).
template <int RB, typename real, typename YT, typename C2>
__device__ __forceinline__ void strip_group(const YT *yp, int64_t Sj, const YT *tc, int bj,
                                            int ncol, int H, bool wr, C2 *dst, int bs, int rows) {
    constexpr int UNR = sizeof(real) == 4 ? 8 : 4;   // strip loads in flight per thread
    YT acc[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = YT{};
    int c = 0;
    for (; c + UNR <= ncol; c += UNR) {
        YT y[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) y[u] = __ldcg(yp + u * Sj);
        yp += UNR * Sj;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
#pragma unroll
            for (int u = 0; u < UNR; ++u) cmsub(acc[r], tc[u * bj + r], y[u]);
        }
        tc += UNR * bj;
    }
    for (; c < ncol; ++c) {
        const YT y = __ldcg(yp);
        yp += Sj;
#pragma unroll
        for (int r = 0; r < RB; ++r) cmsub(acc[r], tc[r], y);
        tc += bj;
    }
    for (int o = 1; o < H; o <<= 1) {
#pragma unroll
        for (int r = 0; r < RB; ++r) shfl_add(acc[r], o);
    }
    if (wr) {
#pragma unroll
        for (int r = 0; r < RB; ++r)
            if (r < rows) add_to(dst[r * bs], acc[r]);
    }
}

// FP64 complex rows by Gauss's three-multiplication product: with the staged
// plane s = re + im of the T block and sx = re + im of each strip value (one
// addition shared by the RB rows), sum_c T y = (sum tr yr - sum ti yi,
// sum s sx - sum tr yr - sum ti yi): three FP64 FMAs per term instead of four,
// on the FP64 pipe that bounds this sweep.
template <int RB>
__device__ __forceinline__ void strip_group3m(const double2 *yp, int64_t Sj, const double2 *tc,
                                              const double *ts, int bj, int ncol, int H, bool wr,
                                              double2 *dst, int bs, int rows) {
    constexpr int UNR = 4;
    double p1[RB], p2[RB], p3[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) p1[r] = p2[r] = p3[r] = 0.0;
    int c = 0;
    for (; c + UNR <= ncol; c += UNR) {
        double2 y[UNR];
        double sx[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) y[u] = __ldcg(yp + u * Sj);
#pragma unroll
        for (int u = 0; u < UNR; ++u) sx[u] = y[u].x + y[u].y;
        yp += UNR * Sj;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const double2 t = tc[u * bj + r];
                p1[r] = fma(t.x, y[u].x, p1[r]);
                p2[r] = fma(t.y, y[u].y, p2[r]);
                p3[r] = fma(ts[u * bj + r], sx[u], p3[r]);
            }
        }
        tc += UNR * bj;
        ts += UNR * bj;
    }
    for (; c < ncol; ++c) {
        const double2 y = __ldcg(yp);
        const double sx = y.x + y.y;
        yp += Sj;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            p1[r] = fma(tc[r].x, y.x, p1[r]);
            p2[r] = fma(tc[r].y, y.y, p2[r]);
            p3[r] = fma(ts[r], sx, p3[r]);
        }
        tc += bj;
        ts += bj;
    }
    double2 acc[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = make_double2(p2[r] - p1[r], (p1[r] + p2[r]) - p3[r]);
    for (int o = 1; o < H; o <<= 1) {
#pragma unroll
        for (int r = 0; r < RB; ++r) shfl_add(acc[r], o);
    }
    if (wr) {
#pragma unroll
        for (int r = 0; r < RB; ++r)
            if (r < rows) add_to(dst[r * bs], acc[r]);
    }
}

// Every tile of one equation: take tickets from the equation's own counter// Every tile of one equation: take tickets from the equation's own counter
// (a.flags->ticket) until they run out.  far_ok = 0 turns the far/near strip
// split off (a batch of equations keeps the GPU busy without it).
template <typename real, bool RL>
__device__ __forceinline__ void sweep_drain(const SweepArgs &a, const int far_ok) {
    using C2 = typename C2T<real>::type;
    using YT = typename std::conditional<RL, real, C2>::type;   // element of C and Y
    using Inv = typename InvT<real>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Inv *inv_s = reinterpret_cast<Inv *>(smem_raw);
    C2 *tile_s = reinterpret_cast<C2 *>(inv_s + a.Pt);
    YT *Ts = reinterpret_cast<YT *>(tile_s + a.Pt);   // SW_KCH x bmax block of T_j
    C2 *Td = tile_s + a.Pt + SW_KCH * a.bmax;         // diagonal blocks of the in-tile modes
    // packed in-tile coordinates and the level schedule of the full box, copied
    // once per CTA (every tile uses the same tables)
    unsigned long long *coord_s = reinterpret_cast<unsigned long long *>(Td + a.tdsize);
    int *sched_s = reinterpret_cast<int *>(coord_s + (a.fast ? a.Pt : 0));
    // element offsets of the box positions (full tiles skip the decode of the
    // packed coordinates)
    int *offs_s = sched_s + (a.fast ? a.Pt : 0);
    const bool offc = a.use_offs != 0;
    // FP64 complex strips: the plane re + im of the staged T block (8-byte aligned
    // after the offsets), present when the plan reserved it
    constexpr bool C3 = sizeof(real) == 8 && !RL;
    const bool G3 = C3 && a.g3;
    double *Tsum = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(offs_s + (offc ? a.Pt : 0)) + 7) & ~(uintptr_t)7);
    __shared__ int s_ticket, s_tile, s_abort, s_full, s_hasfar;
    __shared__ int64_t s_o[MAXM];
    __shared__ int s_be[MAXM], s_cnt[MAXM], s_I[MAXM];
    __shared__ int64_t s_gbase, s_rhs0;
    // modes outside the tile (b_j = 1): the (offset, T value) pairs of their
    // strips, applied entry by entry in stage 1a without extra barriers
    __shared__ int s_npair, s_inlist[MAXM], s_pbase[MAXM];
    // in-tile modes whose block is cut short in this tile (a partial tile's
    // entries are valid when their coordinate is below s_be along these only)
    __shared__ int s_npart, s_pq[MAXM];
    __shared__ int64_t s_pstride[SW_OUT];
    __shared__ YT s_pt[SW_OUT];
    __shared__ double s_den0x, s_den0y;

    if (*(volatile const int *)&a.flags->done) return;
    YT *Y = reinterpret_cast<YT *>(a.Y);
    const int Nm = a.Nm, nin = a.nin, nt = blockDim.x;
    if (a.fast) {
        for (int e = threadIdx.x; e < a.Pt; e += nt) {
            coord_s[e] = a.coord[e];
            sched_s[e] = a.sched_e[e];
            if (offc) offs_s[e] = a.offs[e];
        }
        // (the first __syncthreads of the tile loop orders these stores)
    }

    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(&a.flags->ticket, 1);
            s_ticket = t;
            s_abort = 0;
            if (t < a.ntiles) s_tile = a.order[t];
        }
        __syncthreads();
        if (s_ticket >= a.ntiles) break;
        const int tile = s_tile;

        // tile geometry
        if (threadIdx.x == 0) {
            // tile ids, tile strides and block counts are below 2^31 (plan check):
            // 32-bit divisions
            const unsigned ut = (unsigned)tile, un1 = (unsigned)a.ntiles1;
            const int64_t rhs = ut / un1;
            const unsigned rem = ut - (unsigned)rhs * un1;
            int64_t gb = rhs * a.ntot;
            double dx = a.sig_re, dy = a.sig_im;
            int full = 1;
            for (int j = 0; j < Nm; ++j) {
                const int Ij = (int)((rem / (unsigned)a.TS[j]) % (unsigned)a.Bc[j]);
                const int64_t o = (int64_t)Ij * a.b[j];
                int64_t be = a.n[j] - o;
                if (be > a.b[j]) be = a.b[j];
                else if (be < a.b[j]) full = 0;
                s_I[j] = Ij;
                s_o[j] = o;
                s_be[j] = (int)be;
                s_cnt[j] = (int)(a.n[j] - o - be);
                gb += o * a.S[j];
                if (a.b[j] == 1) {      // modes outside the tile: constant diagonal term
                    dx += a.d[j][2 * o];
                    dy += a.d[j][2 * o + 1];
                }
            }
            s_gbase = gb;
            s_rhs0 = rhs * a.ntot;
            s_den0x = dx;
            s_den0y = dy;
            s_full = full;
            int npq = 0;
            for (int q = 0; q < nin; ++q)
                if (s_be[a.inmode[q]] < a.b[a.inmode[q]]) s_pq[npq++] = q;
            s_npart = npq;
            int np = 0;
            for (int j = 0; j < Nm; ++j) {
                s_inlist[j] = 0;
                const int K = s_cnt[j];
                if (a.qpos[j] >= 0 || K == 0 || np + K > SW_OUT) continue;
                s_inlist[j] = 1;
                s_pbase[j] = np;
                np += K;
            }
            s_npair = np;
            // columns beyond the immediate successor block in some mode
            int hf = 0;
            for (int j = 0; j < Nm; ++j)
                if (!s_inlist[j] && s_cnt[j] > (a.qpos[j] >= 0 ? a.b[j] : 1)) hf = 1;
            s_hasfar = hf;
        }
        __syncthreads();
        const int64_t gbase = s_gbase;
        // packed coordinates serve every tile; a partial tile (be_j < b_j for some
        // in-tile mode) skips the box offsets outside its valid extents
        const bool fastc = a.fast != 0, partial = s_full == 0;
        // packed coordinates c of a box position inside this partial tile's extents
        auto inside = [&](unsigned long long c) {
            for (int k = 0; k < s_npart; ++k) {
                const int q = s_pq[k];
                if ((int)((c >> a.cshift[q]) & a.cmask[q]) >= s_be[a.inmode[q]]) return false;
            }
            return true;
        };
        const int npair = s_npair;
        if (npair > 0) {
            for (int j = 0; j < Nm; ++j) {
                if (!s_inlist[j]) continue;
                const int K = s_cnt[j], base = s_pbase[j];
                const int64_t nj = a.n[j], oj = s_o[j];
                const YT *Tj = reinterpret_cast<const YT *>(RL ? a.Tr[j] : a.T[j]);
                for (int k = threadIdx.x; k < K; k += nt) {
                    s_pstride[base + k] = (int64_t)(1 + k) * a.S[j];
                    s_pt[base + k] = __ldg(Tj + oj + (oj + 1 + k) * nj);
                }
            }
            __syncthreads();
        }

        // stage 1a: C, the FP64 reciprocals of the diagonal sums and the diagonal
        // T blocks -- this tile's own data, loaded before the wait for its
        // successors so that the loads overlap it
        for (int e = threadIdx.x; e < a.Pt; e += nt) {
            int64_t g = gbase;
            bool ok = true;
            double ex = s_den0x, ey = s_den0y;
            if (offc && a.inv_tab) {
                ok = !partial || inside(coord_s[e]);
                g += offs_s[e];
            } else if (fastc) {
                const unsigned long long c = coord_s[e];
                for (int q = 0; q < nin; ++q) {
                    const int j = a.inmode[q];
                    const int t = (int)((c >> a.cshift[q]) & a.cmask[q]);
                    if (partial && t >= s_be[j]) { ok = false; break; }
                    g += (int64_t)t * a.S[j];
                    if (!a.inv_tab) {
                        const int64_t ij = s_o[j] + t;
                        ex += a.d[j][2 * ij];
                        ey += a.d[j][2 * ij + 1];
                    }
                }
            } else {
                int r = e;
                for (int q = 0; q < nin; ++q) {
                    const int j = a.inmode[q];
                    const int bj = a.b[j];
                    const int t = r % bj;
                    r /= bj;
                    if (t >= s_be[j]) { ok = false; break; }
                    g += (int64_t)t * a.S[j];
                    const int64_t ij = s_o[j] + t;
                    ex += a.d[j][2 * ij];
                    ey += a.d[j][2 * ij + 1];
                }
            }
            if (!ok) {
                tile_s[e] = czero<C2>();
                continue;
            }
            tile_s[e] = as_tile(__ldcg(Y + g));
            if (a.inv_tab)       // reciprocals formed once per plan (k_inv_table)
                inv_s[e] = __ldg(reinterpret_cast<const Inv *>(a.inv_tab) + (g - s_rhs0));
            else
                store_inv(crecip_scaled(ex, ey, a.den_scale), inv_s[e]);
        }
        // diagonal blocks T_j[o_j + r, o_j + c] (r < c < be_j) of the in-tile modes
        for (int p = 0; p < nin; ++p) {
            const int j = a.inmode[p];
            const int bj = a.b[j], be = s_be[j];
            const int64_t nj = a.n[j], oj = s_o[j];
            const C2 *Tj = reinterpret_cast<const C2 *>(a.T[j]);
            C2 *dst = Td + a.tdoff[p];
            for (int idx = threadIdx.x; idx < be * be; idx += nt) {
                const int r = idx % be, c = idx / be;
                dst[r + c * bj] = __ldg(Tj + (oj + r) + (oj + c) * nj);
            }
        }

        // stage 1b: contributions of the solved tiles, mode by mode, over the columns
        // of the immediate successor block (near) or beyond it (far)
        // part 0: all columns; 1: beyond the immediate successor block; 2: that block
        auto strips = [&](int part) {
        for (int j = 0; j < Nm; ++j) {
            const int K = s_cnt[j];
            if (K == 0 || s_inlist[j]) continue;
            const int q = a.qpos[j];
            const int bj = q >= 0 ? a.b[j] : 1;     // box extent along mode j
            const int bej = s_be[j];                // valid rows of the block
            const int bs = q >= 0 ? a.BS[q] : 1;
            const int F = a.Pt / bj;                // fibers of the box along mode j
            const int64_t nj = a.n[j], Sj = a.S[j], oj = s_o[j];
            const int64_t kend = oj + bej;
            const YT *Tj = reinterpret_cast<const YT *>(RL ? a.Tr[j] : a.T[j]);
            const int nb = min(bj, K);              // columns of the immediate successor
            const int cb = part == 1 ? nb : 0, ce = part == 2 ? nb : K;
            for (int k0 = cb; k0 < ce; k0 += SW_KCH) {
                const int kk = min(SW_KCH, ce - k0);
                for (int idx = threadIdx.x; idx < bej * kk; idx += nt) {
                    const int r = idx % bej, c = idx / bej;
                    const YT t = __ldg(Tj + (oj + r) + (kend + k0 + c) * nj);
                    Ts[c * bj + r] = t;
                    if constexpr (C3)
                        if (G3) Tsum[c * bj + r] = t.x + t.y;
                }
                __syncthreads();
                // H consecutive lanes share a fiber when the box has fewer fibers
                // than threads (FP32 path): each sums a contiguous share of the
                // columns, and the partial sums meet by shuffles (fixed order)
                int H = 1;
                if (sizeof(real) == 4)
                    while (2 * H <= 8 && 2 * H * F <= nt) H *= 2;    // a power of two
                const int per = (kk + H - 1) / H;
                const int h = (int)threadIdx.x % H;
                for (int fb = 0; fb < F; fb += nt / H) {
                    const int f = fb + (int)threadIdx.x / H;
                    const int e0 = (q >= 0) ? (f / bs) * (bs * bj) + (f % bs) : f;
                    int64_t g0 = gbase;
                    bool ok = f < F;
                    if (ok && offc) {
                        ok = !partial || inside(coord_s[e0]);
                        g0 += offs_s[e0];
                    } else if (ok && fastc) {
                        const unsigned long long c = coord_s[e0];
                        for (int p = 0; p < nin; ++p) {
                            const int t = (int)((c >> a.cshift[p]) & a.cmask[p]);
                            if (partial && t >= s_be[a.inmode[p]]) { ok = false; break; }
                            g0 += (int64_t)t * a.S[a.inmode[p]];
                        }
                    } else if (ok) {
                        int r = e0;
                        for (int p = 0; p < nin; ++p) {
                            const int jj = a.inmode[p];
                            const int b = a.b[jj];
                            const int t = r % b;
                            r /= b;
                            if (t >= s_be[jj]) { ok = false; break; }
                            g0 += (int64_t)t * a.S[jj];
                        }
                    }
                    const int c0 = min(kk, h * per), c1 = ok ? min(kk, c0 + per) : c0;
                    const YT *ybase = Y + g0 + (kend + k0 - oj + c0) * Sj;
                    const int ncol = c1 - c0;
                    for (int rg = 0; rg < bej; rg += SW_RG) {
                        // rows of this group: 1, 2, 4 or 8 accumulators, so that a
                        // block of b_j = 1, 2, 4 rows issues no idle row's FMAs
                        const int rows = min(SW_RG, bej - rg);
                        const YT *tc = Ts + rg + c0 * bj;
                        C2 *dst = tile_s + e0 + rg * bs;
                        const bool wr = ok && h == 0;
                        // FP64 complex with the re + im plane: up to four rows by three
                        // multiplications (eight rows of three sums exceed the registers)
                        bool done = false;
                        if constexpr (C3) {
                            if (G3 && rows <= 4) {
                                const double *tsp = Tsum + rg + c0 * bj;
                                if (rows == 1)
                                    strip_group3m<1>(ybase, Sj, tc, tsp, bj, ncol, H, wr, dst, bs, rows);
                                else if (rows == 2)
                                    strip_group3m<2>(ybase, Sj, tc, tsp, bj, ncol, H, wr, dst, bs, rows);
                                else
                                    strip_group3m<4>(ybase, Sj, tc, tsp, bj, ncol, H, wr, dst, bs, rows);
                                done = true;
                            }
                        }
                        if (done) continue;
                        if (rows == 1)
                            strip_group<1, real>(ybase, Sj, tc, bj, ncol, H, wr, dst, bs, rows);
                        else if (rows == 2)
                            strip_group<2, real>(ybase, Sj, tc, bj, ncol, H, wr, dst, bs, rows);
                        else if (rows <= 4)
                            strip_group<4, real>(ybase, Sj, tc, bj, ncol, H, wr, dst, bs, rows);
                        else
                            strip_group<8, real>(ybase, Sj, tc, bj, ncol, H, wr, dst, bs, rows);
                    }
                }
                __syncthreads();
            }
        }
        };

        // wait (bounded) until every immediate successor I + e_j whose mode has
        // columns beyond it is ready to run: its counter is zero once all of its
        // own successors are solved, among them I + m e_j for every m >= 2, so the
        // far strips can be applied while the successors themselves still run.
        // Only when the sweep is latency-bound (few tiles per level for the
        // resident CTAs): otherwise the extra staging passes cost throughput.
        const bool split = far_ok && a.far_split && s_hasfar;
        if (split) {
        if (threadIdx.x == 0) {
            volatile int *err = &a.flags->err;
            for (int j = 0; j < Nm && !s_abort; ++j) {
                const int K = s_cnt[j];
                if (K == 0 || s_inlist[j]) continue;
                if (K <= (a.qpos[j] >= 0 ? a.b[j] : 1)) continue;
                volatile int *c = a.cnt + tile + a.TS[j];
                const long long t0 = clock64();
                while (*c > 0) {
                    if (*err) { s_abort = 1; break; }
                    if (clock64() - t0 > a.timeout_cycles) {
                        atomicOr(&a.flags->err, ERRBIT_TIMEOUT);
                        s_abort = 1;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            __threadfence();
        }
        __syncthreads();
        if (s_abort) {
            // drain: mark this tile finished so that nothing waits on it
            if (threadIdx.x == 0) {
                const int64_t rem = tile % a.ntiles1;
                for (int j = 0; j < Nm; ++j) {
                    const int Ij = (int)((rem / a.TS[j]) % a.Bc[j]);
                    if (Ij > 0) atomicSub(a.cnt + tile - a.TS[j], 1);
                }
            }
            __syncthreads();
            continue;
        }
        strips(1);
        }

        // wait (bounded) until every immediate successor tile is solved
        if (threadIdx.x == 0) {
            volatile int *c = a.cnt + tile;
            volatile int *err = &a.flags->err;
            const long long t0 = clock64();
            while (*c > 0) {
                if (*err) { s_abort = 1; break; }
                if (clock64() - t0 > a.timeout_cycles) {
                    atomicOr(&a.flags->err, ERRBIT_TIMEOUT);
                    s_abort = 1;
                    break;
                }
                __nanosleep(100);
            }
            __threadfence();
        }
        __syncthreads();
        if (s_abort) {
            // drain: mark this tile finished so that nothing waits on it
            if (threadIdx.x == 0) {
                const int64_t rem = tile % a.ntiles1;
                for (int j = 0; j < Nm; ++j) {
                    const int Ij = (int)((rem / a.TS[j]) % a.Bc[j]);
                    if (Ij > 0) atomicSub(a.cnt + tile - a.TS[j], 1);
                }
            }
            __syncthreads();
            continue;
        }

        // stage 1a': strips of the modes outside the tile (solved tiles), entry
        // by entry
        if (npair > 0) {
            for (int e = threadIdx.x; e < a.Pt; e += nt) {
                int64_t g = gbase;
                bool ok = true;
                if (offc) {
                    ok = !partial || inside(coord_s[e]);
                    g += offs_s[e];
                } else if (fastc) {
                    const unsigned long long c = coord_s[e];
                    for (int q = 0; q < nin; ++q) {
                        const int t = (int)((c >> a.cshift[q]) & a.cmask[q]);
                        if (partial && t >= s_be[a.inmode[q]]) { ok = false; break; }
                        g += (int64_t)t * a.S[a.inmode[q]];
                    }
                } else {
                    int r = e;
                    for (int q = 0; q < nin; ++q) {
                        const int j = a.inmode[q];
                        const int t = r % a.b[j];
                        r /= a.b[j];
                        if (t >= s_be[j]) { ok = false; break; }
                        g += (int64_t)t * a.S[j];
                    }
                }
                if (!ok) continue;
                YT acc{};
                for (int p0 = 0; p0 < npair; p0 += 4) {        // 4 strip loads in flight
                    YT y[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (p0 + u < npair) y[u] = __ldcg(Y + g + s_pstride[p0 + u]);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (p0 + u < npair) cmsub(acc, s_pt[p0 + u], y[u]);
                }
                add_to(tile_s[e], acc);
            }
            __syncthreads();
        }

        strips(split ? 2 : 0);

        if constexpr (RL) rotate_pairs(a, tile_s, s_be, s_o, true);

        // stage 2: in-tile wavefront over index sums measured from the tile's end.
        // SW_SUB consecutive lanes share an entry (a.sub: 4 where the sweep is
        // latency-bound, else 1, which issues fewer instructions): lane `sub`
        // sums the in-tile successors along in-tile modes sub, sub + SW_SUB, ...;
        // the partial sums are combined with shuffles and lane 0 of the group
        // divides.
        const int SW_LG = a.fast ? (a.sub >= 4 ? 2 : a.sub >= 2 ? 1 : 0) : 0;
        const int SW_SUB = 1 << SW_LG;
        for (int lev = 0; lev < a.Lin; ++lev) {
            const int q0 = a.lev_start[lev], q1 = a.lev_start[lev + 1];
            for (int base = q0; base < q1; base += nt >> SW_LG) {
                const int qq = base + ((int)threadIdx.x >> SW_LG);
                const int sub = (int)threadIdx.x & (SW_SUB - 1);
                bool act = qq < q1;
                int e = 0;
                unsigned long long c = 0;
                if (act) {
                    if (fastc) {
                        e = sched_s[qq];
                        c = coord_s[e];
                        if (partial && !inside(c)) act = false;
                    } else {
                        int r = a.sched[qq];
                        for (int p = 0; p < nin; ++p) {
                            const int j = a.inmode[p];
                            const int bj = a.b[j];
                            const int apj = r % bj;
                            r /= bj;
                            if (apj >= s_be[j]) { act = false; break; }
                            e += (s_be[j] - 1 - apj) * a.BS[p];
                        }
                    }
                }
                C2 part = czero<C2>();
                if (act) {
                    for (int p = sub; p < nin; p += SW_SUB) {
                        const int j = a.inmode[p];
                        const int bs = a.BS[p];
                        const int t = fastc ? (int)((c >> a.cshift[p]) & a.cmask[p])
                                            : (e / bs) % a.b[j];
                        const int be = s_be[j];
                        if (t + 1 >= be) continue;
                        const int bj = a.b[j];
                        const C2 *tp = Td + a.tdoff[p] + t + (t + 1) * bj;
                        const C2 *yp = tile_s + e + bs;
                        for (int tt = t + 1; tt < be; ++tt) {     // in-tile successors
                            cmsub(part, *tp, *yp);
                            tp += bj;
                            yp += bs;
                        }
                    }
                }
                for (int o = 1; o < SW_SUB; o <<= 1) {
                    part.x += __shfl_xor_sync(0xffffffffu, part.x, o);
                    part.y += __shfl_xor_sync(0xffffffffu, part.y, o);
                }
                if (act && sub == 0) {
                    C2 num = tile_s[e];
                    num.x += part.x;
                    num.y += part.y;
                    tile_s[e] = apply_inv(num, inv_s[e]);
                }
            }
            __syncthreads();
        }

        if constexpr (RL) rotate_pairs(a, tile_s, s_be, s_o, false);

        // stage 3: store Y and release the tiles that wait on this one
        for (int e = threadIdx.x; e < a.Pt; e += nt) {
            int64_t g = gbase;
            bool ok = true;
            if (offc) {
                ok = !partial || inside(coord_s[e]);
                g += offs_s[e];
            } else if (fastc) {
                const unsigned long long c = coord_s[e];
                for (int p = 0; p < nin; ++p) {
                    const int t = (int)((c >> a.cshift[p]) & a.cmask[p]);
                    if (partial && t >= s_be[a.inmode[p]]) { ok = false; break; }
                    g += (int64_t)t * a.S[a.inmode[p]];
                }
            } else {
                int r = e;
                for (int p = 0; p < nin; ++p) {
                    const int j = a.inmode[p];
                    const int bj = a.b[j];
                    const int t = r % bj;
                    r /= bj;
                    if (t >= s_be[j]) { ok = false; break; }
                    g += (int64_t)t * a.S[j];
                }
            }
            if (ok) __stcg(Y + g, from_tile<YT>(tile_s[e]));
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0 && tile != a.fault_tile) {
            for (int j = 0; j < Nm; ++j)
                if (s_I[j] > 0) atomicSub(a.cnt + tile - a.TS[j], 1);
        }
    }
}

template <typename real, bool RL>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 4 : 3) k_sweep(const __grid_constant__ SweepArgs a) {
    sweep_drain<real, RL>(a, 1);
}

// Batched sweep (many independent equations, one persistent launch): every
// equation keeps its own ticket counter, level-ordered tile list and tile
// counters, so a CTA waits only on tiles of the same equation with smaller
// tickets, which running CTAs hold -- the single-equation argument, whatever
// order the CTAs visit the equations in.  A CTA starts at the equation that
// its share of the summed tile count falls in, drains it, and moves on to the
// first equation after it (cyclically) that still has tickets left; an
// equation's arguments are staged in shared memory while the CTA works on it.
template <typename real, bool RL>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 4 : 3) k_sweep_batch(const __grid_constant__ SweepBatch bt) {
    __shared__ __align__(16) SweepArgs sa;
    __shared__ int s_next;
    const int neq = bt.neq;
    const long long target = (long long)blockIdx.x * bt.cum[neq] / gridDim.x;
    int lo = 0, hi = neq - 1;           // the equation whose tile range holds `target`
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (bt.cum[mid] <= target) lo = mid;
        else hi = mid - 1;
    }
    constexpr int WORDS = (int)(sizeof(SweepArgs) / sizeof(int));
    int cur = lo;
    for (;;) {
        // the first equation from `cur` on (cyclically) that is not finished and
        // has tickets left, all threads looking at one equation each
        __syncthreads();                // the previous equation's readers are done
        if (threadIdx.x == 0) s_next = neq;
        __syncthreads();
        for (int k = threadIdx.x; k < neq; k += blockDim.x) {
            int e = cur + k;
            if (e >= neq) e -= neq;
            const volatile DevFlags *f = bt.flags[e];
            if (!f->done && (long long)f->ticket < bt.cum[e + 1] - bt.cum[e]) atomicMin(&s_next, k);
        }
        __syncthreads();
        if (s_next >= neq) break;
        int e = cur + s_next;
        if (e >= neq) e -= neq;
        cur = e;
        const int *src = reinterpret_cast<const int *>(bt.sa[e]);
        int *dst = reinterpret_cast<int *>(&sa);
        for (int w = threadIdx.x; w < WORDS; w += blockDim.x) dst[w] = __ldg(src + w);
        __syncthreads();
        if (threadIdx.x == 0) {
            sa.Y = bt.Y[e];
            sa.cnt = bt.cnt[e];
            sa.flags = bt.flags[e];
        }
        __syncthreads();
        sweep_drain<real, RL>(sa, bt.far_split);
    }
}

// Tile counters and ticket of every equation of a batched sweep.
__global__ void k_sweep_init_batch(const __grid_constant__ SweepBatch bt) {
    const int64_t total = bt.cum[bt.neq];
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = bt.neq - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (bt.cum[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const SweepArgs *a = bt.sa[lo];
        const int64_t tile = g - bt.cum[lo];
        if (tile == 0) bt.flags[lo]->ticket = 0;
        const int64_t rem = tile % a->ntiles1;
        int c = 0;
        for (int j = 0; j < a->Nm; ++j) {
            const int Ij = (int)((rem / a->TS[j]) % a->Bc[j]);
            c += (Ij < a->Bc[j] - 1);
        }
        bt.cnt[lo][tile] = c;
    }
}

__global__ void k_sweep_init(const __grid_constant__ SweepArgs a) {
    if (blockIdx.x == 0 && threadIdx.x == 0) a.flags->ticket = 0;
    for (int64_t tile = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tile < a.ntiles;
         tile += (int64_t)gridDim.x * blockDim.x) {
        const int64_t rem = tile % a.ntiles1;
        int c = 0;
        for (int j = 0; j < a.Nm; ++j) {
            const int Ij = (int)((rem / a.TS[j]) % a.Bc[j]);
            c += (Ij < a.Bc[j] - 1);
        }
        a.cnt[tile] = c;
    }
}

// Reciprocals 1 / (sigma + sum_j t_{j,i_j i_j}) of every multi-index, formed in
// FP64 once per plan and stored in the sweep's format (double2 on the FP64
// path, the FP32 pair hi/lo on the FP32 path); the sweep then reads them
// instead of spending FP64 instructions on its critical path.
template <typename real>
__global__ void k_inv_table(const __grid_constant__ SweepArgs a, void *tab) {
    using Inv = typename InvT<real>::type;
    Inv *out = reinterpret_cast<Inv *>(tab);
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < a.ntot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        double dx = a.sig_re, dy = a.sig_im;
        int64_t rem = idx;
        for (int j = 0; j < a.Nm; ++j) {
            const int64_t i = rem % a.n[j];
            rem /= a.n[j];
            dx += a.d[j][2 * i];
            dy += a.d[j][2 * i + 1];
        }
        Inv v;
        store_inv(crecip_scaled(dx, dy, a.den_scale), v);
        out[idx] = v;
    }
}

cudaError_t launch_inv_table(int fp64, const SweepArgs &a, void *tab, int num_sms,
                             cudaStream_t st) {
    if (a.ntot <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((a.ntot + 255) / 256, (int64_t)num_sms * 16);
    if (fp64)
        k_inv_table<double><<<(unsigned)blocks, 256, 0, st>>>(a, tab);
    else
        k_inv_table<float><<<(unsigned)blocks, 256, 0, st>>>(a, tab);
    return cudaGetLastError();
}

cudaError_t launch_sweep(int fp64, const SweepArgs &a, int grid, int threads, size_t smem,
                         cudaStream_t st) {
    if (a.ntiles <= 0) return cudaSuccess;
    if (a.real) {
        if (fp64)
            k_sweep<double, true><<<grid, threads, smem, st>>>(a);
        else
            k_sweep<float, true><<<grid, threads, smem, st>>>(a);
    } else if (fp64) {
        k_sweep<double, false><<<grid, threads, smem, st>>>(a);
    } else {
        k_sweep<float, false><<<grid, threads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_sweep_batch(int fp64, int real, const SweepBatch &b, int grid, int threads,
                               size_t smem, cudaStream_t st) {
    if (b.neq <= 0 || b.cum[b.neq] <= 0) return cudaSuccess;
    int64_t blocks = (b.cum[b.neq] + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_sweep_init_batch<<<(unsigned)blocks, 256, 0, st>>>(b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (real) {
        if (fp64)
            k_sweep_batch<double, true><<<grid, threads, smem, st>>>(b);
        else
            k_sweep_batch<float, true><<<grid, threads, smem, st>>>(b);
    } else if (fp64) {
        k_sweep_batch<double, false><<<grid, threads, smem, st>>>(b);
    } else {
        k_sweep_batch<float, false><<<grid, threads, smem, st>>>(b);
    }
    return cudaGetLastError();
}

int sweep_batch_blocks_per_sm(int fp64, int threads, size_t smem, int real) {
    int nb = 0;
    cudaError_t e;
    if (real)
        e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep_batch<double, true>,
                                                                 threads, smem)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep_batch<float, true>,
                                                                 threads, smem);
    else
        e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep_batch<double, false>,
                                                                 threads, smem)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep_batch<float, false>,
                                                                 threads, smem);
    return e == cudaSuccess ? nb : 0;
}

cudaError_t launch_sweep_init(const SweepArgs &a, cudaStream_t st) {
    int64_t blocks = (a.ntiles + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    k_sweep_init<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ----------------------------------------------------- diagonal sweep --
// Remark 1: with every T_j diagonal the sweep has no dependencies and is the
// entrywise (Hadamard) division y = c / (sigma + sum_j t_{j,i_j i_j}) of
// Eq. (yi1i2iNdiag).  One pass over the tensor, HBM-bound: each block takes
// DIAG_CHUNK consecutive entries (8 per thread, loads issued together), the
// tail sums of the columns it touches are decoded once into shared memory,
// and the head sums come from the plan's table.  The sum and its reciprocal
// are FP64; the FP32 path multiplies in FP64 and rounds once.
constexpr int DIAG_THREADS = 256;
constexpr int DIAG_PER = 8;
constexpr int DIAG_CHUNK = DIAG_THREADS * DIAG_PER;
constexpr int DIAG_MAXCOL = DIAG_CHUNK / 2 + 2;   // head product >= 2

template <typename real>
__global__ void __launch_bounds__(DIAG_THREADS) k_sweep_diag(const __grid_constant__ DiagArgs a) {
    using C2 = typename C2T<real>::type;
    if (*(volatile const int *)&a.flags->done) return;
    __shared__ double2 dt[DIAG_MAXCOL];
    C2 *Y = reinterpret_cast<C2 *>(a.Y);
    const double2 *dh = reinterpret_cast<const double2 *>(a.dhead);
    const int P1 = (int)a.P1;
    for (int64_t start = (int64_t)blockIdx.x * DIAG_CHUNK; start < a.total;
         start += (int64_t)gridDim.x * DIAG_CHUNK) {
        const int64_t end = min(start + (int64_t)DIAG_CHUNK, a.total);
        const int64_t q0 = start / P1;
        const int ncol = (int)((end - 1) / P1 - q0) + 1;
        for (int c = threadIdx.x; c < ncol; c += DIAG_THREADS) {
            int64_t q = (q0 + c) % a.Qt;
            double x = 0.0, y = 0.0;
            for (int m = 0; m < a.Nt; ++m) {
                const int64_t i = q % a.tn[m];
                q /= a.tn[m];
                x += a.td[m][2 * i];
                y += a.td[m][2 * i + 1];
            }
            dt[c] = make_double2(x, y);
        }
        __syncthreads();
        const int p0 = (int)(start - q0 * P1);
        C2 v[DIAG_PER];
#pragma unroll
        for (int k = 0; k < DIAG_PER; ++k) {
            const int64_t e = start + threadIdx.x + k * DIAG_THREADS;
            if (e < end) v[k] = __ldcs(Y + e);
        }
#pragma unroll
        for (int k = 0; k < DIAG_PER; ++k) {
            const int64_t e = start + threadIdx.x + k * DIAG_THREADS;
            if (e < end) {
                const int off = p0 + threadIdx.x + k * DIAG_THREADS;
                const int c = off / P1;
                const double2 h = __ldg(dh + (off - c * P1));
                const double2 inv = crecip_scaled(h.x + dt[c].x, h.y + dt[c].y, a.den_scale);
                const double2 cv = to_c(v[k], 0.0);
                double2 r;
                r.x = fma(cv.x, inv.x, -cv.y * inv.y);
                r.y = fma(cv.x, inv.y, cv.y * inv.x);
                __stcs(Y + e, to_c(r, real(0)));
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_sweep_diag(int fp64, const DiagArgs &a, int num_sms, cudaStream_t st) {
    if (a.total <= 0) return cudaSuccess;
    if (a.P1 < 2 || a.P1 > DIAG_HEAD_MAX) return cudaErrorInvalidValue;
    const int64_t chunks = (a.total + DIAG_CHUNK - 1) / DIAG_CHUNK;
    const int grid = (int)std::min<int64_t>(chunks, (int64_t)num_sms * 8);
    if (fp64)
        k_sweep_diag<double><<<grid, DIAG_THREADS, 0, st>>>(a);
    else
        k_sweep_diag<float><<<grid, DIAG_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

int sweep_blocks_per_sm(int fp64, int threads, size_t smem, int real) {
    int nb = 0;
    cudaError_t e;
    if (real)
        e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<double, true>,
                                                                 threads, smem)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<float, true>,
                                                                 threads, smem);
    else
        e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<double, false>,
                                                                 threads, smem)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<float, false>,
                                                                 threads, smem);
    return e == cudaSuccess ? nb : 0;
}

cudaError_t sweep_init_attrs() {
    const int big = 200 * 1024;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_sweep<double, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_sweep<float, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_sweep<double, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_sweep<float, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_sweep_batch<double, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_sweep_batch<float, false>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_sweep_batch<double, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_sweep_batch<float, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

}  // namespace sylv
