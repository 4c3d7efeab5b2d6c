// sm_103a kernels of the N-dimensional Bartels-Stewart solver (the sweep of
// Eq. (yi1i2iN) lives in sweep.cu).
//
//  k_modeprod  one transform pass: the mode-j products of Eq. (CUNU2U1B) /
//              Eq. (XUNU2U1Y) for a group of adjacent modes, applied to a
//              tile staged in shared memory; epilogues fuse the FP64 residual
//              R = B - sum_j A_j (x)_j X, the refinement update X += D, and
//              the subtraction of B that ends Eq. (C) of Theorem 1.
//  small       control kernels (flags, refinement decision, the plan-time
//              scan of the diagonal sums t_{1,i1i1}+...+t_{N,iNiN}).
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "cplx.cuh"
#include "sylv_internal.h"

namespace sylv {

// ---------------------------------------------------------------------------
// Transform pass
// ---------------------------------------------------------------------------

// tile entries loaded per thread before they are stored to shared memory
// (independent loads in flight hide the HBM latency of the staging)
constexpr int STAGE_U = 8;

// two consecutive complex entries of a column-major matrix (16-byte aligned
// when the first index is even)
__device__ __forceinline__ void ldg_pair(const float2 *p, float2 &u, float2 &v) {
    float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    u = make_float2(q.x, q.y);
    v = make_float2(q.z, q.w);
}
__device__ __forceinline__ void ldg_pair(const double2 *p, double2 &u, double2 &v) {
    u = __ldg(p);
    v = __ldg(p + 1);
}

// Rows i0 .. i0+RB-1 of one column of M (x) src along a mode with nm rows at
// stride `inner` in the tile; work item w enumerates (column, row group).
// Returns the tile offset of row i0 (row i0+r is at +r*inner).
template <int RB, typename C2>
__device__ __forceinline__ int mode_rows(const C2 *__restrict__ src, const C2 *__restrict__ M,
                                         int nm, int inner, int w, C2 *acc) {
    const int aa = w % inner;
    const int rest = w / inner;
    const int ng = nm / RB;
    const int ig = rest % ng;
    const int bb = rest / ng;
    const int i0 = ig * RB;
    const C2 *col = src + aa + bb * inner * nm;
    C2 c[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) c[r] = czero<C2>();
    const C2 *mk = M + i0;
    for (int k = 0; k < nm; ++k) {
        const C2 x = col[k * inner];
        if (RB == 1) {
            cmac(c[0], __ldg(mk), x);
        } else {
#pragma unroll
            for (int r = 0; r < RB; r += 2) {
                C2 m0, m1;
                ldg_pair(mk + r, m0, m1);
                cmac(c[r], m0, x);
                cmac(c[r + 1], m1, x);
            }
        }
        mk += nm;
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = c[r];
    return aa + inner * (i0 + nm * bb);
}
// FP64 variant of mode_rows by Gauss's three-multiplication complex product:
// with s = re + im of the matrix entry (the plane stored after the matrix) and
// sx = xr + xi (one addition per loaded entry, shared by the RB rows),
//   re = sum mr xr - sum mi xi,  im = sum s sx - sum mr xr - sum mi xi,
// three FP64 FMAs per (i, k) instead of four.
template <int RB>
__device__ __forceinline__ int mode_rows_3m(const double2 *__restrict__ src,
                                            const double2 *__restrict__ M, int nm, int inner,
                                            int w, double2 *acc) {
    const int aa = w % inner;
    const int rest = w / inner;
    const int ng = nm / RB;
    const int ig = rest % ng;
    const int bb = rest / ng;
    const int i0 = ig * RB;
    const double2 *col = src + aa + bb * inner * nm;
    const double *MS = reinterpret_cast<const double *>(M + nm * nm);
    double p1[RB], p2[RB], p3[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) p1[r] = p2[r] = p3[r] = 0.0;
    const double2 *mk = M + i0;
    const double *sk = MS + i0;
    for (int k = 0; k < nm; ++k) {
        const double2 x = col[k * inner];
        const double sx = x.x + x.y;
        double2 m[RB];
        double s[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) m[r] = __ldg(mk + r);
        if (RB == 1) {
            s[0] = __ldg(sk);
        } else {
#pragma unroll
            for (int r = 0; r < RB; r += 2) {
                const double2 q = __ldg(reinterpret_cast<const double2 *>(sk + r));
                s[r] = q.x;
                s[r + 1] = q.y;
            }
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            p1[r] = fma(m[r].x, x.x, p1[r]);
            p2[r] = fma(m[r].y, x.y, p2[r]);
            p3[r] = fma(s[r], sx, p3[r]);
        }
        mk += nm;
        sk += nm;
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = make_double2(p1[r] - p2[r], (p3[r] - p1[r]) - p2[r]);
    return aa + inner * (i0 + nm * bb);
}

template <typename real, typename Tin, typename Tout, int EPI>
__global__ void __launch_bounds__(256) k_modeprod(const __grid_constant__ MPArgs a) {
    using C2 = typename C2T<real>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.done && *(volatile const int *)a.done) return;

    const int Lt = a.Lt, Rt = a.Rt;
    const int P = (int)a.P;
    const int E = Lt * P * Rt;
    C2 *buf0 = reinterpret_cast<C2 *>(smem_raw);
    C2 *buf1 = buf0 + E;
    const int64_t tl = (int64_t)blockIdx.x % a.tilesL;
    const int64_t tr = (int64_t)blockIdx.x / a.tilesL;
    const int64_t l0 = tl * Lt, r0 = tr * Rt;
    const int64_t L = a.L, R = a.R;
    const int lv = (int)((L - l0) < Lt ? (L - l0) : Lt);      // valid extents
    const int rv = (int)((R - r0) < Rt ? (R - r0) : Rt);
    const Tin *in = reinterpret_cast<const Tin *>(a.in);

    // stage the tile: STAGE_U independent loads in flight per thread
    for (int t0 = threadIdx.x; t0 < E; t0 += STAGE_U * blockDim.x) {
        C2 v[STAGE_U];
#pragma unroll
        for (int u = 0; u < STAGE_U; ++u) {
            const int t = t0 + u * blockDim.x;
            v[u] = czero<C2>();
            if (t < E) {
                const int l = t % Lt;
                const int rest = t / Lt;
                const int p = rest % P;
                const int r = rest / P;
                if (l < lv && r < rv)
                    v[u] = to_c(in[(l0 + l) + L * ((int64_t)p + a.P * (r0 + r))], real());
            }
        }
#pragma unroll
        for (int u = 0; u < STAGE_U; ++u) {
            const int t = t0 + u * blockDim.x;
            if (t < E) {
                buf0[t] = v[u];
                if (EPI == EPI_RESID && a.g3) reinterpret_cast<real *>(buf1)[t] = v[u].x + v[u].y;
            }
        }
    }
    __syncthreads();

    float nd = 0.f, nx = 0.f;
    const int G = a.G;
    if (EPI == EPI_RESID) {
        // sum over the group's modes of A_m (x)_m X, all read from buf0, by
        // Gauss's three-multiplication form of the complex product:
        //   Re = sum ar xr - sum ai xi,  Im = sum (ar + ai)(xr + xi) - sum ar xr - sum ai xi
        // with ar + ai stored after each matrix and xr + xi staged beside the
        // tile, so every (i, k) term costs three FP64 FMAs instead of four
        // (a.g3; the classical product remains for callers without the plane).
        const real *bufS = reinterpret_cast<const real *>(buf1);
        const bool g3 = a.g3 != 0;
        if (G == 1 && g3 && a.rows4 && a.gn[0] >= 8) {
            // one mode: a thread takes RES_RB consecutive rows i of one column (l, r),
            // so every staged x value and its re + im sum feed RES_RB rows (rows past
            // n are skipped); matrix entries are the same across the lanes of a warp
            constexpr int RES_RB = 4;
            const int nm = a.gn[0];
            const C2 *M = reinterpret_cast<const C2 *>(a.mats[0]);
            const real *MS = reinterpret_cast<const real *>(M + nm * nm);
            const int ng = (nm + RES_RB - 1) / RES_RB;
            const int W = Lt * ng * Rt;
            for (int w = threadIdx.x; w < W; w += blockDim.x) {
                const int l = w % Lt;
                const int rest = w / Lt;
                const int i0 = (rest % ng) * RES_RB;
                const int r = rest / ng;
                const int o = l + Lt * nm * r;                // tile index of (l, 0, r)
                const C2 *src = buf0 + o;
                const real *srcS = bufS + o;
                real p1[RES_RB], p2[RES_RB], p3[RES_RB];
#pragma unroll
                for (int q = 0; q < RES_RB; ++q) p1[q] = p2[q] = p3[q] = 0;
                for (int k = 0; k < nm; ++k) {
                    const C2 x = src[k * Lt];
                    const real xs = srcS[k * Lt];
#pragma unroll
                    for (int q = 0; q < RES_RB; ++q) {
                        if (i0 + q >= nm) break;
                        const C2 am = __ldg(M + (i0 + q) + k * nm);
                        const real as = __ldg(MS + (i0 + q) + k * nm);
                        p1[q] = fma(am.x, x.x, p1[q]);
                        p2[q] = fma(am.y, x.y, p2[q]);
                        p3[q] = fma(as, xs, p3[q]);
                    }
                }
                if (l >= lv || r >= rv) continue;
#pragma unroll
                for (int q = 0; q < RES_RB; ++q) {
                    const int i = i0 + q;
                    if (i >= nm) break;
                    const int64_t g = (l0 + l) + L * ((int64_t)i + a.P * (r0 + r));
                    double2 *Rp = reinterpret_cast<double2 *>(a.out);
                    double2 base;
                    if (a.first) {
                        const double2 b = reinterpret_cast<const double2 *>(a.B)[g];
                        const double2 xv = to_c(buf0[o + i * Lt], double());
                        base.x = b.x - (a.sig_re * xv.x - a.sig_im * xv.y);
                        base.y = b.y - (a.sig_re * xv.y + a.sig_im * xv.x);
                    } else {
                        base = Rp[g];
                    }
                    double2 out;
                    out.x = base.x - (double)(p1[q] - p2[q]);
                    out.y = base.y - (double)((p3[q] - p1[q]) - p2[q]);
                    Rp[g] = out;
                }
            }
            return;
        }
        for (int t = threadIdx.x; t < E; t += blockDim.x) {
            int l = t % Lt;
            int rest = t / Lt;
            int p = rest % P;
            int r = rest / P;
            real p1 = 0, p2 = 0, p3 = 0;
            int inner = Lt;
            for (int m = 0; m < G; ++m) {
                const int nm = a.gn[m];
                const C2 *M = reinterpret_cast<const C2 *>(a.mats[m]);
                const real *MS = reinterpret_cast<const real *>(M + nm * nm);
                int aa = t % inner;
                int rr = t / inner;
                int i = rr % nm;
                int bb = rr / nm;
                const int64_t o = aa + (int64_t)bb * inner * nm;
                const C2 *src = buf0 + o;
                const real *srcS = bufS + o;
                if (g3) {
                    for (int k = 0; k < nm; ++k) {
                        const C2 am = __ldg(M + i + k * nm);
                        const real as = __ldg(MS + i + k * nm);
                        const C2 x = src[k * inner];
                        p1 = fma(am.x, x.x, p1);
                        p2 = fma(am.y, x.y, p2);
                        p3 = fma(as, srcS[k * inner], p3);
                    }
                } else {                   // classical: p1 = re, p2 = im, p3 unused
                    for (int k = 0; k < nm; ++k) {
                        const C2 am = __ldg(M + i + k * nm);
                        const C2 x = src[k * inner];
                        p1 = fma(am.x, x.x, p1);
                        p1 = fma(-am.y, x.y, p1);
                        p2 = fma(am.x, x.y, p2);
                        p2 = fma(am.y, x.x, p2);
                    }
                }
                inner *= nm;
            }
            C2 acc;
            if (g3) {
                acc.x = p1 - p2;
                acc.y = (p3 - p1) - p2;
            } else {
                acc.x = p1;
                acc.y = p2;
            }
            if (l < lv && r < rv) {
                int64_t g = (l0 + l) + L * ((int64_t)p + a.P * (r0 + r));
                double2 *Rp = reinterpret_cast<double2 *>(a.out);
                double2 base;
                if (a.first) {
                    const double2 b = reinterpret_cast<const double2 *>(a.B)[g];
                    const double2 x = to_c(buf0[t], double());
                    base.x = b.x - (a.sig_re * x.x - a.sig_im * x.y);
                    base.y = b.y - (a.sig_re * x.y + a.sig_im * x.x);
                } else {
                    base = Rp[g];
                }
                double2 o;
                o.x = base.x - (double)acc.x;
                o.y = base.y - (double)acc.y;
                Rp[g] = o;
            }
        }
        return;
    }

    // composition of the group's mode products (forward / back transform):
    // every mode but the last goes smem -> smem, the last one (or the identity
    // when G == 0) goes straight to global memory through the epilogue.  A
    // thread computes RB consecutive rows i of one column, so every tile
    // element it loads feeds RB complex multiply-adds.
    auto epilogue = [&](int t, C2 acc) {
        int l = t % Lt;
        int rest = t / Lt;
        int p = rest % P;
        int r = rest / P;
        if (l >= lv || r >= rv) return;
        int64_t g = (l0 + l) + L * ((int64_t)p + a.P * (r0 + r));
        if (EPI == EPI_STORE) {
            reinterpret_cast<Tout *>(a.out)[g] = to_c(acc, (decltype(Tout().x))0);
        } else if (EPI == EPI_STORE_NORM) {
            double2 o = to_c(acc, double());
            reinterpret_cast<double2 *>(a.out)[g] = o;
            nx = fmaxf(nx, cabsmax(o));
        } else if (EPI == EPI_SUB) {
            // Eq. (C): out = scale * (exp(tA) products) - B
            const double2 b = reinterpret_cast<const double2 *>(a.B)[g];
            const double2 v = to_c(acc, double());
            double2 o;
            o.x = (a.sig_re * v.x - a.sig_im * v.y) - b.x;
            o.y = (a.sig_re * v.y + a.sig_im * v.x) - b.y;
            reinterpret_cast<double2 *>(a.out)[g] = o;
        } else if (EPI == EPI_ACCUM) {
            double2 *Xp = reinterpret_cast<double2 *>(a.out);
            double2 x = Xp[g];
            double2 dd = to_c(acc, double());
            x.x += dd.x;
            x.y += dd.y;
            Xp[g] = x;
            nd = fmaxf(nd, cabsmax(dd));
            nx = fmaxf(nx, cabsmax(x));
        }
    };
    C2 *src = buf0, *dst = buf1;
    int inner = Lt;
    if (G == 0) {
        for (int t = threadIdx.x; t < E; t += blockDim.x) epilogue(t, src[t]);
    }
    for (int m = 0; m < G; ++m) {
        const int nm = a.gn[m];
        const C2 *M = reinterpret_cast<const C2 *>(a.mats[m]);
        const bool last = (m == G - 1);
        const int rb = (nm % 4 == 0) ? 4 : ((nm % 2 == 0) ? 2 : 1);
        const int W = E / rb;
        for (int w = threadIdx.x; w < W; w += blockDim.x) {
            C2 acc[4];
            int tb;
            if constexpr (sizeof(real) == 8) {
                // three-multiplication products for modes with n >= 8 and at least
                // two rows per thread (the xr + xi addition is shared by the rows);
                // otherwise the extra loads and additions cost more than the saved
                // multiplications (measured: n = 2 passes 23% slower, n = 19 6%)
                if (nm < 8 || rb == 1) {
                    if (rb == 4) tb = mode_rows<4>(src, M, nm, inner, w, acc);
                    else if (rb == 2) tb = mode_rows<2>(src, M, nm, inner, w, acc);
                    else tb = mode_rows<1>(src, M, nm, inner, w, acc);
                } else if (rb == 4) tb = mode_rows_3m<4>(src, M, nm, inner, w, acc);
                else tb = mode_rows_3m<2>(src, M, nm, inner, w, acc);
            } else {
                if (rb == 4) tb = mode_rows<4>(src, M, nm, inner, w, acc);
                else if (rb == 2) tb = mode_rows<2>(src, M, nm, inner, w, acc);
                else tb = mode_rows<1>(src, M, nm, inner, w, acc);
            }
            for (int r = 0; r < rb; ++r) {
                const int t = tb + r * inner;
                if (!last) dst[t] = acc[r];
                else epilogue(t, acc[r]);
            }
        }
        if (!last) {
            __syncthreads();
            C2 *tmp = src; src = dst; dst = tmp;
            inner *= nm;
        }
    }
    if (EPI == EPI_STORE_NORM || EPI == EPI_ACCUM) {
        nd = warp_max(nd);
        nx = warp_max(nx);
        if ((threadIdx.x & 31) == 0) {
            if (EPI == EPI_ACCUM) atomic_max_nonneg(&a.flags->dmax, nd);
            atomic_max_nonneg(&a.flags->xmax, nx);
        }
    }
}

// FP32 pass over a group of G adjacent modes that all have n = 2 (the small-n
// workloads): the 2 x 2 products are radix-2 butterflies between tile entries
// whose p indices differ in one bit.  Instead of G shared-memory sweeps, the
// tile is staged once; butterflies on the five lowest bits of p run across the
// lanes of a warp (shuffles) when the tile's rows are single entries (Lt = 1),
// and the other bits run in registers, four bits per round, each thread
// holding the 16 entries of one base index (consecutive threads on consecutive
// shared-memory words).  The epilogue is the general pass's.
template <typename Tin, typename Tout, int EPI>
__global__ void __launch_bounds__(256) k_modeprod_n2(const __grid_constant__ MPArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float2 Ms[MAXG][4];                 // 2 x 2 matrices, column-major
    if (a.done && *(volatile const int *)a.done) return;

    const int Lt = a.Lt, Rt = a.Rt, G = a.G;
    const int P = 1 << G;
    const int E = Lt * P * Rt;
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    const int64_t tl = (int64_t)blockIdx.x % a.tilesL;
    const int64_t tr = (int64_t)blockIdx.x / a.tilesL;
    const int64_t l0 = tl * Lt, r0 = tr * Rt;
    const int64_t L = a.L, R = a.R;
    const int lv = (int)((L - l0) < Lt ? (L - l0) : Lt);
    const int rv = (int)((R - r0) < Rt ? (R - r0) : Rt);
    const Tin *in = reinterpret_cast<const Tin *>(a.in);
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;

    if (tid < 4 * G)
        Ms[tid >> 2][tid & 3] = __ldg(reinterpret_cast<const float2 *>(a.mats[tid >> 2]) + (tid & 3));
    // stage the tile: STAGE_U independent loads in flight per thread
    for (int t0 = tid; t0 < E; t0 += STAGE_U * nt) {
        float2 v[STAGE_U];
#pragma unroll
        for (int u = 0; u < STAGE_U; ++u) {
            const int t = t0 + u * nt;
            v[u] = make_float2(0.f, 0.f);
            if (t < E) {
                const int l = t % Lt;
                const int rest = t / Lt;
                const int p = rest & (P - 1);
                const int r = rest >> G;
                if (l < lv && r < rv)
                    v[u] = to_c(in[(l0 + l) + L * ((int64_t)p + a.P * (r0 + r))], float());
            }
        }
#pragma unroll
        for (int u = 0; u < STAGE_U; ++u)
            if (t0 + u * nt < E) buf[t0 + u * nt] = v[u];
    }
    __syncthreads();

    // y_i = M[i, 0] x_0 + M[i, 1] x_1 for the pair (x_0, x_1) along mode m
    auto bfly = [&](int m, float2 &x0, float2 &x1) {
        const float2 m00 = Ms[m][0], m10 = Ms[m][1], m01 = Ms[m][2], m11 = Ms[m][3];
        float2 y0 = make_float2(0.f, 0.f), y1 = make_float2(0.f, 0.f);
        cmac(y0, m00, x0); cmac(y0, m01, x1);
        cmac(y1, m10, x0); cmac(y1, m11, x1);
        x0 = y0;
        x1 = y1;
    };
    int m0 = 0;
    if (Lt == 1) {
        // bits 0..w-1 of p across the lanes: 32 consecutive entries per warp step
        const int w = G < 5 ? G : 5;
        for (int base = (tid & ~31); base < E; base += nt) {
            const int t = base + lane;
            float2 x = t < E ? buf[t] : make_float2(0.f, 0.f);
            for (int b = 0; b < w; ++b) {
                const float2 y = make_float2(__shfl_xor_sync(0xffffffffu, x.x, 1 << b),
                                             __shfl_xor_sync(0xffffffffu, x.y, 1 << b));
                const bool hi = (lane >> b) & 1;
                const float2 mx = Ms[b][hi ? 3 : 0], my = Ms[b][hi ? 1 : 2];  // M[hi,hi], M[hi,1-hi]
                float2 o = make_float2(0.f, 0.f);
                cmac(o, mx, x);
                cmac(o, my, y);
                x = o;
            }
            if (t < E) buf[t] = x;
        }
        m0 = w;
        __syncthreads();
    }
    // remaining bits in registers, up to four per round
    for (; m0 < G; m0 += 4) {
        const int k = (G - m0) < 4 ? (G - m0) : 4;
        const int nb = E >> k;
        const int hib = G - m0 - k;                 // bits of p above the round
        for (int bi = tid; bi < nb; bi += nt) {
            const int l = bi % Lt;
            int rest = bi / Lt;
            const int plo = rest & ((1 << m0) - 1);
            rest >>= m0;
            const int phi = rest & ((1 << hib) - 1);
            const int r = rest >> hib;
            const int tb = l + Lt * (plo + (phi << (m0 + k)) + P * r);
            const int st = Lt << m0;
            float2 x[16];
#pragma unroll
            for (int s2 = 0; s2 < 16; ++s2)
                if (s2 < (1 << k)) x[s2] = buf[tb + st * s2];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                if (b >= k) break;
#pragma unroll
                for (int s2 = 0; s2 < 16; ++s2)
                    if (s2 < (1 << k) && !((s2 >> b) & 1)) bfly(m0 + b, x[s2], x[s2 | (1 << b)]);
            }
#pragma unroll
            for (int s2 = 0; s2 < 16; ++s2)
                if (s2 < (1 << k)) buf[tb + st * s2] = x[s2];
        }
        __syncthreads();
    }

    float nd = 0.f, nx = 0.f;
    if (EPI == EPI_ACCUM) {
        // X += D: the X reads of STAGE_U entries issued together
        for (int t0 = tid; t0 < E; t0 += STAGE_U * nt) {
            int64_t gg[STAGE_U];
            double2 xv[STAGE_U];
#pragma unroll
            for (int u = 0; u < STAGE_U; ++u) {
                const int t = t0 + u * nt;
                gg[u] = -1;
                if (t < E) {
                    const int l = t % Lt;
                    const int rest = t / Lt;
                    const int p = rest & (P - 1);
                    const int r = rest >> G;
                    if (l < lv && r < rv) gg[u] = (l0 + l) + L * ((int64_t)p + a.P * (r0 + r));
                }
                if (gg[u] >= 0) xv[u] = reinterpret_cast<const double2 *>(a.out)[gg[u]];
            }
#pragma unroll
            for (int u = 0; u < STAGE_U; ++u) {
                if (gg[u] < 0) continue;
                const double2 dd = to_c(buf[t0 + u * nt], double());
                double2 x = xv[u];
                x.x += dd.x;
                x.y += dd.y;
                reinterpret_cast<double2 *>(a.out)[gg[u]] = x;
                nd = fmaxf(nd, cabsmax(dd));
                nx = fmaxf(nx, cabsmax(x));
            }
        }
    }
    for (int t = tid; EPI != EPI_ACCUM && t < E; t += nt) {
        const int l = t % Lt;
        const int rest = t / Lt;
        const int p = rest & (P - 1);
        const int r = rest >> G;
        if (l >= lv || r >= rv) continue;
        const int64_t g = (l0 + l) + L * ((int64_t)p + a.P * (r0 + r));
        const float2 acc = buf[t];
        if (EPI == EPI_STORE) {
            reinterpret_cast<Tout *>(a.out)[g] = to_c(acc, (decltype(Tout().x))0);
        } else if (EPI == EPI_STORE_NORM) {
            const double2 o = to_c(acc, double());
            reinterpret_cast<double2 *>(a.out)[g] = o;
            nx = fmaxf(nx, cabsmax(o));
        }
    }
    if (EPI == EPI_STORE_NORM || EPI == EPI_ACCUM) {
        nd = warp_max(nd);
        nx = warp_max(nx);
        if (lane == 0) {
            if (EPI == EPI_ACCUM) atomic_max_nonneg(&a.flags->dmax, nd);
            atomic_max_nonneg(&a.flags->xmax, nx);
        }
    }
}

template <typename real, typename Tin, typename Tout, int EPI>
static cudaError_t set_smem_attr() {
    return cudaFuncSetAttribute(k_modeprod<real, Tin, Tout, EPI>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_modeprod(int fp64, int in_kind, int out_kind, int epi, const MPArgs &a,
                            size_t smem, cudaStream_t st) {
    if (in_kind == ELEM_R32 || in_kind == ELEM_R64)
        return launch_modeprod_real(fp64, in_kind, out_kind, epi, a, smem, st);
    int64_t tiles = a.tilesL * ((a.R + a.Rt - 1) / a.Rt);
    if (tiles <= 0) return cudaSuccess;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)tiles), block(256);
    if (fp64) {
        if (in_kind != ELEM_C128 || out_kind != ELEM_C128) return cudaErrorInvalidValue;
        if (epi == EPI_STORE)
            k_modeprod<double, double2, double2, EPI_STORE><<<grid, block, smem, st>>>(a);
        else if (epi == EPI_RESID)
            k_modeprod<double, double2, double2, EPI_RESID><<<grid, block, smem, st>>>(a);
        else if (epi == EPI_SUB)
            k_modeprod<double, double2, double2, EPI_SUB><<<grid, block, smem, st>>>(a);
        else
            return cudaErrorInvalidValue;
    } else {
        bool all2 = a.G >= 2 && a.Lt * ((int64_t)1 << a.G) * a.Rt <= (1 << 30);
        for (int m = 0; m < a.G; ++m) all2 = all2 && a.gn[m] == 2;
        if (all2) {                  // groups of n = 2 modes: butterflies
            if (epi == EPI_STORE && in_kind == ELEM_C128 && out_kind == ELEM_C64)
                k_modeprod_n2<double2, float2, EPI_STORE><<<grid, block, smem, st>>>(a);
            else if (epi == EPI_STORE && in_kind == ELEM_C64 && out_kind == ELEM_C64)
                k_modeprod_n2<float2, float2, EPI_STORE><<<grid, block, smem, st>>>(a);
            else if (epi == EPI_STORE_NORM && in_kind == ELEM_C64 && out_kind == ELEM_C128)
                k_modeprod_n2<float2, double2, EPI_STORE_NORM><<<grid, block, smem, st>>>(a);
            else if (epi == EPI_ACCUM && in_kind == ELEM_C64 && out_kind == ELEM_C128)
                k_modeprod_n2<float2, double2, EPI_ACCUM><<<grid, block, smem, st>>>(a);
            else
                return cudaErrorInvalidValue;
            return cudaGetLastError();
        }
        if (epi == EPI_STORE && in_kind == ELEM_C128 && out_kind == ELEM_C64)
            k_modeprod<float, double2, float2, EPI_STORE><<<grid, block, smem, st>>>(a);
        else if (epi == EPI_STORE && in_kind == ELEM_C64 && out_kind == ELEM_C64)
            k_modeprod<float, float2, float2, EPI_STORE><<<grid, block, smem, st>>>(a);
        else if (epi == EPI_STORE_NORM && in_kind == ELEM_C64 && out_kind == ELEM_C128)
            k_modeprod<float, float2, double2, EPI_STORE_NORM><<<grid, block, smem, st>>>(a);
        else if (epi == EPI_ACCUM && in_kind == ELEM_C64 && out_kind == ELEM_C128)
            k_modeprod<float, float2, double2, EPI_ACCUM><<<grid, block, smem, st>>>(a);
        else
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Control kernels
// ---------------------------------------------------------------------------
__global__ void k_solve_init(DevFlags *f) {
    if (threadIdx.x == 0) {
        f->done = 0;
        f->err = 0;
        f->ticket = 0;
        f->iters = 0;
        f->dmax = 0;
        f->xmax = 0;
        f->dprev = 0.f;
        f->est = 0.f;
        f->lastcorr = 0.f;
        f->xlast = 0;
    }
}

// step 0: record ||X_0||; step k >= 1: estimate the error after X_k = X_{k-1} + D_k.
__global__ void k_refine_decide(DevFlags *f, float rtol, int step, int max_refine) {
    if (threadIdx.x != 0 || f->done) return;
    float dmax = __uint_as_float(f->dmax);
    float xmax = __uint_as_float(f->xmax);
    f->xlast = f->xmax;
    if (step == 0) {
        f->dprev = xmax;
        f->dmax = 0;
        f->xmax = 0;
        if (!(xmax == xmax) || xmax > FLT_MAX) { f->err |= ERRBIT_NAN; f->done = 1; }
        else if (xmax == 0.f) f->done = 1;              // B = 0 gives X = 0 exactly
        return;
    }
    float rel = xmax > 0.f ? dmax / xmax : 0.f;
    float rho = f->dprev > 0.f ? dmax / f->dprev : 1.f;
    float est = rho * rel;
    f->iters = step;
    f->lastcorr = rel;
    f->est = est;
    f->dprev = dmax;
    f->dmax = 0;
    f->xmax = 0;
    if (!(rel == rel) || xmax > FLT_MAX) {
        f->err |= ERRBIT_NAN;
        f->done = 1;
    } else if (10.f * est <= rtol || dmax == 0.f) {
        f->done = 1;
    } else if ((step >= 2 && rho >= 1.f) || step >= max_refine) {
        f->err |= ERRBIT_NOTCONV;
        f->done = 1;
    }
}

// min / max of |sigma + sum_j d_j[i_j]| over every multi-index; out3[2] counts
// non-finite sums.  out3[0] starts at ~0ull, out3[1] and out3[2] at 0.
__global__ void k_den_minmax(int Nm, const __grid_constant__ SweepArgs a,
                             unsigned long long *out3) {
    double mn = DBL_MAX, mx = 0.0;
    unsigned long long bad = 0;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < a.ntot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        double dx = a.sig_re, dy = a.sig_im;
        int64_t rem = idx;
        for (int j = 0; j < Nm; ++j) {
            int64_t i = rem % a.n[j];
            rem /= a.n[j];
            dx += a.d[j][2 * i];
            dy += a.d[j][2 * i + 1];
        }
        double m = hypot(dx, dy);
        if (!isfinite(m)) ++bad;
        else { mn = fmin(mn, m); mx = fmax(mx, m); }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(out3 + 0, (unsigned long long)__double_as_longlong(mn));
        atomicMax(out3 + 1, (unsigned long long)__double_as_longlong(mx));
        if (bad) atomicAdd(out3 + 2, bad);
    }
}

cudaError_t launch_solve_init(DevFlags *f, cudaStream_t st) {
    k_solve_init<<<1, 32, 0, st>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_refine_decide(DevFlags *f, float rtol, int step, int max_refine,
                                 cudaStream_t st) {
    k_refine_decide<<<1, 32, 0, st>>>(f, rtol, step, max_refine);
    return cudaGetLastError();
}

cudaError_t launch_den_minmax(int Nm, const int64_t *n, const double *const *d, double sig_re,
                              double sig_im, int64_t ntot, unsigned long long *out3,
                              cudaStream_t st) {
    SweepArgs a{};
    a.Nm = Nm;
    for (int j = 0; j < Nm; ++j) { a.n[j] = n[j]; a.d[j] = d[j]; }
    a.sig_re = sig_re;
    a.sig_im = sig_im;
    a.ntot = ntot;
    int64_t blocks = (ntot + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    if (blocks < 1) blocks = 1;
    k_den_minmax<<<(unsigned)blocks, 256, 0, st>>>(Nm, a, out3);
    return cudaGetLastError();
}

cudaError_t kernels_init(int) {
    cudaError_t e;
    if ((e = set_smem_attr<double, double2, double2, EPI_STORE>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<double, double2, double2, EPI_RESID>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<double, double2, double2, EPI_SUB>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<float, double2, float2, EPI_STORE>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<float, float2, float2, EPI_STORE>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<float, float2, double2, EPI_STORE_NORM>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<float, float2, double2, EPI_ACCUM>()) != cudaSuccess) return e;
    const int big = 200 * 1024;
    if ((e = cudaFuncSetAttribute(k_modeprod_n2<double2, float2, EPI_STORE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_modeprod_n2<float2, float2, EPI_STORE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_modeprod_n2<float2, double2, EPI_STORE_NORM>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_modeprod_n2<float2, double2, EPI_ACCUM>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess)
        return e;
    if ((e = modeprod_tc_init_attrs()) != cudaSuccess) return e;
    if ((e = modeprod_tcw_init_attrs()) != cudaSuccess) return e;
    if ((e = resid_oz_init_attrs()) != cudaSuccess) return e;
    if ((e = modeprod_real_init_attrs()) != cudaSuccess) return e;
    return sweep_init_attrs();
}

}  // namespace sylv
