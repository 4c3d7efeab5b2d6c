// sm_103a kernels of the N-dimensional Bartels-Stewart solver.
//
//  k_modeprod  one transform pass: the mode-j products of Eq. (CUNU2U1B) /
//              Eq. (XUNU2U1Y) for a group of adjacent modes, applied to a
//              tile staged in shared memory; epilogues fuse the FP64 residual
//              R = B - sum_j A_j (x)_j X and the refinement update X += D.
//  k_sweep     the triangular sweep of Eq. (yi1i2iN) as a persistent,
//              dependency-counted wavefront over tiles: a tile starts once its
//              immediate successors along every mode are solved; inside a tile
//              the entries are solved level by level (in-tile index sums).
//  small       control kernels (flags, counters, refinement decision, the
//              plan-time scan of the diagonal sums t_{1,i1i1}+...+t_{N,iNiN}).
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "sylv_internal.h"

namespace sylv {

template <typename real> struct C2T;
template <> struct C2T<float> { using type = float2; };
template <> struct C2T<double> { using type = double2; };

__device__ __forceinline__ float2 to_c(float2 v, float) { return v; }
__device__ __forceinline__ float2 to_c(double2 v, float) {
    return make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ double2 to_c(float2 v, double) {
    return make_double2((double)v.x, (double)v.y);
}
__device__ __forceinline__ double2 to_c(double2 v, double) { return v; }

template <typename C2> __device__ __forceinline__ C2 czero() { C2 z; z.x = 0; z.y = 0; return z; }

// acc += m * x
template <typename C2> __device__ __forceinline__ void cmac(C2 &acc, C2 m, C2 x) {
    acc.x = fma(m.x, x.x, acc.x);
    acc.x = fma(-m.y, x.y, acc.x);
    acc.y = fma(m.x, x.y, acc.y);
    acc.y = fma(m.y, x.x, acc.y);
}
// acc -= t * y
template <typename C2> __device__ __forceinline__ void cmsub(C2 &acc, C2 t, C2 y) {
    acc.x = fma(-t.x, y.x, acc.x);
    acc.x = fma(t.y, y.y, acc.x);
    acc.y = fma(-t.x, y.y, acc.y);
    acc.y = fma(-t.y, y.x, acc.y);
}

// n / d in FP64 with Smith's scaling (Smith, CACM 5(8), 1962).
__device__ __forceinline__ double2 cdiv(double2 n, double2 d) {
    double2 q;
    if (fabs(d.y) <= fabs(d.x)) {
        double r = d.y / d.x;
        double inv = 1.0 / (d.x + d.y * r);
        q.x = (n.x + n.y * r) * inv;
        q.y = (n.y - n.x * r) * inv;
    } else {
        double r = d.x / d.y;
        double inv = 1.0 / (d.x * r + d.y);
        q.x = (n.x * r + n.y) * inv;
        q.y = (n.y * r - n.x) * inv;
    }
    return q;
}

__device__ __forceinline__ float cabsmax(float2 v) { return fmaxf(fabsf(v.x), fabsf(v.y)); }
__device__ __forceinline__ float cabsmax(double2 v) {
    return fmaxf(fabsf((float)v.x), fabsf((float)v.y));
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned *addr, float v) {
    // non-negative floats order like their bit patterns; NaN maps to a large value
    unsigned u = (v == v) ? __float_as_uint(v) : 0x7f800000u;
    atomicMax(addr, u);
}

__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------------------
// Transform pass
// ---------------------------------------------------------------------------
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

    for (int t = threadIdx.x; t < E; t += blockDim.x) {
        int l = t % Lt;
        int rest = t / Lt;
        int p = rest % P;
        int r = rest / P;
        C2 v = czero<C2>();
        if (l < lv && r < rv) v = to_c(in[(l0 + l) + L * ((int64_t)p + a.P * (r0 + r))], real());
        buf0[t] = v;
    }
    __syncthreads();

    float nd = 0.f, nx = 0.f;
    const int G = a.G;
    if (EPI == EPI_RESID) {
        // sum over the group's modes of A_m (x)_m X, all read from buf0
        for (int t = threadIdx.x; t < E; t += blockDim.x) {
            int l = t % Lt;
            int rest = t / Lt;
            int p = rest % P;
            int r = rest / P;
            C2 acc = czero<C2>();
            int inner = Lt;
            for (int m = 0; m < G; ++m) {
                const int nm = a.gn[m];
                const C2 *M = reinterpret_cast<const C2 *>(a.mats[m]);
                int aa = t % inner;
                int rr = t / inner;
                int i = rr % nm;
                int bb = rr / nm;
                const C2 *src = buf0 + aa + (int64_t)bb * inner * nm;
                for (int k = 0; k < nm; ++k) cmac(acc, __ldg(M + i + k * nm), src[k * inner]);
                inner *= nm;
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
    // when G == 0) goes straight to global memory through the epilogue
    C2 *src = buf0, *dst = buf1;
    int inner = Lt;
    for (int m = 0; m + 1 < G; ++m) {
        const int nm = a.gn[m];
        const C2 *M = reinterpret_cast<const C2 *>(a.mats[m]);
        for (int t = threadIdx.x; t < E; t += blockDim.x) {
            int aa = t % inner;
            int rr = t / inner;
            int i = rr % nm;
            int bb = rr / nm;
            const C2 *col = src + aa + (int64_t)bb * inner * nm;
            C2 acc = czero<C2>();
            for (int k = 0; k < nm; ++k) cmac(acc, __ldg(M + i + k * nm), col[k * inner]);
            dst[t] = acc;
        }
        __syncthreads();
        C2 *tmp = src; src = dst; dst = tmp;
        inner *= nm;
    }
    {
        const int nm = G > 0 ? a.gn[G - 1] : 1;
        const C2 *M = G > 0 ? reinterpret_cast<const C2 *>(a.mats[G - 1]) : nullptr;
        for (int t = threadIdx.x; t < E; t += blockDim.x) {
            C2 acc;
            if (G == 0) {
                acc = src[t];
            } else {
                int aa = t % inner;
                int rr = t / inner;
                int i = rr % nm;
                int bb = rr / nm;
                const C2 *col = src + aa + (int64_t)bb * inner * nm;
                acc = czero<C2>();
                for (int k = 0; k < nm; ++k) cmac(acc, __ldg(M + i + k * nm), col[k * inner]);
            }
            int l = t % Lt;
            int rest = t / Lt;
            int p = rest % P;
            int r = rest / P;
            if (l >= lv || r >= rv) continue;
            int64_t g = (l0 + l) + L * ((int64_t)p + a.P * (r0 + r));
            if (EPI == EPI_STORE) {
                reinterpret_cast<Tout *>(a.out)[g] = to_c(acc, (decltype(Tout().x))0);
            } else if (EPI == EPI_STORE_NORM) {
                double2 o = to_c(acc, double());
                reinterpret_cast<double2 *>(a.out)[g] = o;
                nx = fmaxf(nx, cabsmax(o));
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

template <typename real, typename Tin, typename Tout, int EPI>
static cudaError_t set_smem_attr() {
    return cudaFuncSetAttribute(k_modeprod<real, Tin, Tout, EPI>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_modeprod(int fp64, int in_kind, int out_kind, int epi, const MPArgs &a,
                            size_t smem, cudaStream_t st) {
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
        else
            return cudaErrorInvalidValue;
    } else {
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
// Triangular sweep
// ---------------------------------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(256) k_sweep(const __grid_constant__ SweepArgs a) {
    using C2 = typename C2T<real>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *tile_s = reinterpret_cast<C2 *>(smem_raw);
    __shared__ int s_ticket, s_tile;
    __shared__ int64_t s_o[MAXM];
    __shared__ int s_be[MAXM];
    __shared__ int s_I[MAXM];
    __shared__ int64_t s_gbase;
    __shared__ double s_den0x, s_den0y;
    __shared__ int s_abort;

    if (*(volatile const int *)&a.flags->done) return;
    C2 *Y = reinterpret_cast<C2 *>(a.Y);
    const int Nm = a.Nm, nin = a.nin;

    for (;;) {
        if (threadIdx.x == 0) {
            int t = atomicAdd(&a.flags->ticket, 1);
            s_ticket = t;
            s_abort = 0;
            if (t < a.ntiles) {
                int tile = a.order[t];
                s_tile = tile;
                volatile int *c = a.cnt + tile;
                volatile int *err = &a.flags->err;
                long long t0 = clock64();
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
        }
        __syncthreads();
        const int ticket = s_ticket;
        if (ticket >= a.ntiles) break;
        const int tile = s_tile;
        if (s_abort) {
            // drain: mark this tile finished so that nothing waits on it
            if (threadIdx.x == 0) {
                int64_t rem = tile % a.ntiles1;
                for (int j = 0; j < Nm; ++j) {
                    int Ij = (int)((rem / a.TS[j]) % a.Bc[j]);
                    if (Ij > 0) atomicSub(a.cnt + tile - a.TS[j], 1);
                }
            }
            __syncthreads();
            continue;
        }

        // tile geometry
        if (threadIdx.x == 0) {
            int64_t rhs = tile / a.ntiles1;
            int64_t rem = tile % a.ntiles1;
            int64_t gb = rhs * a.ntot;
            double dx = a.sig_re, dy = a.sig_im;
            for (int j = 0; j < Nm; ++j) {
                int Ij = (int)((rem / a.TS[j]) % a.Bc[j]);
                int64_t o = (int64_t)Ij * a.b[j];
                int64_t be = a.n[j] - o;
                if (be > a.b[j]) be = a.b[j];
                s_I[j] = Ij;
                s_o[j] = o;
                s_be[j] = (int)be;
                gb += o * a.S[j];
                if (a.b[j] == 1) {     // modes outside the tile: constant diagonal term
                    dx += a.d[j][2 * o];
                    dy += a.d[j][2 * o + 1];
                }
            }
            s_gbase = gb;
            s_den0x = dx;
            s_den0y = dy;
        }
        __syncthreads();
        const int64_t gbase = s_gbase;

        // stage 1: load C and subtract the contributions of solved tiles
        for (int e = threadIdx.x; e < a.Pt; e += blockDim.x) {
            int64_t g = gbase;
            bool ok = true;
            int tj[MAXM];
            for (int q = 0; q < nin; ++q) {
                int j = a.inmode[q];
                int t = (e / a.BS[q]) % a.b[j];
                if (t >= s_be[j]) ok = false;
                tj[q] = t;
                g += (int64_t)t * a.S[j];
            }
            if (!ok) continue;
            C2 acc = __ldcg(Y + g);
            int q = 0;
            for (int j = 0; j < Nm; ++j) {
                int t = 0;
                if (q < nin && a.inmode[q] == j) { t = tj[q]; ++q; }
                const int64_t nj = a.n[j];
                const int64_t ij = s_o[j] + t;
                const int64_t kend = s_o[j] + s_be[j];
                if (kend >= nj) continue;
                const C2 *Tj = reinterpret_cast<const C2 *>(a.T[j]);
                const int64_t Sj = a.S[j];
                for (int64_t k = kend; k < nj; ++k)
                    cmsub(acc, __ldg(Tj + ij + k * nj), __ldcg(Y + g + (k - ij) * Sj));
            }
            tile_s[e] = acc;
        }
        __syncthreads();

        // stage 2: in-tile wavefront over index sums measured from the tile's end
        for (int lev = 0; lev < a.Lin; ++lev) {
            const int q0 = a.lev_start[lev], q1 = a.lev_start[lev + 1];
            for (int qq = q0 + threadIdx.x; qq < q1; qq += blockDim.x) {
                const int ap = a.sched[qq];
                int e = 0;
                bool ok = true;
                int tj[MAXM];
                for (int q = 0; q < nin; ++q) {
                    int j = a.inmode[q];
                    int apj = (ap / a.BS[q]) % a.b[j];
                    if (apj >= s_be[j]) { ok = false; break; }
                    int t = s_be[j] - 1 - apj;
                    tj[q] = t;
                    e += t * a.BS[q];
                }
                if (!ok) continue;
                C2 num = tile_s[e];
                double dx = s_den0x, dy = s_den0y;
                for (int q = 0; q < nin; ++q) {
                    const int j = a.inmode[q];
                    const int64_t nj = a.n[j];
                    const int64_t ij = s_o[j] + tj[q];
                    dx += a.d[j][2 * ij];
                    dy += a.d[j][2 * ij + 1];
                    const C2 *Tj = reinterpret_cast<const C2 *>(a.T[j]);
                    const int bs = a.BS[q];
                    for (int t = tj[q] + 1; t < s_be[j]; ++t) {   // in-tile successors
                        const int64_t k = s_o[j] + t;
                        cmsub(num, __ldg(Tj + ij + k * nj), tile_s[e + (t - tj[q]) * bs]);
                    }
                }
                double2 y = cdiv(to_c(num, double()), make_double2(dx, dy));
                tile_s[e] = to_c(y, real());
            }
            __syncthreads();
        }

        // stage 3: store Y and release the tiles that wait on this one
        for (int e = threadIdx.x; e < a.Pt; e += blockDim.x) {
            int64_t g = gbase;
            bool ok = true;
            for (int q = 0; q < nin; ++q) {
                int j = a.inmode[q];
                int t = (e / a.BS[q]) % a.b[j];
                if (t >= s_be[j]) { ok = false; break; }
                g += (int64_t)t * a.S[j];
            }
            if (ok) __stcg(Y + g, tile_s[e]);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int j = 0; j < Nm; ++j)
                if (s_I[j] > 0) atomicSub(a.cnt + tile - a.TS[j], 1);
        }
    }
}

__global__ void k_sweep_init(const __grid_constant__ SweepArgs a) {
    if (blockIdx.x == 0 && threadIdx.x == 0) a.flags->ticket = 0;
    for (int64_t tile = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; tile < a.ntiles;
         tile += (int64_t)gridDim.x * blockDim.x) {
        int64_t rem = tile % a.ntiles1;
        int c = 0;
        for (int j = 0; j < a.Nm; ++j) {
            int Ij = (int)((rem / a.TS[j]) % a.Bc[j]);
            c += (Ij < a.Bc[j] - 1);
        }
        a.cnt[tile] = c;
    }
}

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
    }
}

// step 0: record ||X_0||; step k >= 1: estimate the error after X_k = X_{k-1} + D_k.
__global__ void k_refine_decide(DevFlags *f, float rtol, int step, int max_refine) {
    if (threadIdx.x != 0 || f->done) return;
    float dmax = __uint_as_float(f->dmax);
    float xmax = __uint_as_float(f->xmax);
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

cudaError_t launch_sweep(int fp64, const SweepArgs &a, int grid, int threads, size_t smem,
                         cudaStream_t st) {
    if (a.ntiles <= 0) return cudaSuccess;
    if (fp64)
        k_sweep<double><<<grid, threads, smem, st>>>(a);
    else
        k_sweep<float><<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sweep_init(const SweepArgs &a, cudaStream_t st) {
    int64_t blocks = (a.ntiles + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    k_sweep_init<<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
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

int sweep_blocks_per_sm(int fp64, int threads, size_t smem) {
    int nb = 0;
    cudaError_t e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<double>,
                                                                         threads, smem)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep<float>,
                                                                         threads, smem);
    return e == cudaSuccess ? nb : 0;
}

cudaError_t kernels_init(int) {
    cudaError_t e;
    if ((e = set_smem_attr<double, double2, double2, EPI_STORE>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<double, double2, double2, EPI_RESID>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<float, double2, float2, EPI_STORE>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<float, float2, float2, EPI_STORE>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<float, float2, double2, EPI_STORE_NORM>()) != cudaSuccess) return e;
    if ((e = set_smem_attr<float, float2, double2, EPI_ACCUM>()) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_sweep<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  200 * 1024)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_sweep<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  200 * 1024)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

}  // namespace sylv
