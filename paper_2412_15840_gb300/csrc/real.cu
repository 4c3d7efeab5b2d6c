// Mode products of the real-arithmetic variant: real A_j = Q_j T_j Q_j^T, real
// tensors.  The forward transform C = Q_N^T (x)_N (... (Q_1^T (x)_1 B)) and the
// back transform X = Q_N (x)_N (... (Q_1 (x)_1 Y)) (Eqs. (CUNU2U1B) and
// (XUNU2U1Y) with the orthogonal Q_j in place of the unitary U_j), and the FP64
// residual R = B - sigma X - sum_j A_j (x)_j X of the refinement.
//
// The pass has the shape of the complex one: a tile of Lt x P x Rt entries
// (P the product of the group's mode sizes) is staged in shared memory, the
// group's mode products are composed smem -> smem, and the last one goes to
// global memory through the epilogue.  A thread computes RB consecutive rows
// of one column, so every staged entry it loads feeds RB multiply-adds.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "cplx.cuh"
#include "sylv_internal.h"

namespace sylv {

namespace {

template <int RB, typename T>
__device__ __forceinline__ int mode_rows_r(const T *__restrict__ src, const T *__restrict__ M,
                                           int nm, int inner, int w, T *acc) {
    const int aa = w % inner;
    const int rest = w / inner;
    const int ng = nm / RB;
    const int ig = rest % ng;
    const int bb = rest / ng;
    const int i0 = ig * RB;
    const T *col = src + aa + bb * inner * nm;
    T c[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) c[r] = T(0);
    const T *mk = M + i0;
    // RB consecutive rows of one column of M start at a multiple of RB (nm and
    // i0 are multiples of RB): 16-byte vector loads when RB * sizeof(T) >= 16
    constexpr int VW = 16 / sizeof(T);                    // entries per 16 bytes
    for (int k = 0; k < nm; ++k) {
        const T x = col[k * inner];
        T m[RB];
        if constexpr (RB >= VW) {
#pragma unroll
            for (int r = 0; r < RB; r += VW) {
                if constexpr (sizeof(T) == 4) {
                    const float4 q = __ldg(reinterpret_cast<const float4 *>(mk + r));
                    m[r] = q.x; m[r + 1] = q.y; m[r + 2] = q.z; m[r + 3] = q.w;
                } else {
                    const double2 q = __ldg(reinterpret_cast<const double2 *>(mk + r));
                    m[r] = q.x; m[r + 1] = q.y;
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < RB; ++r) m[r] = __ldg(mk + r);
        }
#pragma unroll
        for (int r = 0; r < RB; ++r) c[r] = fma(m[r], x, c[r]);
        mk += nm;
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = c[r];
    return aa + inner * (i0 + nm * bb);
}

__device__ __forceinline__ float absf(double v) { return fabsf((float)v); }

template <typename real, typename Tin, typename Tout, int EPI>
__global__ void __launch_bounds__(256) k_modeprod_r(const __grid_constant__ MPArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.done && *(volatile const int *)a.done) return;

    const int Lt = a.Lt, Rt = a.Rt;
    const int P = (int)a.P;
    const int E = Lt * P * Rt;
    real *buf0 = reinterpret_cast<real *>(smem_raw);
    real *buf1 = buf0 + E;
    const int64_t tl = (int64_t)blockIdx.x % a.tilesL;
    const int64_t tr = (int64_t)blockIdx.x / a.tilesL;
    const int64_t l0 = tl * Lt, r0 = tr * Rt;
    const int64_t L = a.L, R = a.R;
    const int lv = (int)((L - l0) < Lt ? (L - l0) : Lt);
    const int rv = (int)((R - r0) < Rt ? (R - r0) : Rt);
    const Tin *in = reinterpret_cast<const Tin *>(a.in);

    for (int t = threadIdx.x; t < E; t += blockDim.x) {
        const int l = t % Lt;
        const int rest = t / Lt;
        const int p = rest % P;
        const int r = rest / P;
        real v = real(0);
        if (l < lv && r < rv) v = (real)in[(l0 + l) + L * ((int64_t)p + a.P * (r0 + r))];
        buf0[t] = v;
    }
    __syncthreads();

    const int G = a.G;
    if (EPI == EPI_RESID) {
        // R = (first ? B - sigma X : R) - sum over the group's modes of A_m (x)_m X
        for (int t = threadIdx.x; t < E; t += blockDim.x) {
            const int l = t % Lt;
            const int rest = t / Lt;
            const int p = rest % P;
            const int r = rest / P;
            real acc = real(0);
            int inner = Lt;
            for (int m = 0; m < G; ++m) {
                const int nm = a.gn[m];
                const real *M = reinterpret_cast<const real *>(a.mats[m]);
                const int aa = t % inner;
                const int rr = t / inner;
                const int i = rr % nm;
                const int bb = rr / nm;
                const real *src = buf0 + aa + (int64_t)bb * inner * nm;
                for (int k = 0; k < nm; ++k) acc = fma(__ldg(M + i + k * nm), src[k * inner], acc);
                inner *= nm;
            }
            if (l < lv && r < rv) {
                const int64_t g = (l0 + l) + L * ((int64_t)p + a.P * (r0 + r));
                double *Rp = reinterpret_cast<double *>(a.out);
                const double base = a.first
                    ? reinterpret_cast<const double *>(a.B)[g] - a.sig_re * (double)buf0[t]
                    : Rp[g];
                Rp[g] = base - (double)acc;
            }
        }
        return;
    }

    float nd = 0.f, nx = 0.f;
    auto epilogue = [&](int t, real acc) {
        const int l = t % Lt;
        const int rest = t / Lt;
        const int p = rest % P;
        const int r = rest / P;
        if (l >= lv || r >= rv) return;
        const int64_t g = (l0 + l) + L * ((int64_t)p + a.P * (r0 + r));
        if (EPI == EPI_STORE) {
            reinterpret_cast<Tout *>(a.out)[g] = (Tout)acc;
        } else if (EPI == EPI_STORE_NORM) {
            const double o = (double)acc;
            reinterpret_cast<double *>(a.out)[g] = o;
            nx = fmaxf(nx, absf(o));
        } else if (EPI == EPI_ACCUM) {
            double *Xp = reinterpret_cast<double *>(a.out);
            const double dd = (double)acc;
            const double x = Xp[g] + dd;
            Xp[g] = x;
            nd = fmaxf(nd, absf(dd));
            nx = fmaxf(nx, absf(x));
        }
    };
    real *src = buf0, *dst = buf1;
    int inner = Lt;
    if (G == 0) {
        for (int t = threadIdx.x; t < E; t += blockDim.x) epilogue(t, src[t]);
    }
    for (int m = 0; m < G; ++m) {
        const int nm = a.gn[m];
        const real *M = reinterpret_cast<const real *>(a.mats[m]);
        const bool last = (m == G - 1);
        const int rb = (nm % 8 == 0) ? 8 : (nm % 4 == 0) ? 4 : ((nm % 2 == 0) ? 2 : 1);
        const int W = E / rb;
        for (int w = threadIdx.x; w < W; w += blockDim.x) {
            real acc[8];
            int tb;
            if (rb == 8) tb = mode_rows_r<8>(src, M, nm, inner, w, acc);
            else if (rb == 4) tb = mode_rows_r<4>(src, M, nm, inner, w, acc);
            else if (rb == 2) tb = mode_rows_r<2>(src, M, nm, inner, w, acc);
            else tb = mode_rows_r<1>(src, M, nm, inner, w, acc);
            for (int r = 0; r < rb; ++r) {
                const int t = tb + r * inner;
                if (!last) dst[t] = acc[r];
                else epilogue(t, acc[r]);
            }
        }
        if (!last) {
            __syncthreads();
            real *tmp = src; src = dst; dst = tmp;
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

// The first mode (L = 1) in FP32: out[:, c] = M in[:, c] for every column c of
// the n x (ntot nrhs / n) view.  A CTA keeps M (n x n) in shared memory and
// walks tiles of CT1 columns: the tile is staged transposed (column index
// fastest, rows padded to CT1 + 4 floats), and each thread computes 4 x 4
// outputs from one float4 of M and one float4 of the tile per k.  Needs n a
// multiple of 4, n <= MODE1_NMAX.
constexpr int CT1 = 64;
constexpr int CT1P = CT1 + 4;
constexpr int MODE1_NMAX = 128;

template <typename Tin, typename Tout, int EPI>
__global__ void __launch_bounds__(256) k_mode1_r(const __grid_constant__ MPArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.done && *(volatile const int *)a.done) return;
    const int n = a.gn[0];
    float *Ms = reinterpret_cast<float *>(smem_raw);        // n x n, column-major
    float *Xs = Ms + n * n;                                 // n rows of CT1P floats
    const float *M = reinterpret_cast<const float *>(a.mats[0]);
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) Ms[i] = __ldg(M + i);
    const Tin *in = reinterpret_cast<const Tin *>(a.in);
    const int64_t cols = a.R;                               // columns of the view
    const int64_t tiles = (cols + CT1 - 1) / CT1;
    const int nq = n / 4;
    const int items = nq * (CT1 / 4);
    float nd = 0.f, nx = 0.f;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t c0 = tile * CT1;
        const int cv = (int)(cols - c0 < CT1 ? cols - c0 : CT1);
        __syncthreads();                                    // Xs of the previous tile consumed
        const Tin *src = in + c0 * n;
        for (int base = 0; base < n * CT1; base += 8 * 256) {
            Tin v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = base + u * 256 + (int)threadIdx.x;
                v[u] = (idx < n * cv) ? src[idx] : Tin(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = base + u * 256 + (int)threadIdx.x;
                if (idx < n * CT1) Xs[(idx % n) * CT1P + idx / n] = (float)v[u];
            }
        }
        __syncthreads();
        for (int it = threadIdx.x; it < items; it += blockDim.x) {
            const int ri = it % nq, ci = it / nq;
            float acc[4][4] = {};
            const float *mp = Ms + 4 * ri;
            const float *xp = Xs + 4 * ci;
            for (int k = 0; k < n; ++k) {
                const float4 m = *reinterpret_cast<const float4 *>(mp + k * n);
                const float4 x = *reinterpret_cast<const float4 *>(xp + k * CT1P);
                const float mv[4] = {m.x, m.y, m.z, m.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(mv[r], xv[c], acc[r][c]);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int col = 4 * ci + c;
                if (col >= cv) continue;
                const int64_t g = (c0 + col) * n + 4 * ri;
                if (EPI == EPI_STORE) {
                    if constexpr (sizeof(Tout) == 4) {
                        *reinterpret_cast<float4 *>(reinterpret_cast<float *>(a.out) + g) =
                            make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
                    } else {
#pragma unroll
                        for (int r = 0; r < 4; ++r) reinterpret_cast<Tout *>(a.out)[g + r] = (Tout)acc[r][c];
                    }
                } else {
                    double *Xp = reinterpret_cast<double *>(a.out);
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const double d = (double)acc[r][c];
                        if (EPI == EPI_STORE_NORM) {
                            Xp[g + r] = d;
                            nx = fmaxf(nx, absf(d));
                        } else {
                            const double x = Xp[g + r] + d;
                            Xp[g + r] = x;
                            nd = fmaxf(nd, absf(d));
                            nx = fmaxf(nx, absf(x));
                        }
                    }
                }
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
cudaError_t set_attr() {
    return cudaFuncSetAttribute(k_modeprod_r<real, Tin, Tout, EPI>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace

cudaError_t launch_modeprod_real(int fp64, int in_kind, int out_kind, int epi, const MPArgs &a,
                                 size_t smem, cudaStream_t st) {
    const int64_t tiles = a.tilesL * ((a.R + a.Rt - 1) / a.Rt);
    if (tiles <= 0) return cudaSuccess;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)tiles), block(256);
    if (fp64) {
        if (in_kind != ELEM_R64 || out_kind != ELEM_R64) return cudaErrorInvalidValue;
        if (epi == EPI_STORE)
            k_modeprod_r<double, double, double, EPI_STORE><<<grid, block, smem, st>>>(a);
        else if (epi == EPI_RESID)
            k_modeprod_r<double, double, double, EPI_RESID><<<grid, block, smem, st>>>(a);
        else
            return cudaErrorInvalidValue;
    } else {
        // first mode (L = 1), one mode per pass, n a multiple of 4: the tiled kernel
        if (a.G == 1 && a.L == 1 && a.gn[0] % 4 == 0 && a.gn[0] <= MODE1_NMAX) {
            const int n = a.gn[0];
            const size_t sm = (size_t)(n * n + n * CT1P) * sizeof(float);
            const int64_t t1 = (a.R + CT1 - 1) / CT1;
            int dev = 0, sms = 1;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const unsigned g1 = (unsigned)std::max<int64_t>(1, std::min<int64_t>(t1, (int64_t)sms * 4));
            if (epi == EPI_STORE && in_kind == ELEM_R64 && out_kind == ELEM_R32)
                k_mode1_r<double, float, EPI_STORE><<<g1, block, sm, st>>>(a);
            else if (epi == EPI_STORE && in_kind == ELEM_R32 && out_kind == ELEM_R32)
                k_mode1_r<float, float, EPI_STORE><<<g1, block, sm, st>>>(a);
            else if (epi == EPI_STORE_NORM && in_kind == ELEM_R32 && out_kind == ELEM_R64)
                k_mode1_r<float, double, EPI_STORE_NORM><<<g1, block, sm, st>>>(a);
            else if (epi == EPI_ACCUM && in_kind == ELEM_R32 && out_kind == ELEM_R64)
                k_mode1_r<float, double, EPI_ACCUM><<<g1, block, sm, st>>>(a);
            else
                return cudaErrorInvalidValue;
            return cudaGetLastError();
        }
        if (epi == EPI_STORE && in_kind == ELEM_R64 && out_kind == ELEM_R32)
            k_modeprod_r<float, double, float, EPI_STORE><<<grid, block, smem, st>>>(a);
        else if (epi == EPI_STORE && in_kind == ELEM_R32 && out_kind == ELEM_R32)
            k_modeprod_r<float, float, float, EPI_STORE><<<grid, block, smem, st>>>(a);
        else if (epi == EPI_STORE_NORM && in_kind == ELEM_R32 && out_kind == ELEM_R64)
            k_modeprod_r<float, float, double, EPI_STORE_NORM><<<grid, block, smem, st>>>(a);
        else if (epi == EPI_ACCUM && in_kind == ELEM_R32 && out_kind == ELEM_R64)
            k_modeprod_r<float, float, double, EPI_ACCUM><<<grid, block, smem, st>>>(a);
        else
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t modeprod_real_init_attrs() {
    cudaError_t e;
    if ((e = set_attr<double, double, double, EPI_STORE>()) != cudaSuccess) return e;
    if ((e = set_attr<double, double, double, EPI_RESID>()) != cudaSuccess) return e;
    if ((e = set_attr<float, double, float, EPI_STORE>()) != cudaSuccess) return e;
    if ((e = set_attr<float, float, float, EPI_STORE>()) != cudaSuccess) return e;
    if ((e = set_attr<float, float, double, EPI_STORE_NORM>()) != cudaSuccess) return e;
    if ((e = set_attr<float, float, double, EPI_ACCUM>()) != cudaSuccess) return e;
    const int big = 200 * 1024;
    if ((e = cudaFuncSetAttribute(k_mode1_r<double, float, EPI_STORE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_mode1_r<float, float, EPI_STORE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_mode1_r<float, double, EPI_STORE_NORM>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, big)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_mode1_r<float, double, EPI_ACCUM>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

}  // namespace sylv
