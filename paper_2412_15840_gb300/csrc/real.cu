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
    return set_attr<float, float, double, EPI_ACCUM>();
}

}  // namespace sylv
