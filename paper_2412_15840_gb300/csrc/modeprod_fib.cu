// Transform pass over one mode with a short fibre (FP32 path, n <= 24), on the
// CUDA cores.
//
// View the tensor along mode j as (L, n, R).  One thread owns one fibre
// x[l, :, r]: it loads the n entries, forms
//
//   out[l, i, r] = sum_k M[i, k] x[l, k, r]      (M = U^* or U; Eq. (CUNU2U1B)
//                                                  and Eq. (XUNU2U1Y))
//
// in registers, and stores the n results.  Consecutive threads take
// consecutive l, so for L >= 32 every load and store instruction of a warp
// touches contiguous memory.  M sits in shared memory, rows padded to the
// register block with zeros, and every lane of a warp reads the same entry
// at the same time (a broadcast).  No tile is staged and no barrier is taken
// after the one that publishes M: the n independent loads of each resident
// thread keep HBM busy, where a tensor-core pass over 64-row tiles of a short
// fibre spends its time on per-tile bookkeeping.  Cost: 4n FP32 FMAs per entry
// (76 at n = 19); every entry is read and written once.
//
// A thread computes the outputs in chunks of NI rows (NI = NX up to 20, half
// of NX above), so that the n loaded values and one chunk of accumulators fit
// in registers.  A fibre is read completely before any of its results is
// written, so the pass may run in place.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "cplx.cuh"
#include "sylv_internal.h"

namespace sylv {

constexpr int FIB_THREADS = 256;

template <int NX> struct FibChunk { static constexpr int NI = NX <= 20 ? NX : NX / 2; };

template <int NX, typename Tin, typename Tout, int EPI>
__global__ void __launch_bounds__(FIB_THREADS) k_modeprod_fib(const __grid_constant__ MPArgs a) {
    constexpr int NI = FibChunk<NX>::NI;
    constexpr int NPAD = NX;                     // padded row length of M in shared memory
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *Ms = reinterpret_cast<float2 *>(smem_raw);   // Ms[k * NPAD + i] = M[i, k]
    if (a.done && *(volatile const int *)a.done) return;

    const int n = a.gn[0];
    const float2 *M = reinterpret_cast<const float2 *>(a.mats[0]);   // column-major n x n
    for (int e = threadIdx.x; e < n * NPAD; e += blockDim.x) {
        const int k = e / NPAD, i = e - k * NPAD;
        Ms[e] = i < n ? __ldg(M + i + (int64_t)k * n) : make_float2(0.f, 0.f);
    }
    __syncthreads();

    const int64_t L = a.L;
    const int64_t F = L * a.R;                   // fibres
    const int64_t Ln = L * n;
    const Tin *in = reinterpret_cast<const Tin *>(a.in);
    float nd = 0.f, nx = 0.f;
    const int64_t stride = (int64_t)gridDim.x * FIB_THREADS;
    for (int64_t f = (int64_t)blockIdx.x * FIB_THREADS + threadIdx.x; f < F; f += stride) {
        const int64_t r = f / L;
        const int64_t base = (f - r * L) + Ln * r;   // entry (l, 0, r)
        float2 x[NX];
#pragma unroll
        for (int k = 0; k < NX; ++k)
            x[k] = k < n ? to_c(__ldg(in + base + (int64_t)k * L), float())
                         : make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < NX / NI; ++c) {
            const int i0 = c * NI;
            if (i0 >= n) break;
            float2 acc[NI];
#pragma unroll
            for (int i = 0; i < NI; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < NX; ++k) {
                if (k >= n) break;
                const float4 *mk = reinterpret_cast<const float4 *>(Ms + k * NPAD + i0);
#pragma unroll
                for (int i = 0; i < NI; i += 2) {
                    const float4 m = mk[i >> 1];
                    cmac(acc[i], make_float2(m.x, m.y), x[k]);
                    cmac(acc[i + 1], make_float2(m.z, m.w), x[k]);
                }
            }
#pragma unroll
            for (int i = 0; i < NI; ++i) {
                if (i0 + i >= n) break;
                const int64_t g = base + (int64_t)(i0 + i) * L;
                if (EPI == EPI_STORE) {
                    reinterpret_cast<Tout *>(a.out)[g] = to_c(acc[i], (decltype(Tout().x))0);
                } else if (EPI == EPI_STORE_NORM) {
                    const double2 o = to_c(acc[i], double());
                    reinterpret_cast<double2 *>(a.out)[g] = o;
                    nx = fmaxf(nx, cabsmax(o));
                } else if (EPI == EPI_ACCUM) {
                    double2 *Xp = reinterpret_cast<double2 *>(a.out) + g;
                    double2 xv = *Xp;
                    const double2 dd = to_c(acc[i], double());
                    xv.x += dd.x;
                    xv.y += dd.y;
                    *Xp = xv;
                    nd = fmaxf(nd, cabsmax(dd));
                    nx = fmaxf(nx, cabsmax(xv));
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

int fib_nx(int n) {
    if (n < 1 || n > FIB_NMAX) return 0;
    if (n <= 8) return 8;
    if (n <= 12) return 12;
    if (n <= 16) return 16;
    if (n <= 20) return 20;
    return 24;
}

template <int NX>
static cudaError_t launch_nx(int in_kind, int out_kind, int epi, const MPArgs &a, unsigned grid,
                             size_t smem, cudaStream_t st) {
    if (epi == EPI_STORE && in_kind == ELEM_C128 && out_kind == ELEM_C64)
        k_modeprod_fib<NX, double2, float2, EPI_STORE><<<grid, FIB_THREADS, smem, st>>>(a);
    else if (epi == EPI_STORE && in_kind == ELEM_C64 && out_kind == ELEM_C64)
        k_modeprod_fib<NX, float2, float2, EPI_STORE><<<grid, FIB_THREADS, smem, st>>>(a);
    else if (epi == EPI_STORE_NORM && in_kind == ELEM_C64 && out_kind == ELEM_C128)
        k_modeprod_fib<NX, float2, double2, EPI_STORE_NORM><<<grid, FIB_THREADS, smem, st>>>(a);
    else if (epi == EPI_ACCUM && in_kind == ELEM_C64 && out_kind == ELEM_C128)
        k_modeprod_fib<NX, float2, double2, EPI_ACCUM><<<grid, FIB_THREADS, smem, st>>>(a);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_modeprod_fib(int in_kind, int out_kind, int epi, const MPArgs &a, int num_sms,
                                cudaStream_t st) {
    if (a.G != 1) return cudaErrorInvalidValue;
    const int nx = fib_nx(a.gn[0]);
    if (nx == 0) return cudaErrorInvalidValue;
    const int64_t F = a.L * a.R;
    if (F <= 0) return cudaSuccess;
    // grid-stride: eight CTAs per SM (about four waves of the resident ones)
    const int64_t want = (F + FIB_THREADS - 1) / FIB_THREADS;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms * 8));
    const size_t smem = (size_t)a.gn[0] * nx * sizeof(float2);
    switch (nx) {
    case 8: return launch_nx<8>(in_kind, out_kind, epi, a, grid, smem, st);
    case 12: return launch_nx<12>(in_kind, out_kind, epi, a, grid, smem, st);
    case 16: return launch_nx<16>(in_kind, out_kind, epi, a, grid, smem, st);
    case 20: return launch_nx<20>(in_kind, out_kind, epi, a, grid, smem, st);
    default: return launch_nx<24>(in_kind, out_kind, epi, a, grid, smem, st);
    }
}

}  // namespace sylv
