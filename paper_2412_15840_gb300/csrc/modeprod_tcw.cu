// Warp-specialised tensor-core transform pass (tcgen05, kind::tf32, 3xTF32) for
// the FP32 path: the same product as k_modeprod_tc (modeprod_tc.cu),
//
//   out[l, i, r] = sum_k M[i, k] X[l, k, r]     (M = U^* or U; Eqs. (CUNU2U1B) and
//                                                 (XUNU2U1Y))
//
// as the real GEMM D (128 x 2n) = A (128 x n) B (n x 2n) on tiles of 64
// consecutive l of one r, for modes whose stride L is a multiple of 64 and
// n <= 64, with the tile's data moved by the tensor memory accelerator and
// every stage of the pipeline on warps of its own:
//
//   warp 0       TMA producer: one cp.async.bulk.tensor load per tile of the
//                raw complex64 block (128 floats x n, the tile's 64 l of every
//                k) into a ring of two raw slots;
//   warps 2..5   converters: raw slot -> registers (slot released), then the
//                TF32 hi and lo images of A in the K-major no-swizzle layout
//                of the MMA, one half of K after the other (one A stage, each
//                half with its own full / free barriers);
//   warp 1       MMA issuer: per half of K, A_lo B_hi + A_hi B_lo + A_hi B_hi
//                into one of two TMEM accumulators, committed to mbarriers that
//                free that half of the A stage (the converters write the next
//                tile's first half while the second half's MMAs run) and hand
//                the accumulator to the epilogue;
//   warps 6..13  epilogue: two warps per TMEM lane quadrant drain the
//                accumulator, recombine the complex parts and store.
//
// Stages hand over through mbarriers only (no CTA barrier inside the tile
// loop): raw full/free, A full/free, accumulator full/free.  Every wait is
// bounded; on a timeout the kernel records SYLV_ERR_TIMEOUT, lets issued
// copies and MMAs finish, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <mutex>

#include "cplx.cuh"
#include "sylv_internal.h"
#include "tc_ptx.cuh"

namespace sylv {

namespace {

constexpr int TCW_WARPS = 14;
constexpr int TCW_THREADS = 32 * TCW_WARPS;
constexpr int TCW_CONV0 = 2, TCW_NCONV = 4;   // converter warps 2..5
constexpr int TCW_EPI0 = 6, TCW_NEPI = 8;     // epilogue warps 6..13
constexpr int TCW_CONV_THREADS = 32 * TCW_NCONV;
constexpr int TCW_MAXN = 64;
constexpr int TCW_MAXU = TCW_MAXN / TCW_NCONV; // staging units per converter lane

// K steps (of 8) in the first half of the A stage: halves pay from 6 steps on
// (n >= 48); below that the whole of K is one stage and the second half unused
__device__ __forceinline__ int tcw_half_steps(int steps) { return steps >= 6 ? steps / 2 : steps; }

__device__ __forceinline__ uint32_t kmaj_off(int row, int k, uint32_t lbo, uint32_t sbo) {
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 2) * lbo + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 3) * 4u;
}

}  // namespace

template <int EPI>
__global__ void __launch_bounds__(TCW_THREADS, 1)
k_modeprod_tcw(const __grid_constant__ TCArgs a, const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar_b, bar_afull[2], bar_afree[2];
    __shared__ __align__(8) uint64_t bar_rfull[2], bar_rfree[2], bar_dfull[2], bar_dfree[2];
    __shared__ uint32_t tmem_base_s;
    __shared__ int s_fail;
    if (a.done && *(volatile const int *)a.done) return;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.n, Kp = a.Kp;
    const uint32_t abytes = (uint32_t)a.abytes, lboA = (uint32_t)a.lboA, sboA = (uint32_t)a.sboA;
    const uint32_t rawbytes = (uint32_t)n * 512u;
    unsigned char *Bhi = sm, *Blo = sm + a.bimg_bytes;
    unsigned char *Ahi = sm + 2 * (size_t)a.bimg_bytes, *Alo = Ahi + abytes;
    // raw slots start on a 128-byte boundary of the shared window (TMA destination)
    const uint32_t rawoff = (uint32_t)(2 * (size_t)a.bimg_bytes + 2 * (size_t)abytes);
    unsigned char *raw = sm + (((smem_u32(sm) + rawoff + 127u) & ~127u) - smem_u32(sm));

    if (tid == 0) {
        s_fail = 0;
        mbar_init(&bar_b, 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(&bar_afull[s], TCW_CONV_THREADS);
            mbar_init(&bar_afree[s], 1);
            mbar_init(&bar_rfull[s], 1);
            mbar_init(&bar_rfree[s], TCW_CONV_THREADS);
            mbar_init(&bar_dfull[s], 1);
            mbar_init(&bar_dfree[s], TCW_NEPI);
        }
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base_s, (uint32_t)(2 * a.tmem_cols));
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    const int64_t L = a.L;
    const int64_t tilesL = L / 64;
    const int64_t ntile = tilesL * a.R;
    const int64_t G = gridDim.x;
    float nd = 0.f, nx = 0.f;

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            mbar_arrive_expect_tx(&bar_b, 2u * (uint32_t)a.bimg_bytes);
            bulk_g2s(Bhi, a.bimg, (uint32_t)a.bimg_bytes, &bar_b);
            bulk_g2s(Blo, a.bimg + a.bimg_bytes, (uint32_t)a.bimg_bytes, &bar_b);
            prefetch_tensormap(&tmap);
            int64_t issued = 0;
            for (int64_t k = 0;; ++k) {
                const int64_t t = blockIdx.x + k * G;
                if (t >= ntile || *(volatile int *)&s_fail) break;
                const int s = (int)(k & 1);
                if (k >= 2 && !mbar_wait(&bar_rfree[s], (uint32_t)(((k >> 1) - 1) & 1))) {
                    s_fail = 1;
                    break;
                }
                const int64_t r = t / tilesL;
                const int l0 = (int)((t - r * tilesL) * 64);
                mbar_arrive_expect_tx(&bar_rfull[s], rawbytes);
                tma_load_3d(raw + (size_t)s * rawbytes, &tmap, 2 * l0, 0, (int)r, &bar_rfull[s]);
                issued = k + 1;
            }
            // copies still in flight land before the CTA may exit
            for (int64_t k = issued - 2 < 0 ? 0 : issued - 2; k < issued; ++k)
                if (!mbar_wait(&bar_rfull[k & 1], (uint32_t)((k >> 1) & 1))) s_fail = 1;
            if (!mbar_wait(&bar_b, 0)) s_fail = 1;
        }
    } else if (warp == 1) {
        // -------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(128, a.Np);
            const uint32_t bhi = smem_u32(Bhi), blo = smem_u32(Blo);
            const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo);
            const uint32_t ka = 2u * lboA;
            const int steps = Kp / 8;
            const int sh = tcw_half_steps(steps);   // K steps of the first half
            if (!mbar_wait(&bar_b, 0)) s_fail = 1;
            int64_t commits[2] = {0, 0};       // commits to bar_afree[h]
            for (int64_t k = 0; !*(volatile int *)&s_fail; ++k) {
                const int64_t t = blockIdx.x + k * G;
                if (t >= ntile) break;
                const int b = (int)(k & 1);
                if (k >= 2 && !mbar_wait(&bar_dfree[b], (uint32_t)(((k >> 1) - 1) & 1))) {
                    s_fail = 1;
                    break;
                }
                const uint32_t d = tmem + (uint32_t)(b * a.tmem_cols);
                // each half of K as soon as the converters have written it:
                // A_lo B_hi + A_hi B_lo + A_hi B_hi, small terms first
                const int nh = sh < steps ? 2 : 1;
                for (int h = 0; h < nh; ++h) {
                    if (!mbar_wait(&bar_afull[h], (uint32_t)(k & 1))) { s_fail = 1; break; }
                    tc_fence_after();
                    const int s0 = h ? sh : 0, s1 = h ? steps : sh;
                    for (int s = s0; s < s1; ++s)
                        mma_tf32(d, smem_desc(alo + ka * s, lboA, sboA),
                                 smem_desc(bhi + 256u * s, 128u, (uint32_t)a.sboB), idesc,
                                 s > 0);
                    for (int s = s0; s < s1; ++s)
                        mma_tf32(d, smem_desc(ahi + ka * s, lboA, sboA),
                                 smem_desc(blo + 256u * s, 128u, (uint32_t)a.sboB), idesc, 1u);
                    for (int s = s0; s < s1; ++s)
                        mma_tf32(d, smem_desc(ahi + ka * s, lboA, sboA),
                                 smem_desc(bhi + 256u * s, 128u, (uint32_t)a.sboB), idesc, 1u);
                    mma_commit(&bar_afree[h]);
                    ++commits[h];
                }
                if (*(volatile int *)&s_fail) break;
                mma_commit(&bar_dfull[b]);
            }
            // MMAs still in flight complete before TMEM is released
            for (int h = 0; h < 2; ++h)
                if (commits[h] > 0 && !mbar_wait(&bar_afree[h], (uint32_t)((commits[h] - 1) & 1)))
                    s_fail = 1;
        }
    } else if (warp < TCW_EPI0) {
        // --------------------------------------------------------- converters
        // unit u of converter warp cw: 8 consecutive float4 rows (m4) x 4 k; a
        // lane takes m4 = 8 (u & 3) + (lane & 7), k = 4 (u >> 2) + (lane >> 3)
        const int cw = warp - TCW_CONV0;
        for (int64_t k = 0; !*(volatile int *)&s_fail; ++k) {
            const int64_t t = blockIdx.x + k * G;
            if (t >= ntile) break;
            const int s = (int)(k & 1);
            if (!mbar_wait(&bar_rfull[s], (uint32_t)((k >> 1) & 1))) { s_fail = 1; break; }
            const float *rs = reinterpret_cast<const float *>(raw + (size_t)s * rawbytes);
            float x[TCW_MAXU][4];
#pragma unroll
            for (int j = 0; j < TCW_MAXU; ++j) {
                const int u = cw + TCW_NCONV * j;
                const int m4 = (u & 3) * 8 + (lane & 7);
                const int kk = (u >> 2) * 4 + (lane >> 3);
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (u < Kp && kk < n) v = *reinterpret_cast<const float4 *>(rs + kk * 128 + 4 * m4);
                x[j][0] = v.x; x[j][1] = v.y; x[j][2] = v.z; x[j][3] = v.w;
            }
            fence_proxy_async_smem();
            mbar_arrive(&bar_rfree[s]);
            // each half of K of the A stage is free once the previous tile's MMAs
            // on it completed; units j < jh hold the first half's k
            const int jh = 2 * tcw_half_steps(Kp / 8);
            const int nh = jh < Kp / 4 ? 2 : 1;
            bool bad = false;
            for (int h = 0; h < nh && !bad; ++h) {
                if (k >= 1 && !mbar_wait(&bar_afree[h], (uint32_t)((k - 1) & 1))) {
                    bad = true;
                    break;
                }
#pragma unroll
                for (int j = 0; j < TCW_MAXU; ++j) {
                    const int u = cw + TCW_NCONV * j;
                    if (u >= Kp || (j < jh) != (h == 0)) continue;
                    const int m4 = (u & 3) * 8 + (lane & 7);
                    const int kk = (u >> 2) * 4 + (lane >> 3);
                    const uint32_t off = kmaj_off(4 * m4, kk, lboA, sboA);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float hv = tf32_rna(x[j][q]);
                        *reinterpret_cast<float *>(Ahi + off + 16u * q) = hv;
                        *reinterpret_cast<float *>(Alo + off + 16u * q) = x[j][q] - hv;
                    }
                }
                fence_proxy_async_smem();
                mbar_arrive(&bar_afull[h]);
            }
            if (bad) { s_fail = 1; break; }
        }
    } else {
        // ----------------------------------------------------------- epilogue
        // TMEM lane m = 32 q + lane holds row (ll, cc) = (m / 2, m % 2) of the
        // tile; the two warps of a quadrant take alternate 16-column chunks
        const int q = warp & 3, half = (warp - TCW_EPI0) >> 2;
        const int m = 32 * q + lane;
        const int ll = m >> 1, cc = m & 1;
        for (int64_t k = 0; !*(volatile int *)&s_fail; ++k) {
            const int64_t t = blockIdx.x + k * G;
            if (t >= ntile) break;
            const int b = (int)(k & 1);
            if (!mbar_wait(&bar_dfull[b], (uint32_t)((k >> 1) & 1))) { s_fail = 1; break; }
            tc_fence_after();
            const uint32_t trow = tmem + (uint32_t)(b * a.tmem_cols) + ((uint32_t)(32 * q) << 16);
            const int64_t r = t / tilesL;
            const int64_t base = (t - r * tilesL) * 64 + ll + L * n * r;   // (l, 0, r)
            for (int i0 = 16 * half; i0 < n; i0 += 32) {
                uint32_t va[16], vb[16];
                tmem_ld16(trow + (uint32_t)i0, va);
                tmem_ld16(trow + (uint32_t)(n + i0), vb);
                tmem_wait_ld();
                float o[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float av = __uint_as_float(va[j]);
                    const float pb = __shfl_xor_sync(0xffffffffu, __uint_as_float(vb[j]), 1);
                    o[j] = cc == 0 ? av - pb : av + pb;
                }
#pragma unroll
                for (int t2 = 0; t2 < 8; ++t2) {
                    const float send = cc == 0 ? o[2 * t2 + 1] : o[2 * t2];
                    const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
                    const float re = cc == 0 ? o[2 * t2] : recv;
                    const float im = cc == 0 ? recv : o[2 * t2 + 1];
                    const int i = i0 + 2 * t2 + cc;
                    if (i < n) {
                        const int64_t g = base + (int64_t)i * L;
                        if (EPI == EPI_STORE) {
                            reinterpret_cast<float2 *>(a.out)[g] = make_float2(re, im);
                        } else if (EPI == EPI_STORE_NORM) {
                            reinterpret_cast<double2 *>(a.out)[g] = make_double2(re, im);
                            nx = fmaxf(nx, fmaxf(fabsf(re), fabsf(im)));
                        } else if (EPI == EPI_ACCUM) {
                            double2 *xp = reinterpret_cast<double2 *>(a.out) + g;
                            double2 xv = *xp;
                            xv.x += (double)re;
                            xv.y += (double)im;
                            *xp = xv;
                            nd = fmaxf(nd, fmaxf(fabsf(re), fabsf(im)));
                            nx = fmaxf(nx, fmaxf(fabsf((float)xv.x), fabsf((float)xv.y)));
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_dfree[b]);
        }
        if (EPI == EPI_STORE_NORM || EPI == EPI_ACCUM) {
            nd = warp_max(nd);
            nx = warp_max(nx);
            if (lane == 0 && a.flags) {
                if (EPI == EPI_ACCUM) atomic_max_nonneg(&a.flags->dmax, nd);
                atomic_max_nonneg(&a.flags->xmax, nx);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (s_fail && tid == 0 && a.flags) atomicOr(&a.flags->err, ERRBIT_TIMEOUT);
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)(2 * a.tmem_cols));
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        else
            cudaGetLastError();
    });
    return g_encode;
}

size_t tcw_smem(const TCArgs &a) {
    return 2 * (size_t)a.bimg_bytes + 2 * (size_t)a.abytes + 128 + 2 * (size_t)a.n * 512;
}

}  // namespace

// Launches the warp-specialised pass, or returns cudaErrorNotSupported when
// the pass does not qualify (first mode, complex128 input, L not a multiple
// of 64, n > 64, or no tensor-map encoder); the caller then runs k_modeprod_tc.
cudaError_t launch_modeprod_tcw(int epi, const TCArgs &a, int num_sms, cudaStream_t st) {
    if (a.mode1 || a.in_c128 || a.L % 64 != 0 || a.n > TCW_MAXN || a.n < 8 || a.L <= 0 ||
        a.R <= 0 || a.R > 0x7fffffffLL || 2 * a.L > 0xffffffffLL)
        return cudaErrorNotSupported;
    if (epi != EPI_STORE && epi != EPI_STORE_NORM && epi != EPI_ACCUM)
        return cudaErrorNotSupported;
    const size_t smem = tcw_smem(a);
    if (smem > (size_t)TC_SMEM_MAX) return cudaErrorNotSupported;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc || (reinterpret_cast<uintptr_t>(a.in) & 15)) return cudaErrorNotSupported;
    // the complex64 tensor as floats: (2L, n, R), the tile box (128, n, 1)
    CUtensorMap tm;
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * a.L), (cuuint64_t)a.n, (cuuint64_t)a.R};
    const cuuint64_t strides[2] = {(cuuint64_t)(8 * a.L), (cuuint64_t)(8 * a.L * a.n)};
    const cuuint32_t box[3] = {128u, (cuuint32_t)a.n, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(a.in), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorNotSupported;
    const int64_t ntile = (a.L / 64) * a.R;
    const int grid = (int)(ntile < num_sms ? ntile : num_sms);
    if (epi == EPI_STORE)
        k_modeprod_tcw<EPI_STORE><<<grid, TCW_THREADS, smem, st>>>(a, tm);
    else if (epi == EPI_STORE_NORM)
        k_modeprod_tcw<EPI_STORE_NORM><<<grid, TCW_THREADS, smem, st>>>(a, tm);
    else
        k_modeprod_tcw<EPI_ACCUM><<<grid, TCW_THREADS, smem, st>>>(a, tm);
    return cudaGetLastError();
}

cudaError_t modeprod_tcw_init_attrs() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_modeprod_tcw<EPI_STORE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_MAX)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_modeprod_tcw<EPI_STORE_NORM>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_MAX)) !=
            cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_modeprod_tcw<EPI_ACCUM>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_MAX);
}

}  // namespace sylv
