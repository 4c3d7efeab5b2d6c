// Tensor-core transform pass (tcgen05, kind::tf32) for the FP32 path.
//
// One mode j with L = prod_{m<j} n_m >= 64 and 32 <= n_j <= 80; view the
// complex64 tensor as (L, n, R).  For every tile (64 consecutive l, one r):
//
//   out[l, i, r] = sum_k M[i, k] X[l, k, r]          (M = U^* or U; Eq. (CUNU2U1B)
//                                                      and Eq. (XUNU2U1Y))
//
// is the real GEMM  D (128 x 2n) = A (128 x n) * B (n x 2n)  with
//   A[(l,c), k] = component c of X[l, k, r]     (the tile's interleaved floats),
//   B[k, i]     = Re M[i, k],   B[k, n + i] = Im M[i, k],
// and the complex result is recombined in the epilogue, where the two rows of
// one l sit in adjacent TMEM lanes (one shuffle):
//   out_re = D[(l,re), i] - D[(l,im), n+i],   out_im = D[(l,im), i] + D[(l,re), n+i].
//
// Precision: 3xTF32.  A = A_hi + A_lo and B = B_hi + B_lo with hi rounded to
// TF32 (cvt.rna.tf32), D = A_lo B_hi + A_hi B_lo + A_hi B_hi accumulated in FP32
// in TMEM; this keeps the FP32 accuracy of the CUDA-core pass, which the
// refinement's one-step convergence needs.
//
// Data movement: B_hi / B_lo are built by the plan in the exact shared-memory
// layout and copied once per CTA by the bulk-copy (TMA) engine onto an
// mbarrier; A is staged through registers because every element is split
// into hi and lo on its way into shared memory.  Operands use the K-major,
// no-swizzle canonical layout: 8 rows x 16 bytes per core matrix, core
// matrices along K at LBO = 128 bytes, 8-row groups at SBO (A: padded by 16
// bytes so that the staging stores are free of bank conflicts).  The next
// tile's A is loaded into registers while the current tile's MMAs and
// epilogue run.
//
// One thread issues the 3 * n/8 MMAs of a tile and commits them to an
// mbarrier; four warps stage A and drain TMEM (warp w owns lanes 32w..32w+31).
// Every wait is bounded; on a timeout the kernel records SYLV_ERR_TIMEOUT,
// frees its TMEM and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "cplx.cuh"
#include "sylv_internal.h"

namespace sylv {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait on an mbarrier phase; false after ~2^24 polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int it = 0; it < (1 << 24); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 64) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;     // descriptor version of the tcgen05 family
    return d;                   // base offset 0, absolute LBO mode, layout: no swizzle
}

// instruction descriptor: D F32, A/B TF32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (row, k) in a K-major, no-swizzle operand
__device__ __forceinline__ uint32_t kmaj_off(int row, int k, uint32_t sbo) {
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 2) * 128u + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 3) * 4u;
}

}  // namespace

constexpr int TC_NU = 20;     // staging units per warp: Kp / 4 <= 20 for n <= 80

template <int EPI>
__global__ void __launch_bounds__(128, 1) k_modeprod_tc(const __grid_constant__ TCArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar_b;
    __shared__ __align__(8) uint64_t mbar_mma;
    __shared__ uint32_t tmem_base_s;
    __shared__ int s_fail;
    if (a.done && *(volatile const int *)a.done) return;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.n, Kp = a.Kp;
    unsigned char *Bhi = sm;
    unsigned char *Blo = sm + a.bimg_bytes;
    unsigned char *Ahi = sm + 2 * a.bimg_bytes;
    unsigned char *Alo = Ahi + 16 * a.sboA;

    if (tid == 0) {
        s_fail = 0;
        mbar_init(&mbar_b, 1);
        mbar_init(&mbar_mma, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base_s, (uint32_t)a.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (tid == 0) {
        mbar_arrive_expect_tx(&mbar_b, 2u * (uint32_t)a.bimg_bytes);
        bulk_g2s(Bhi, a.bimg, (uint32_t)a.bimg_bytes, &mbar_b);
        bulk_g2s(Blo, a.bimg + a.bimg_bytes, (uint32_t)a.bimg_bytes, &mbar_b);
    }
    if (!mbar_wait(&mbar_b, 0)) s_fail = 1;
    __syncthreads();

    const uint32_t idesc = idesc_tf32(128, a.Np);
    const uint32_t ahi = smem_u32(Ahi), alo = smem_u32(Alo);
    const uint32_t bhi = smem_u32(Bhi), blo = smem_u32(Blo);
    const int64_t L = a.L;
    const bool evenL = (L & 1) == 0;
    const int64_t ntile = a.tilesL * a.R;
    uint32_t phase = 0;
    float nd = 0.f, nx = 0.f;

    // A of the next tile is fetched into registers while the current tile's
    // MMAs and epilogue run (TC_NU units of 8 float4 x 4 k per warp, Kp <= 80)
    float x[TC_NU][4];
    auto fetch = [&](int64_t t) {
        const int64_t rr = t / a.tilesL;
        const int64_t ll0 = (t % a.tilesL) * 64;
        const int lvv = (int)((L - ll0) < 64 ? (L - ll0) : 64);
        const float *src = a.in + 2 * (ll0 + rr * L * n);
#pragma unroll
        for (int b = 0; b < TC_NU; ++b) {
            const int u = warp + 4 * b;
            const int m4 = (u & 3) * 8 + (lane & 7);      // float4 index along the 128 rows
            const int k = (u >> 2) * 4 + (lane >> 3);
            x[b][0] = x[b][1] = x[b][2] = x[b][3] = 0.f;
            if (u < Kp && k < n) {
                // 16-byte loads need an even L (the k stride is 8 L bytes); else 8-byte
                const float *p = src + 2 * (int64_t)k * L + 4 * m4;
                if (2 * m4 + 1 < lvv) {
                    if (evenL) {
                        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
                        x[b][0] = v.x; x[b][1] = v.y; x[b][2] = v.z; x[b][3] = v.w;
                    } else {
                        const float2 v0 = __ldg(reinterpret_cast<const float2 *>(p));
                        const float2 v1 = __ldg(reinterpret_cast<const float2 *>(p + 2));
                        x[b][0] = v0.x; x[b][1] = v0.y; x[b][2] = v1.x; x[b][3] = v1.y;
                    }
                } else if (2 * m4 < lvv) {
                    const float2 v0 = __ldg(reinterpret_cast<const float2 *>(p));
                    x[b][0] = v0.x;
                    x[b][1] = v0.y;
                }
            }
        }
    };
    if ((int64_t)blockIdx.x < ntile) fetch(blockIdx.x);

    for (int64_t tile = blockIdx.x; tile < ntile && !s_fail; tile += gridDim.x) {
        const int64_t r = tile / a.tilesL;
        const int64_t l0 = (tile % a.tilesL) * 64;
        const int lv = (int)((L - l0) < 64 ? (L - l0) : 64);

        // stage A: split the fetched values into TF32 hi and lo
#pragma unroll
        for (int b = 0; b < TC_NU; ++b) {
            const int u = warp + 4 * b;
            if (u >= Kp) continue;
            const int m4 = (u & 3) * 8 + (lane & 7);
            const int k = (u >> 2) * 4 + (lane >> 3);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float h = tf32_rna(x[b][j]);
                const uint32_t off = kmaj_off(4 * m4 + j, k, (uint32_t)a.sboA);
                *reinterpret_cast<float *>(Ahi + off) = h;
                *reinterpret_cast<float *>(Alo + off) = x[b][j] - h;
            }
        }
        fence_proxy_async_smem();
        __syncthreads();

        if (tid == 0) {
            tc_fence_after();
            const int steps = Kp / 8;
            for (int s = 0; s < steps; ++s)     // small terms first
                mma_tf32(tmem, smem_desc(alo + 256u * s, 128u, (uint32_t)a.sboA),
                         smem_desc(bhi + 256u * s, 128u, (uint32_t)a.sboB), idesc, s > 0);
            for (int s = 0; s < steps; ++s)
                mma_tf32(tmem, smem_desc(ahi + 256u * s, 128u, (uint32_t)a.sboA),
                         smem_desc(blo + 256u * s, 128u, (uint32_t)a.sboB), idesc, 1u);
            for (int s = 0; s < steps; ++s)
                mma_tf32(tmem, smem_desc(ahi + 256u * s, 128u, (uint32_t)a.sboA),
                         smem_desc(bhi + 256u * s, 128u, (uint32_t)a.sboB), idesc, 1u);
            mma_commit(&mbar_mma);
        }
        if (tile + gridDim.x < ntile) fetch(tile + gridDim.x);
        if (!mbar_wait(&mbar_mma, phase)) s_fail = 1;
        phase ^= 1u;
        tc_fence_after();

        // epilogue: TMEM lane m = 32 warp + lane holds row (l, c) = (m / 2, m % 2)
        const int m = 32 * warp + lane;
        const int ll = m >> 1, c = m & 1;
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
        for (int i0 = 0; i0 < n; i0 += 16) {
            uint32_t va[16], vb[16];
            tmem_ld16(trow + (uint32_t)i0, va);
            tmem_ld16(trow + (uint32_t)(n + i0), vb);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int i = i0 + j;
                const float av = __uint_as_float(va[j]);
                const float pb = __shfl_xor_sync(0xffffffffu, __uint_as_float(vb[j]), 1);
                const float o = c == 0 ? av - pb : av + pb;
                if (i < n && ll < lv) {
                    const int64_t g = 2 * (l0 + ll + (int64_t)i * L + r * L * n) + c;
                    if (EPI == EPI_STORE) {
                        reinterpret_cast<float *>(a.out)[g] = o;
                    } else if (EPI == EPI_STORE_NORM) {
                        reinterpret_cast<double *>(a.out)[g] = (double)o;
                        nx = fmaxf(nx, fabsf(o));
                    } else if (EPI == EPI_ACCUM) {
                        double *xp = reinterpret_cast<double *>(a.out) + g;
                        const double xn = *xp + (double)o;
                        *xp = xn;
                        nd = fmaxf(nd, fabsf(o));
                        nx = fmaxf(nx, fabsf((float)xn));
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }

    if (EPI == EPI_STORE_NORM || EPI == EPI_ACCUM) {
        nd = warp_max(nd);
        nx = warp_max(nx);
        if (lane == 0 && a.flags) {
            if (EPI == EPI_ACCUM) atomic_max_nonneg(&a.flags->dmax, nd);
            atomic_max_nonneg(&a.flags->xmax, nx);
        }
    }
    if (s_fail && tid == 0 && a.flags) atomicOr(&a.flags->err, ERRBIT_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

cudaError_t launch_modeprod_tc(int epi, const TCArgs &a, int grid, size_t smem, cudaStream_t st) {
    if (a.tilesL * a.R <= 0) return cudaSuccess;
    if (epi == EPI_STORE)
        k_modeprod_tc<EPI_STORE><<<grid, 128, smem, st>>>(a);
    else if (epi == EPI_STORE_NORM)
        k_modeprod_tc<EPI_STORE_NORM><<<grid, 128, smem, st>>>(a);
    else if (epi == EPI_ACCUM)
        k_modeprod_tc<EPI_ACCUM><<<grid, 128, smem, st>>>(a);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t modeprod_tc_init_attrs() {
    cudaError_t e;
    const int bytes = 220 * 1024;   // below the 227 KB opt-in limit, leaving room for static smem
    if ((e = cudaFuncSetAttribute(k_modeprod_tc<EPI_STORE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_modeprod_tc<EPI_STORE_NORM>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) !=
        cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_modeprod_tc<EPI_ACCUM>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

uint32_t tc_idesc(int M, int N) { return idesc_tf32(M, N); }

}  // namespace sylv
