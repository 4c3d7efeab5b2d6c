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
#include "tc_ptx.cuh"

namespace sylv {


constexpr int TC_WARPS = 16;              // four per TMEM lane quadrant
constexpr int TC_THREADS = 32 * TC_WARPS;
constexpr int TC_NU = 5;                  // staging units per thread: 32 n / 512 <= 5 for n <= 80

// byte offset of element (row, k) in a K-major, no-swizzle operand with
// K-adjacent core matrices `lbo` bytes apart and 8-row groups `sbo` apart
__device__ __forceinline__ uint32_t kmaj_off2(int row, int k, uint32_t lbo, uint32_t sbo) {
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 2) * lbo + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 3) * 4u;
}

// M1 = 0: modes with L >= 64 (tile rows: 64 consecutive l, re/im interleaved);
// M1 = 1: the first mode (tile rows: 64 consecutive columns r).  IN128: the
// input is complex128 (first forward pass of the first mode).
template <int EPI, int M1, int IN128>
__global__ void __launch_bounds__(TC_THREADS, 1) k_modeprod_tc(const __grid_constant__ TCArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar_b;
    __shared__ __align__(8) uint64_t mbar_mma[2];
    __shared__ uint32_t tmem_base_s;
    __shared__ int s_fail;
    if (a.done && *(volatile const int *)a.done) return;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.n, Kp = a.Kp;
    const int nbuf = a.nbuf;
    const uint32_t abytes = (uint32_t)a.abytes;             // one A image (hi or lo)
    const uint32_t lboA = (uint32_t)a.lboA, sboA = (uint32_t)a.sboA;
    unsigned char *Bhi = sm;
    unsigned char *Blo = sm + a.bimg_bytes;
    unsigned char *Abase = sm + 2 * a.bimg_bytes;             // buffer b: hi, lo at 2 b abytes

    if (tid == 0) {
        s_fail = 0;
        mbar_init(&mbar_b, 1);
        mbar_init(&mbar_mma[0], 1);
        mbar_init(&mbar_mma[1], 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base_s, (uint32_t)(a.tmem_cols * nbuf));
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
    const uint32_t bhi = smem_u32(Bhi), blo = smem_u32(Blo);
    const int64_t L = a.L;
    const bool evenL = (L & 1) == 0;
    const bool aligned = (L & 63) == 0;
    const int64_t ntile = M1 ? (a.R + 63) / 64 : (L * a.R + 63) / 64;
    const int half_n = n >> 1;
    uint32_t phase[2] = {0u, 0u};
    float nd = 0.f, nx = 0.f;

    // The tile's values are fetched into registers one tile ahead.
    //  M1 = 0: unit b of a thread: float4 index m4 (4 rows) along the 128 rows
    //          at one k (lanes along m4: coalesced along l);
    //  M1 = 1: unit b: flat float4 f = tid + 256 b of the contiguous tile,
    //          column p = f / (n/2), entries k = 2 (f % (n/2)) and k + 1.
    float x[TC_NU][4];
    auto fetch = [&](int64_t t) {
        if (M1) {
            const int64_t p0 = t * 64;
            const int lvv = (int)((a.R - p0) < 64 ? (a.R - p0) : 64);
#pragma unroll
            for (int b = 0; b < TC_NU; ++b) {
                const int f = tid + TC_THREADS * b;
                const int p = f / half_n, k = 2 * (f - p * half_n);
                x[b][0] = x[b][1] = x[b][2] = x[b][3] = 0.f;
                if (p < lvv) {
                    const int64_t e = (p0 + p) * n + k;       // complex index
                    if (IN128) {
                        const double2 *src = reinterpret_cast<const double2 *>(a.in) + e;
                        const double2 v0 = __ldg(src), v1 = __ldg(src + 1);
                        x[b][0] = (float)v0.x; x[b][1] = (float)v0.y;
                        x[b][2] = (float)v1.x; x[b][3] = (float)v1.y;
                    } else {
                        const float4 v = __ldg(reinterpret_cast<const float4 *>(
                            reinterpret_cast<const float2 *>(a.in) + e));
                        x[b][0] = v.x; x[b][1] = v.y; x[b][2] = v.z; x[b][3] = v.w;
                    }
                }
            }
            return;
        }
        // rows P = 64 t + d (d < 64) of the flattened (l, r) index, l = P mod L
        const int64_t P0 = t * 64;
        const int64_t r0 = P0 / L;
        const int l0 = (int)(P0 - r0 * L);
        const int64_t LR = L * a.R;
        const float *in = reinterpret_cast<const float *>(a.in);
#pragma unroll
        for (int b = 0; b < TC_NU; ++b) {
            const int u = warp + TC_WARPS * b;
            const int m4 = (u & 3) * 8 + (lane & 7);
            const int k = (u >> 2) * 4 + (lane >> 3);
            x[b][0] = x[b][1] = x[b][2] = x[b][3] = 0.f;
            if (u < Kp && k < n && P0 + 2 * m4 < LR) {
                // (a tile never straddles two r when 64 divides L)
                const int q = aligned ? 0 : (l0 + 2 * m4) / (int)L;
                const int l = l0 + 2 * m4 - q * (int)L;
                const int64_t c0 = l + L * ((int64_t)k + (int64_t)n * (r0 + q));
                const float *p = in + 2 * c0;
                const bool second = P0 + 2 * m4 + 1 < LR;
                if (second && l + 1 < L && evenL) {       // both rows adjacent: 16 bytes
                    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
                    x[b][0] = v.x; x[b][1] = v.y; x[b][2] = v.z; x[b][3] = v.w;
                } else {
                    const float2 v0 = __ldg(reinterpret_cast<const float2 *>(p));
                    x[b][0] = v0.x; x[b][1] = v0.y;
                    if (second) {
                        const int64_t c1 = l + 1 < L ? c0 + 1
                                                     : L * ((int64_t)k + (int64_t)n * (r0 + q + 1));
                        const float2 v1 = __ldg(reinterpret_cast<const float2 *>(in + 2 * c1));
                        x[b][2] = v1.x; x[b][3] = v1.y;
                    }
                }
            }
        }
    };
    // split the fetched values into TF32 hi and lo in A buffer `buf`
    auto stage = [&](int buf) {
        unsigned char *Ahi = Abase + 2u * buf * abytes;
        unsigned char *Alo = Ahi + abytes;
#pragma unroll
        for (int b = 0; b < TC_NU; ++b) {
            if (M1) {
                // (re_k, im_k, re_k+1, im_k+1) of column p -> rows 2p (re), 2p+1 (im)
                const int f = tid + TC_THREADS * b;
                const int p = f / half_n, k = 2 * (f - p * half_n);
                if (p >= 64) continue;
                float h[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) h[j] = tf32_rna(x[b][j]);
                const uint32_t o0 = kmaj_off2(2 * p, k, lboA, sboA);
                *reinterpret_cast<float2 *>(Ahi + o0) = make_float2(h[0], h[2]);
                *reinterpret_cast<float2 *>(Ahi + o0 + 16) = make_float2(h[1], h[3]);
                *reinterpret_cast<float2 *>(Alo + o0) =
                    make_float2(x[b][0] - h[0], x[b][2] - h[2]);
                *reinterpret_cast<float2 *>(Alo + o0 + 16) =
                    make_float2(x[b][1] - h[1], x[b][3] - h[3]);
                continue;
            }
            const int u = warp + TC_WARPS * b;
            if (u >= Kp) continue;
            const int m4 = (u & 3) * 8 + (lane & 7);
            const int k = (u >> 2) * 4 + (lane >> 3);
            // rows 4 m4 .. 4 m4 + 3 share an 8-row group: 16 bytes apart
            const uint32_t off = kmaj_off2(4 * m4, k, lboA, sboA);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float h = tf32_rna(x[b][j]);
                *reinterpret_cast<float *>(Ahi + off + 16u * j) = h;
                *reinterpret_cast<float *>(Alo + off + 16u * j) = x[b][j] - h;
            }
        }
        fence_proxy_async_smem();
    };
    // one thread: D[acc] = A_lo B_hi + A_hi B_lo + A_hi B_hi, small terms first;
    // a K step (8 TF32) spans two K-adjacent core matrices
    auto issue = [&](int buf) {
        const uint32_t ahi = smem_u32(Abase + 2u * buf * abytes), alo = ahi + abytes;
        const uint32_t d = tmem + (uint32_t)(buf * a.tmem_cols);
        const uint32_t ka = 2u * lboA;
        tc_fence_after();
        const int steps = Kp / 8;
        for (int s = 0; s < steps; ++s)
            mma_tf32(d, smem_desc(alo + ka * s, lboA, sboA),
                     smem_desc(bhi + 256u * s, 128u, (uint32_t)a.sboB), idesc, s > 0);
        for (int s = 0; s < steps; ++s)
            mma_tf32(d, smem_desc(ahi + ka * s, lboA, sboA),
                     smem_desc(blo + 256u * s, 128u, (uint32_t)a.sboB), idesc, 1u);
        for (int s = 0; s < steps; ++s)
            mma_tf32(d, smem_desc(ahi + ka * s, lboA, sboA),
                     smem_desc(bhi + 256u * s, 128u, (uint32_t)a.sboB), idesc, 1u);
        mma_commit(&mbar_mma[buf]);
    };
    // TMEM lane m = 32 (warp & 3) + lane holds row (p, c) = (m / 2, m % 2) of the
    // tile; the four warps of a lane quadrant take every fourth 16-column chunk
    const int q = warp & 3, quarter = warp >> 2;
    const int m = 32 * q + lane;
    const int ll = m >> 1, cc = m & 1;
    auto epilogue = [&](int64_t t, int buf) {
        const uint32_t trow = tmem + (uint32_t)(buf * a.tmem_cols) + ((uint32_t)(32 * q) << 16);
        if (M1) {
            // complex64 out[p, i]: after one exchange with the partner lane, lane
            // c holds out[p, i0 + 8c .. i0 + 8c + 7] (64 contiguous bytes)
            const int64_t p0 = t * 64;
            const bool live = p0 + ll < a.R;
            float2 *orow = reinterpret_cast<float2 *>(a.out) + (p0 + ll) * n;
            for (int i0 = 16 * quarter; i0 < n; i0 += 64) {
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
                float4 w[4];
#pragma unroll
                for (int t2 = 0; t2 < 8; ++t2) {
                    const float send = cc == 0 ? o[8 + t2] : o[t2];
                    const float recv = __shfl_xor_sync(0xffffffffu, send, 1);
                    const float re = cc == 0 ? o[t2] : recv;
                    const float im = cc == 0 ? recv : o[8 + t2];
                    if (t2 & 1) { w[t2 >> 1].z = re; w[t2 >> 1].w = im; }
                    else { w[t2 >> 1].x = re; w[t2 >> 1].y = im; }
                }
                const int ib = i0 + 8 * cc;
                if (live && ib < n) {
                    float4 *dst = reinterpret_cast<float4 *>(orow + ib);
#pragma unroll
                    for (int v = 0; v < 4; ++v) dst[v] = w[v];
                }
            }
            return;
        }
        // complex out[l, i]: lane c of a pair stores the columns i0 + 2t + c
        // (t < 8) after one exchange per column pair; row pair ll is the
        // flattened row P = 64 t + ll
        const int64_t P = t * 64 + ll;
        const bool live = P < L * a.R;
        const int64_t rP = aligned ? (t * 64) / L : P / L;
        const int64_t base = (P - rP * L) + L * n * rP;          // complex index of (l, 0, r)
        for (int i0 = 16 * quarter; i0 < n; i0 += 64) {
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
                if (i < n && live) {
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
    };

    // pipeline: with two buffers the MMAs of tile t+1 run while tile t drains
    // (`pending` is uniform across the block: MMAs issued and not yet waited for)
    const int64_t G = gridDim.x;
    int64_t tile = blockIdx.x;
    bool pending[2] = {false, false};
    if (tile < ntile && !s_fail) {
        fetch(tile);
        stage(0);
        __syncthreads();
        if (tid == 0) issue(0);
        pending[0] = true;
        if (tile + G < ntile) fetch(tile + G);
    }
    for (int it = 0; tile < ntile && !s_fail; tile += G, ++it) {
        const int cur = nbuf == 2 ? (it & 1) : 0;
        const int64_t next = tile + G;
        if (nbuf == 2 && next < ntile) {
            stage(cur ^ 1);
            __syncthreads();
            if (tid == 0) issue(cur ^ 1);
            pending[cur ^ 1] = true;
            if (next + G < ntile) fetch(next + G);
        }
        if (!mbar_wait(&mbar_mma[cur], phase[cur])) s_fail = 1;
        phase[cur] ^= 1u;
        pending[cur] = false;
        tc_fence_after();
        epilogue(tile, cur);
        tc_fence_before();
        __syncthreads();
        if (nbuf == 1 && next < ntile && !s_fail) {
            stage(0);
            __syncthreads();
            if (tid == 0) issue(0);
            pending[0] = true;
            if (next + G < ntile) fetch(next + G);
        }
    }
    // after a timeout: let MMAs still in flight finish before TMEM is released
    for (int b = 0; b < 2; ++b)
        if (pending[b] && !mbar_wait(&mbar_mma[b], phase[b])) s_fail = 1;

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
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)(a.tmem_cols * nbuf));
}

cudaError_t launch_modeprod_tc(int epi, const TCArgs &a, int grid, size_t smem, cudaStream_t st) {
    if (a.tilesL * a.R <= 0) return cudaSuccess;
    if (a.mode1) {
        // first-mode pass: never the last pass of a transform (complex64 out)
        if (epi != EPI_STORE || (a.n & 7) || a.n > 80) return cudaErrorInvalidValue;
        if (a.in_c128)
            k_modeprod_tc<EPI_STORE, 1, 1><<<grid, TC_THREADS, smem, st>>>(a);
        else
            k_modeprod_tc<EPI_STORE, 1, 0><<<grid, TC_THREADS, smem, st>>>(a);
        return cudaGetLastError();
    }
    if (a.in_c128) return cudaErrorInvalidValue;
    if (epi == EPI_STORE)
        k_modeprod_tc<EPI_STORE, 0, 0><<<grid, TC_THREADS, smem, st>>>(a);
    else if (epi == EPI_STORE_NORM)
        k_modeprod_tc<EPI_STORE_NORM, 0, 0><<<grid, TC_THREADS, smem, st>>>(a);
    else if (epi == EPI_ACCUM)
        k_modeprod_tc<EPI_ACCUM, 0, 0><<<grid, TC_THREADS, smem, st>>>(a);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <int EPI, int M1, int IN128>
static cudaError_t tc_attr() {
    return cudaFuncSetAttribute(k_modeprod_tc<EPI, M1, IN128>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_MAX);
}

cudaError_t modeprod_tc_init_attrs() {
    cudaError_t e;
    if ((e = tc_attr<EPI_STORE, 0, 0>()) != cudaSuccess) return e;
    if ((e = tc_attr<EPI_STORE_NORM, 0, 0>()) != cudaSuccess) return e;
    if ((e = tc_attr<EPI_ACCUM, 0, 0>()) != cudaSuccess) return e;
    if ((e = tc_attr<EPI_STORE, 1, 0>()) != cudaSuccess) return e;
    return tc_attr<EPI_STORE, 1, 1>();
}

}  // namespace sylv
