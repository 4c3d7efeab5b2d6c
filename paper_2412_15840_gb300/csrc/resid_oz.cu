// Residual passes of the mixed path with the mode products on the bf16 tensor
// cores, exact to ~2^-46 (precision SYLV_MIXED_FP32_EMU).
//
// One pass applies one mode j of
//     R = B - sigma X - sum_j A_j (x)_j X        (the refinement residual)
// to a complex128 X.  The FP64 product A_j (x)_j X is replaced by an exact
// integer computation in the style of Ozaki's error-free splitting:
//   * X / 2^eX and A / 2^eA (eX, eA powers of two above the largest entry) are
//     written as 6 signed base-256 digits each, v = sum_t xi_t 256^-(t+1)
//     (truncation error < 2^-47 of the largest entry); every digit is an
//     integer of magnitude <= 255, exact in bf16;
//   * each digit pair (t, u) is one bf16 GEMM whose products (< 2^16) and sums
//     over k (< n 2^16 <= 2^22) are exact in the FP32 accumulator;
//   * pairs with t + u = 0, 1, 2 accumulate in their own TMEM accumulator
//     (still exact: at most 3 n 2^16 < 2^24); the pairs with t + u = 3, 4, 5
//     share a fourth accumulator, lowest order first, each group entered with
//     scale-input-d = 8 (D = A B + 2^-8 D), whose FP32 rounding stays below
//     2^-46 of the result;
//   * the epilogue recombines the complex parts exactly (TwoSum), combines the
//     four accumulators in FP32 pairs (Horner in base 256) and subtracts the
//     result from R kept as FP32 pairs (hi, lo).
// Digit pairs with t + u > 5 are dropped (< 2^-45 relative).  The scalar sigma
// of the singleton modes is folded into the first mode's digits (A_1 + sigma I).
//
// The base an update is added to and the form of its result are runtime modes,
// so one kernel serves every pass of the residual and of the Theorem 1 evolve:
//   in:  OZ_IN_B      bsign * B, split into FP32 pairs by integer operations
//                     (no FP64 arithmetic in the pass);
//        OZ_IN_PAIRS  the FP32 pairs the previous pass wrote;
//        OZ_IN_ZERO   nothing (a plain product A (x)_j X);
//   out: OZ_OUT_PAIRS FP32 pairs for the next pass;
//        OZ_OUT_C64   complex64 (the residual, input of the correction solve);
//        OZ_OUT_C128  complex128 (W = B + sum_j A_j (x)_j X0 and the exp(t A_j)
//                     products of the evolve, whose inputs are complex128).
// `neg` chooses base - A (x)_j X (the residual) or base + A (x)_j X.
//
// Tiles follow the tensor-core transform pass: 64 consecutive rows of the
// flattened (l, r) index for a later mode (M1 = 0), 64 consecutive columns for
// the first mode (M1 = 1).  The GEMM per digit pair is D(128 x 2n) = Xd(128 x n) Ad(n x 2n),
// rows (p, re/im), columns [Re A^T | Im A^T].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "cplx.cuh"
#include "sylv_internal.h"
#include "tc_ptx.cuh"

namespace sylv {

namespace {

constexpr int OZ_WARPS = 16;
constexpr int OZ_THREADS = 32 * OZ_WARPS;
constexpr int OZ_EL = 8;            // complex entries per thread and tile: 64 n / 512 <= 8

// element (row, k) of a K-major, no-swizzle bf16 operand
__device__ __forceinline__ uint32_t kmaj_off_b16(int row, int k, uint32_t lbo, uint32_t sbo) {
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * lbo + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

// 48-bit fixed-point magnitude of x / 2^ex (|x| < 2^(ex-1)) and its sign
__device__ __forceinline__ uint64_t fixed48(double x, int ex, uint32_t &neg) {
    const uint64_t bits = (uint64_t)__double_as_longlong(x);
    neg = (uint32_t)(bits >> 63);
    const int eb = (int)((bits >> 52) & 0x7FF);
    if (eb == 0) return 0;                                // zero or subnormal: below 2^-1022
    const uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    int sh = ex + 1027 - eb;                              // F = m 2^(E - ex - 4)
    if (sh > 63) sh = 63;
    if (sh < 0) sh = 0;                                   // (only if |x| exceeds the scale)
    return m >> sh;
}

__device__ __forceinline__ uint16_t digit_bf16(uint64_t F, int t, uint32_t neg) {
    const uint32_t d = (uint32_t)(F >> (40 - 8 * t)) & 0xFFu;
    const __nv_bfloat16 b = __float2bfloat16_rn((float)d);     // exact: d <= 255
    return (uint16_t)(__bfloat16_as_ushort(b) | (d ? (neg << 15) : 0u));
}

// x = hi + lo with hi = fl32(x) and lo = fl32(x - hi), by integer operations on
// the FP64 bit pattern (no FP64 arithmetic); exact to ~2^-48 |x| for |x| in
// the FP32 range, zero for zero and FP64 subnormals
__device__ __forceinline__ void split_double(double x, float &hi, float &lo) {
    const uint64_t bits = (uint64_t)__double_as_longlong(x);
    const int eb = (int)((bits >> 52) & 0x7FF);
    if (eb == 0) { hi = 0.f; lo = 0.f; return; }
    if (eb == 0x7FF) { hi = (float)x; lo = 0.f; return; }
    const uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);     // 53-bit significand
    uint64_t mh = m >> 29;                                              // 24 bits, nearest-even
    const uint64_t rem = m & ((1ull << 29) - 1);
    if (rem > (1ull << 28) || (rem == (1ull << 28) && (mh & 1))) ++mh;
    const int e = eb - 1023;
    const int r = (int)((int64_t)m - (int64_t)(mh << 29));             // |r| <= 2^28
    float h = ldexpf(__uint2float_rn((uint32_t)mh), e - 23);
    float l = ldexpf(__int2float_rn(r), e - 52);
    if (bits >> 63) { h = -h; l = -l; }
    hi = h;
    lo = l;
}

// 16-byte asynchronous global -> shared copy (L2 only), per-thread completion
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// FP32 pairs (hi, lo): error-free sum and the usual double-float addition
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_add(float &h, float &l, float bh, float bl) {
    float s, e;
    two_sum(h, bh, s, e);
    e += l + bl;
    h = s + e;
    l = e - (h - s);
}

}  // namespace

template <int M1>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_resid_oz(const __grid_constant__ OzArgs a) {
    const double2 *Xg = reinterpret_cast<const double2 *>(a.X);
    const double2 *Bg = reinterpret_cast<const double2 *>(a.B);
    const float4 *Rin = reinterpret_cast<const float4 *>(a.Rin);
    float4 *Rout = reinterpret_cast<float4 *>(a.Rout);
    float2 *Rc64 = reinterpret_cast<float2 *>(a.Rc64);
    double2 *Rc128 = reinterpret_cast<double2 *>(a.Rc64);
    // operand read by the epilogue, its sign, and the output format (see OzArgs)
    const int in_mode = a.in_mode, out_mode = a.out_mode;
    const float vsign = a.neg ? 1.f : -1.f;       // R = base - value, or base + value
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar_a;
    __shared__ __align__(8) uint64_t mbar_mma;
    __shared__ uint32_t tmem_base_s;
    __shared__ int s_fail;
    if (a.done && *(volatile const int *)a.done) return;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = a.n, Kp = a.Kp, Np = a.Np;
    unsigned char *Aimg = sm;                                  // 6 digit images of A
    unsigned char *Ximg = sm + 6 * a.aimg_bytes;               // 6 digit images of X
    // epilogue operands (R pairs or B), fetched once the MMAs no longer read the
    // X digits: slot-major, 16 bytes per thread and slot
    unsigned char *Rs = sm + a.rstage_off;
    const uint32_t lboX = (uint32_t)a.lboX, sboX = (uint32_t)a.sboX;

    if (tid == 0) {
        s_fail = 0;
        mbar_init(&mbar_a, 1);
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
        mbar_arrive_expect_tx(&mbar_a, 6u * (uint32_t)a.aimg_bytes);
        for (int u = 0; u < 6; ++u)
            bulk_g2s(Aimg + u * a.aimg_bytes, a.aimg + (size_t)u * a.aimg_bytes,
                     (uint32_t)a.aimg_bytes, &mbar_a);
    }
    // zero the X digit images once: the K padding (k >= n) must stay zero
    for (int w = tid; w < 6 * a.ximg_bytes / 16; w += OZ_THREADS)
        reinterpret_cast<uint4 *>(Ximg)[w] = make_uint4(0u, 0u, 0u, 0u);
    if (!mbar_wait(&mbar_a, 0)) s_fail = 1;

    // scale exponent of X: 2^eX > 2 max|X| (max(|re|, |im|) of the current X)
    const float xl = __uint_as_float(a.flags->xlast);
    const int eX = xl > 0.f ? ilogbf(xl) + 2 : 0;
    const int escale = eX + a.eA - 16;                         // value = 2^escale * Horner sum
    const uint32_t idesc = idesc_bf16(128, Np);
    const int64_t L = a.L;
    const bool aligned = (L & 63) == 0;      // 64-row tiles never straddle two r
    const int64_t ntile = M1 ? (a.R + 63) / 64 : (L * a.R + 63) / 64;
    const int ksteps = Kp / 16;
    uint32_t phase = 0;

    // the tile's complex entries: e = tid + 512 b; non-M1: p = e % 64 (lanes
    // along l, coalesced), k = e / 64; M1: k = e % n (lanes along k), p = e / n
    double2 xv[OZ_EL];
    auto tile_base = [&](int64_t t, int64_t &r, int64_t &p0, int &pv) {
        if (M1) {
            r = 0;
            p0 = t * 64;
            pv = (int)((a.R - p0) < 64 ? (a.R - p0) : 64);
        } else {
            // rows P = 64 t + p of the flattened (l, r) index: r = first row's r,
            // p0 = first row's l
            const int64_t P0 = t * 64, LR = L * a.R;
            r = P0 / L;
            p0 = P0 - r * L;
            pv = (int)((LR - P0) < 64 ? (LR - P0) : 64);
        }
    };
    auto coord = [&](int e, int &p, int &k) {
        if (M1) { p = e / n; k = e - p * n; }
        else { p = e & 63; k = e >> 6; }
    };
    auto gidx = [&](int64_t r, int64_t p0, int p, int k) -> int64_t {
        if (M1) return (p0 + p) * n + k;
        const int q = aligned ? 0 : (int)(p0 + p) / (int)L;   // rows past the end of r
        const int64_t l = p0 + p - (int64_t)q * L;
        return l + L * ((int64_t)k + (int64_t)n * (r + q));
    };
    auto fetch = [&](int64_t t) {
        int64_t r, p0;
        int pv;
        tile_base(t, r, p0, pv);
#pragma unroll
        for (int b = 0; b < OZ_EL; ++b) {
            const int e = tid + OZ_THREADS * b;
            int p, k;
            coord(e, p, k);
            xv[b] = make_double2(0.0, 0.0);
            if (e < 64 * n && p < pv) xv[b] = __ldg(Xg + gidx(r, p0, p, k));
        }
    };
    // the epilogue's operand slots lie inside the X digit images (no room after them)
    const bool rs_in_x = a.rstage_off < 6 * a.aimg_bytes + 6 * a.ximg_bytes;
    auto stage = [&]() {
        // K padding (k >= n) of every digit image: zero again when the epilogue's
        // staging area may have overwritten it
        for (int w = tid; rs_in_x && w < 6 * 128 * (Kp - n); w += OZ_THREADS) {
            const int img = w / (128 * (Kp - n)), rem = w - img * 128 * (Kp - n);
            const int row = rem & 127, k = n + (rem >> 7);
            *reinterpret_cast<uint16_t *>(Ximg + img * a.ximg_bytes +
                                          kmaj_off_b16(row, k, lboX, sboX)) = 0;
        }
#pragma unroll
        for (int b = 0; b < OZ_EL; ++b) {
            const int e = tid + OZ_THREADS * b;
            if (e >= 64 * n) continue;
            int p, k;
            coord(e, p, k);
            uint32_t nr, ni;
            const uint64_t Fr = fixed48(xv[b].x, eX, nr);
            const uint64_t Fi = fixed48(xv[b].y, eX, ni);
            const uint32_t o = kmaj_off_b16(2 * p, k, lboX, sboX);    // row 2p; 2p+1 is +16 B
#pragma unroll
            for (int t = 0; t < 6; ++t) {
                unsigned char *img = Ximg + t * a.ximg_bytes;
                *reinterpret_cast<uint16_t *>(img + o) = digit_bf16(Fr, t, nr);
                *reinterpret_cast<uint16_t *>(img + o + 16) = digit_bf16(Fi, t, ni);
            }
        }
        fence_proxy_async_smem();
    };
    // 21 digit-pair GEMMs: accumulators 0..2 hold t + u = 0, 1, 2; accumulator
    // 3 takes t + u = 5, then 4, then 3, each group entered with D = AB + D/256
    auto issue = [&]() {
        tc_fence_after();
        const uint32_t xb = smem_u32(Ximg), ab = smem_u32(Aimg);
        auto pair = [&](uint32_t acc, int t, int u, bool first, bool scaled) {
            for (int s = 0; s < ksteps; ++s) {
                const uint64_t ad = smem_desc(xb + t * a.ximg_bytes + 2u * lboX * s, lboX, sboX);
                const uint64_t bd = smem_desc(ab + u * a.aimg_bytes + 256u * s, 128u,
                                              (uint32_t)a.sboAd);
                if (s == 0 && scaled) mma_bf16_scaled8(acc, ad, bd, idesc);
                else mma_bf16(acc, ad, bd, idesc, (first && s == 0) ? 0u : 1u);
            }
        };
        for (int d = 0; d < 3; ++d) {
            const uint32_t acc = tmem + (uint32_t)(d * Np);
            for (int t = 0; t <= d; ++t) pair(acc, t, d - t, t == 0, false);
        }
        const uint32_t acc3 = tmem + (uint32_t)(3 * Np);
        for (int d = 5; d >= 3; --d)
            for (int t = 0; t <= d; ++t) pair(acc3, t, d - t, d == 5 && t == 0, d < 5 && t == 0);
        mma_commit(&mbar_mma);
    };

    // epilogue: TMEM lane m = 32 (warp & 3) + lane is row (p, c); the four
    // warps of a lane quadrant take 8-column chunks in turn
    const int q = warp & 3, quarter = warp >> 2;
    const int m = 32 * q + lane;
    const int pl = m >> 1, cc = m & 1;
    auto epilogue = [&](int64_t t) {
        int64_t r, p0;
        int pv;
        tile_base(t, r, p0, pv);
        const bool live = pl < pv;
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
        // the values this lane updates: slot 4 c + t2 holds column 8 quarter + 32 c + 2 t2 + cc
        {
            int slot = 0;
            for (int i0 = 8 * quarter; i0 < n; i0 += 32)
                for (int t2 = 0; t2 < 4; ++t2, ++slot) {
                    const int i = i0 + 2 * t2 + cc;
                    if (!live || i >= n || in_mode == OZ_IN_ZERO) continue;
                    const int64_t g = gidx(r, p0, pl, i);
                    const void *src = in_mode == OZ_IN_B ? (const void *)(Bg + g)
                                                          : (const void *)(Rin + g);
                    cp_async16(Rs + ((size_t)slot * OZ_THREADS + tid) * 16, src);
                }
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        int slot = 0;
        for (int i0 = 8 * quarter; i0 < n; i0 += 32) {
            float sh[8], sl[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) sh[j] = sl[j] = 0.f;
            for (int d = 3; d >= 0; --d) {
                uint32_t va[8], vb[8];
                tmem_ld8(trow + (uint32_t)(d * Np + i0), va);
                tmem_ld8(trow + (uint32_t)(d * Np + n + i0), vb);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float av = __uint_as_float(va[j]);
                    float pb = __shfl_xor_sync(0xffffffffu, __uint_as_float(vb[j]), 1);
                    if (cc == 0) pb = -pb;
                    float vh, vlo;
                    two_sum(av, pb, vh, vlo);                 // exact complex recombination
                    sh[j] *= 0.00390625f;                      // Horner step: S = S / 256 + v
                    sl[j] *= 0.00390625f;
                    df_add(sh[j], sl[j], vh, vlo);
                }
            }
            cp_async_wait_all();
            // lane c keeps columns i0 + 2 t2 + c: exchange halves of the pairs
#pragma unroll
            for (int t2 = 0; t2 < 4; ++t2, ++slot) {
                const int j0 = 2 * t2, j1 = 2 * t2 + 1;
                const float send_h = cc == 0 ? sh[j1] : sh[j0];
                const float send_l = cc == 0 ? sl[j1] : sl[j0];
                const float rh = __shfl_xor_sync(0xffffffffu, send_h, 1);
                const float rl = __shfl_xor_sync(0xffffffffu, send_l, 1);
                // (re, im) of column i as FP32 pairs, scaled by 2^escale
                float reh = cc == 0 ? sh[j0] : rh, rel = cc == 0 ? sl[j0] : rl;
                float imh = cc == 0 ? rh : sh[j1], iml = cc == 0 ? rl : sl[j1];
                reh = ldexpf(reh, escale); rel = ldexpf(rel, escale);
                imh = ldexpf(imh, escale); iml = ldexpf(iml, escale);
                const int i = i0 + 2 * t2 + cc;
                if (!live || i >= n) continue;
                const int64_t g = gidx(r, p0, pl, i);
                const unsigned char *sv = Rs + ((size_t)slot * OZ_THREADS + tid) * 16;
                // base: B (FP64, split into FP32 pairs by integer operations; sigma is
                // folded into the first mode's digits), R pairs, or zero
                float xr = 0.f, lr = 0.f, xi = 0.f, li = 0.f;
                if (in_mode == OZ_IN_B) {
                    const double2 bv = *reinterpret_cast<const double2 *>(sv);
                    split_double(bv.x, xr, lr);
                    split_double(bv.y, xi, li);
                    xr *= a.bsign; lr *= a.bsign; xi *= a.bsign; li *= a.bsign;
                } else if (in_mode == OZ_IN_PAIRS) {
                    const float4 rv = *reinterpret_cast<const float4 *>(sv);
                    xr = rv.x; xi = rv.y; lr = rv.z; li = rv.w;
                }
                df_add(xr, lr, vsign * reh, vsign * rel);
                df_add(xi, li, vsign * imh, vsign * iml);
                if (out_mode == OZ_OUT_C64)
                    Rc64[g] = make_float2(xr + lr, xi + li);
                else if (out_mode == OZ_OUT_C128)
                    Rc128[g] = make_double2((double)xr + (double)lr, (double)xi + (double)li);
                else
                    Rout[g] = make_float4(xr, xi, lr, li);
            }
        }
    };

    const int64_t G = gridDim.x;
    int64_t tile = blockIdx.x;
    bool pending = false;
    if (tile < ntile && !s_fail) fetch(tile);
    __syncthreads();                         // digit images zeroed, A images resident
    for (; tile < ntile && !s_fail; tile += G) {
        stage();
        __syncthreads();
        if (tid == 0) issue();
        pending = true;
        if (tile + G < ntile) fetch(tile + G);
        if (!mbar_wait(&mbar_mma, phase)) s_fail = 1;
        phase ^= 1u;
        pending = false;
        tc_fence_after();
        epilogue(tile);
        tc_fence_before();
        __syncthreads();
    }
    if (pending && !mbar_wait(&mbar_mma, phase)) s_fail = 1;
    if (s_fail && tid == 0) atomicOr(&a.flags->err, ERRBIT_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

cudaError_t launch_resid_oz(const OzArgs &a, int grid, size_t smem, cudaStream_t st) {
    if (a.n < 8 || a.n > 64) return cudaErrorInvalidValue;
    if (a.mode1)
        k_resid_oz<1><<<grid, OZ_THREADS, smem, st>>>(a);
    else
        k_resid_oz<0><<<grid, OZ_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

// max(|re|, |im|) of a complex128 tensor into flags->xlast (float bits): the
// digit scale of the next pass's input
__global__ void k_maxabs(const double2 *x, int64_t count, DevFlags *flags) {
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, cabsmax(x[i]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&flags->xlast, m);
}

cudaError_t launch_maxabs(const void *x, int64_t count, DevFlags *flags, int num_sms,
                          cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(&flags->xlast, 0, sizeof(unsigned), st);
    if (e != cudaSuccess || count <= 0) return e;
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, (int64_t)num_sms * 8);
    k_maxabs<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<const double2 *>(x), count,
                                               flags);
    return cudaGetLastError();
}

cudaError_t resid_oz_init_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k_resid_oz<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TC_SMEM_MAX);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_resid_oz<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                TC_SMEM_MAX);
}

}  // namespace sylv
