// Complex arithmetic and small helpers shared by the sm_103a kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

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

// 1 / d in FP64 with Smith's scaling
__device__ __forceinline__ double2 crecip(double2 d) {
    double2 q;
    if (fabs(d.y) <= fabs(d.x)) {
        double r = d.y / d.x;
        double inv = 1.0 / (d.x + d.y * r);
        q.x = inv;
        q.y = -r * inv;
    } else {
        double r = d.x / d.y;
        double inv = 1.0 / (d.x * r + d.y);
        q.x = r * inv;
        q.y = -inv;
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

// 1 / d in FP64 for a diagonal sum d: `s` is a power of two chosen at plan
// time so that |s*d|^2 neither overflows nor underflows for any diagonal sum
// of the plan; 1/d = s * conj(s*d) / |s*d|^2, with the correctly rounded FP64
// reciprocal __drcp_rn.
__device__ __forceinline__ double2 crecip_scaled(double dx, double dy, double s) {
    const double ux = dx * s, uy = dy * s;
    const double r = __drcp_rn(fma(ux, ux, uy * uy)) * s;
    return make_double2(ux * r, -uy * r);
}

}  // namespace sylv
