// Reciprocal formats of the triangular sweep's diagonal sums (sweep.cu).
#pragma once

#include <cuda_runtime.h>

#include "cplx.cuh"

namespace sylv {

// The reciprocal of a diagonal sum is formed in FP64 in stage 1 and applied in
// the in-tile wavefront: as double2 on the FP64 path; on the FP32 path as the
// pair hi = fl32(1/den), lo = fl32(1/den - hi), so that the wavefront, which is
// latency-critical, issues no instruction on GB300's narrow FP64 pipe.
template <typename real> struct InvT;
template <> struct InvT<double> { using type = double2; };
template <> struct InvT<float> { using type = float4; };

__device__ __forceinline__ void store_inv(double2 r, double2 &o) { o = r; }
__device__ __forceinline__ void store_inv(double2 r, float4 &o) {
    const float hx = (float)r.x, hy = (float)r.y;
    o = make_float4(hx, hy, (float)(r.x - (double)hx), (float)(r.y - (double)hy));
}
__device__ __forceinline__ double2 apply_inv(double2 n, double2 v) {
    return make_double2(n.x * v.x - n.y * v.y, n.x * v.y + n.y * v.x);
}
__device__ __forceinline__ float2 apply_inv(float2 n, float4 v) {
    float tx = fmaf(n.x, v.z, -n.y * v.w);      // n * lo first, then n * hi
    float ty = fmaf(n.x, v.w, n.y * v.z);
    tx = fmaf(-n.y, v.y, tx);
    ty = fmaf(n.y, v.x, ty);
    return make_float2(fmaf(n.x, v.x, tx), fmaf(n.x, v.y, ty));
}

}  // namespace sylv
