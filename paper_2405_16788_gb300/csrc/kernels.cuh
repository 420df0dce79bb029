// Device helpers for the query kernels: the regularized kernel factor, the far
// test, compensated sums and warp-aggregated atomics.
#pragma once

#include "common.cuh"

namespace dip {

// Floats per node moment row: 3 per channel, padded to whole float4s.
__host__ __device__ constexpr int srow(int cp) { return (3 * cp + 3) & ~3; }

// rho(t) = erf(t) - (2t/sqrt(pi)) exp(-t^2)  (Sec. 4.1, eq. regularized_poisson).
// Above kTCut, 1 - rho < 1e-8 and rho rounds to 1 in float.  Below kTSeries
// the two terms cancel, so rho(t)/t^3 is taken from its Maclaurin series,
// obtained by integrating rho'(t) = (4/sqrt(pi)) t^2 exp(-t^2) term by term:
//   rho(t)/t^3 = (4/sqrt(pi)) sum_k (-1)^k t^(2k) / (k! (2k+3)).
// Seven terms leave a relative error below 1e-8 at t = 0.5.
constexpr float kTCut = 4.5f;
constexpr float kTSeries = 0.5f;
constexpr float kTwoOverSqrtPi = 1.1283791670955126f;
constexpr float kSer0 = 0.7522527780636751f;
constexpr float kSer1 = -0.45135166683820505f;
constexpr float kSer2 = 0.16119702387078752f;
constexpr float kSer3 = -0.0417918210035375f;
constexpr float kSer4 = 0.008548327023450852f;
constexpr float kSer5 = -0.0014466399578147598f;
constexpr float kSer6 = 0.00020895910501768752f;

// rho(d / eps) / d^3 for d^2 = d2 > 0 and inv_eps = 1/eps (+inf for eps = 0).
__device__ __forceinline__ float rho_over_d3(float d2, float inv_eps) {
    const float inv_d = rsqrtf(d2);
    const float inv_d3 = inv_d * inv_d * inv_d;
    const float t = d2 * inv_d * inv_eps;
    if (t >= kTCut) return inv_d3;
    const float u = t * t;
    if (t < kTSeries) {
        float p = kSer6;
        p = fmaf(p, u, kSer5);
        p = fmaf(p, u, kSer4);
        p = fmaf(p, u, kSer3);
        p = fmaf(p, u, kSer2);
        p = fmaf(p, u, kSer1);
        p = fmaf(p, u, kSer0);
        return p * (inv_eps * inv_eps * inv_eps);
    }
    const float rho = erff(t) - kTwoOverSqrtPi * t * __expf(-u);
    return rho * inv_d3;
}

// Kahan-compensated add: s + (c) tracks the sum, c holds the lost low part
// with the sign convention sum = s - c.
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// Sum V per-lane values over the warp and add the V totals to dst[0..V) with
// as few shuffles and atomics as possible: halve the vector across lane pairs
// while V is even (a reduce-scatter), finish the odd remainder with a
// butterfly, then one lane per group issues the atomics for its slice.
// Must be called by all 32 lanes.
template <int V>
__device__ __forceinline__ void warp_reduce_add(float (&v)[V], float* dst, int lane) {
    constexpr int H = (V % 2) ? 0 : (V % 4) ? 1 : (V % 8) ? 2 : (V % 16) ? 3 : (V % 32) ? 4 : 5;
    int base = 0;
#pragma unroll
    for (int s = 0; s < H; ++s) {
        const int off = 16 >> s;
        const int half = V >> (s + 1);
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const float send = up ? v[j] : v[j + half];
            const float keep = up ? v[j + half] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
        if (up) base += half;
    }
    constexpr int VR = V >> H;
#pragma unroll
    for (int off = 16 >> H; off > 0; off >>= 1) {
#pragma unroll
        for (int j = 0; j < VR; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
    }
    if ((lane & ((32 >> H) - 1)) == 0) {
#pragma unroll
        for (int j = 0; j < VR; ++j)
            if (v[j] != 0.0f) atomicAdd(dst + base + j, v[j]);
    }
}

}  // namespace dip
