// Device helpers for the query kernels: the regularized kernel factor, the far
// test, compensated sums and warp-aggregated atomics.
#pragma once

#include "common.cuh"

namespace dip {

// Floats per node moment row: 3 per channel, padded to whole float4s.
__host__ __device__ constexpr int srow(int cp) { return (3 * cp + 3) & ~3; }
// bf16 values per row of the bf16 moment copy: 3 per channel, padded to whole
// 16-byte vectors.
__host__ __device__ constexpr int srow16(int cp) { return (3 * cp + 7) & ~7; }

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

// Desingularized radial factor 1 / max(d, delta)^3 with delta = 1/inv_eps (the
// ablation kernel with a cutoff in the denominator); inv_eps = +inf gives
// 1/d^3.
__device__ __forceinline__ float desing_over_d3(float d2, float inv_eps) {
    const float inv_d = rsqrtf(d2);
    const float t = d2 * inv_d * inv_eps;  // d / delta
    if (t >= 1.0f) return inv_d * inv_d * inv_d;
    return inv_eps * inv_eps * inv_eps;
}

// The radial factor of the tree's kernel (kernel is uniform across a launch).
__device__ __forceinline__ float radial_over_d3(float d2, float inv_eps, int kernel) {
    return kernel == 0 ? rho_over_d3(d2, inv_eps) : desing_over_d3(d2, inv_eps);
}

// Bring the bytes [p, p + bytes) into L1 ahead of their loads: lane i
// prefetches the i-th 128-byte line of the range (bytes <= 32 lines), one
// instruction for the warp.  The forward reads an opened leaf's point records
// and attribute rows one point after another; prefetched, they come from L1
// (value forward -2%, gradient forward -3%; the attribute adjoint, with its
// heavier L1 traffic, lost 5%).
__device__ __forceinline__ void prefetch_l1(const void* p, int bytes, int lane) {
    const uintptr_t b = reinterpret_cast<uintptr_t>(p);
    const uintptr_t line = (b & ~uintptr_t(127)) + 128u * (uintptr_t)lane;
    if (line < b + (uintptr_t)bytes) asm volatile("prefetch.global.L1 [%0];" ::"l"(line));
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

// Adjoint warp sums without data-dependent selects.  Within a chunk of CH
// channels (1, 2 or 4) the lanes split the channels by their lane bits: after
// exchanging with lane^16 (and lane^8 for CH = 4) a lane holds the running
// sums of exactly one channel, kept(lane); a butterfly over the remaining lane
// bits completes that channel's sum, and the lowest lane of each group issues
// the atomics.  Because the channel a lane keeps or hands on at each exchange
// depends only on its lane bits, the upstream gradient is permuted once per
// packet (lane_channel_order) and every exchange is a plain shuffle and add.
//
// lane_channel_order: ord[0] = the channel kept to the end, ord[1] = the one
// handed to lane^8 (CH = 4), then the two handed to lane^16.
template <int CH>
__device__ __forceinline__ void lane_channel_order(int lane, int (&ord)[CH]) {
    if constexpr (CH == 4) {
        const int p0 = (lane & 16) ? 2 : 0, b3 = (lane >> 3) & 1;
        ord[0] = p0 + b3;        // kept
        ord[1] = p0 + 1 - b3;    // kept at the first exchange, handed on at the second
        ord[2] = ord[0] ^ 2;     // handed to lane^16
        ord[3] = ord[1] ^ 2;
    } else if constexpr (CH == 2) {
        ord[0] = (lane & 16) ? 1 : 0;
        ord[1] = ord[0] ^ 1;
    } else {
        ord[0] = 0;
    }
}

// Lanes in a reduction group of the final channel: the lowest one owns it.
template <int CH>
__device__ __forceinline__ bool lane_owns(int lane) {
    return (lane & (CH == 4 ? 7 : CH == 2 ? 15 : 31)) == 0;
}

// Far node: gp = this chunk's gradient in lane_channel_order; adds
// sum over lanes of v (x) g^c into dst[3c + axis] for the chunk's channels.
template <int CH>
__device__ __forceinline__ void adjoint_far_reduce(float vx, float vy, float vz, const float* gp,
                                                   float* dst, int kept, int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    float a0 = vx * gp[0], a1 = vy * gp[0], a2 = vz * gp[0];
    if constexpr (CH == 4) {
        float a3 = vx * gp[1], a4 = vy * gp[1], a5 = vz * gp[1];
        a0 += __shfl_xor_sync(FULL, vx * gp[2], 16);
        a1 += __shfl_xor_sync(FULL, vy * gp[2], 16);
        a2 += __shfl_xor_sync(FULL, vz * gp[2], 16);
        a3 += __shfl_xor_sync(FULL, vx * gp[3], 16);
        a4 += __shfl_xor_sync(FULL, vy * gp[3], 16);
        a5 += __shfl_xor_sync(FULL, vz * gp[3], 16);
        a0 += __shfl_xor_sync(FULL, a3, 8);
        a1 += __shfl_xor_sync(FULL, a4, 8);
        a2 += __shfl_xor_sync(FULL, a5, 8);
    } else if constexpr (CH == 2) {
        a0 += __shfl_xor_sync(FULL, vx * gp[1], 16);
        a1 += __shfl_xor_sync(FULL, vy * gp[1], 16);
        a2 += __shfl_xor_sync(FULL, vz * gp[1], 16);
    }
    // The remaining lane bits (B and below) finish the three axis sums as a
    // reduce-scatter over four slots (x, y, z, 0): bit B splits them {x, y} /
    // {z, 0}, bit B/2 one slot each, a butterfly does the rest; one lane per
    // slot then adds it.
    constexpr int B = CH == 4 ? 4 : CH == 2 ? 8 : 16;
    const bool hb = (lane & B) != 0, lb = (lane & (B / 2)) != 0;
    const float k0 = (hb ? a2 : a0) + __shfl_xor_sync(FULL, hb ? a0 : a2, B);
    const float k1 = (hb ? 0.0f : a1) + __shfl_xor_sync(FULL, hb ? a1 : 0.0f, B);
    float r = (lb ? k1 : k0) + __shfl_xor_sync(FULL, lb ? k0 : k1, B / 2);
#pragma unroll
    for (int off = B / 4; off > 0; off >>= 1) r += __shfl_xor_sync(FULL, r, off);
    const int axis = (hb ? 2 : 0) + (lb ? 1 : 0);
    if ((lane & (B / 2 - 1)) == 0 && axis < 3 && r != 0.0f) atomicAdd(dst + 3 * kept + axis, r);
}

// Opened-leaf points, two at once: ka, kb the lanes' kernel values for
// points a and b; adds sum over lanes of ka g^c into dst_a[c] and of kb g^c
// into dst_a[stride + c] (b's row; skipped when !two).  The channel exchanges
// are those of adjoint_far_reduce (one value per channel instead of three);
// bit B then splits the pair (one shuffle) where each point alone would need a
// full butterfly: 9 shuffles for two points at CH = 4 instead of 12.
template <int CH>
__device__ __forceinline__ void adjoint_point_pair_reduce(float ka, float kb, const float* gp,
                                                          float* dst_a, int stride, bool two,
                                                          int kept, int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    float a0 = ka * gp[0], b0 = kb * gp[0];
    if constexpr (CH == 4) {
        float a1 = ka * gp[1], b1 = kb * gp[1];
        a0 += __shfl_xor_sync(FULL, ka * gp[2], 16);
        a1 += __shfl_xor_sync(FULL, ka * gp[3], 16);
        b0 += __shfl_xor_sync(FULL, kb * gp[2], 16);
        b1 += __shfl_xor_sync(FULL, kb * gp[3], 16);
        a0 += __shfl_xor_sync(FULL, a1, 8);
        b0 += __shfl_xor_sync(FULL, b1, 8);
    } else if constexpr (CH == 2) {
        a0 += __shfl_xor_sync(FULL, ka * gp[1], 16);
        b0 += __shfl_xor_sync(FULL, kb * gp[1], 16);
    }
    constexpr int B = CH == 4 ? 4 : CH == 2 ? 8 : 16;
    const bool hb = (lane & B) != 0;
    float r = (hb ? b0 : a0) + __shfl_xor_sync(FULL, hb ? a0 : b0, B);
#pragma unroll
    for (int off = B / 2; off > 0; off >>= 1) r += __shfl_xor_sync(FULL, r, off);
    if ((lane & (B - 1)) == 0 && (two || !hb) && r != 0.0f)
        atomicAdd(dst_a + (hb ? stride : 0) + kept, r);
}

// Generalized forms of the far-node reduction (a vector per channel) and of a
// one-point reduction (a scalar per channel): the lane supplies its values
// already in lane_channel_order (v[3i + k] for channel ord[i], axis k).
template <int CH>
__device__ __forceinline__ void adjoint_vec_reduce(const float (&v)[3 * CH], float* dst, int kept,
                                                   int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    float a0 = v[0], a1 = v[1], a2 = v[2];
    if constexpr (CH == 4) {
        float a3 = v[3] + __shfl_xor_sync(FULL, v[9], 16);
        float a4 = v[4] + __shfl_xor_sync(FULL, v[10], 16);
        float a5 = v[5] + __shfl_xor_sync(FULL, v[11], 16);
        a0 += __shfl_xor_sync(FULL, v[6], 16);
        a1 += __shfl_xor_sync(FULL, v[7], 16);
        a2 += __shfl_xor_sync(FULL, v[8], 16);
        a0 += __shfl_xor_sync(FULL, a3, 8);
        a1 += __shfl_xor_sync(FULL, a4, 8);
        a2 += __shfl_xor_sync(FULL, a5, 8);
    } else if constexpr (CH == 2) {
        a0 += __shfl_xor_sync(FULL, v[3], 16);
        a1 += __shfl_xor_sync(FULL, v[4], 16);
        a2 += __shfl_xor_sync(FULL, v[5], 16);
    }
    // The remaining lane bits (B and below) finish the three axis sums as a
    // reduce-scatter over four slots (x, y, z, 0): bit B splits them {x, y} /
    // {z, 0}, bit B/2 one slot each, a butterfly does the rest; one lane per
    // slot then adds it.
    constexpr int B = CH == 4 ? 4 : CH == 2 ? 8 : 16;
    const bool hb = (lane & B) != 0, lb = (lane & (B / 2)) != 0;
    const float k0 = (hb ? a2 : a0) + __shfl_xor_sync(FULL, hb ? a0 : a2, B);
    const float k1 = (hb ? 0.0f : a1) + __shfl_xor_sync(FULL, hb ? a1 : 0.0f, B);
    float r = (lb ? k1 : k0) + __shfl_xor_sync(FULL, lb ? k0 : k1, B / 2);
#pragma unroll
    for (int off = B / 4; off > 0; off >>= 1) r += __shfl_xor_sync(FULL, r, off);
    const int axis = (hb ? 2 : 0) + (lb ? 1 : 0);
    if ((lane & (B / 2 - 1)) == 0 && axis < 3 && r != 0.0f) atomicAdd(dst + 3 * kept + axis, r);
}

template <int CH>
__device__ __forceinline__ void adjoint_scalar_reduce(const float (&v)[CH], float* dst, int kept,
                                                      int lane) {
    constexpr unsigned FULL = 0xffffffffu;
    float a0 = v[0];
    if constexpr (CH == 4) {
        const float a1 = v[1] + __shfl_xor_sync(FULL, v[3], 16);
        a0 += __shfl_xor_sync(FULL, v[2], 16);
        a0 += __shfl_xor_sync(FULL, a1, 8);
    } else if constexpr (CH == 2) {
        a0 += __shfl_xor_sync(FULL, v[1], 16);
    }
#pragma unroll
    for (int off = (CH == 4 ? 4 : CH == 2 ? 8 : 16); off > 0; off >>= 1)
        a0 += __shfl_xor_sync(FULL, a0, off);
    if (lane_owns<CH>(lane) && a0 != 0.0f) atomicAdd(dst + kept, a0);
}

}  // namespace dip
