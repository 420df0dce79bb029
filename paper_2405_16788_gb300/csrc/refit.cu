// Tree update of the node moments (Sec. 6.1, eq. farfield_dipole_features;
// Sec. 6.3: refreshed at the start of every iteration) and the second stage
// of the adjoint (Sec. 6.2; App. C, eq. farfield_features_gradient).
//
// Moments are stored as S_t^c = A~_t n~_t^c = sum_{m in t} A_m n_m mu_m^c, so the
// far field needs no division by A~_t and stage 2 needs no multiplication by
// A_m / A~_t: d mu_m^c = (A_m n_m) . sum_{t holding m} dS_t^c.
#include "kernels.cuh"
#include "tree.cuh"

namespace dip {
namespace {

template <typename AT>
__device__ __forceinline__ float to_f(AT v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename AT>
__device__ __forceinline__ AT from_f(float v);
template <>
__device__ __forceinline__ float from_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Bottom-up without a pass per level.  The subtree of node t is the preorder
// range [t, skip[t]), so with P[u] = the sum of the leaf moments of the nodes
// before u in preorder, an internal node's moment is S_t = P[skip[t]] - P[t].
// The leaf moments are float sums over their points; P is taken in 64-bit
// fixed point with one scale 2^k per moment column, chosen from the column's
// largest leaf moment so that no partial sum can overflow.  Integer sums are
// exact and do not depend on the order of the additions, so the result does
// not depend on how the scan is split across threads; the only roundings are
// each leaf moment's conversion to a multiple of 2^-k (exact unless it is
// below 2^-18 of the column's largest) and each node's difference back to
// float.  Four launches: leaves (and the column maxima), tile sums (the last
// tile to finish scans them), the prefix P, the internal nodes.
constexpr int kRefitThreads = 256;
constexpr int kRefitPer = 4;  // consecutive nodes per thread in the scan passes
constexpr int kRefitTile = kRefitThreads * kRefitPer;
constexpr int kFixChunk = 12;  // moment columns per register block
constexpr int kFixNonFinite = 0x7fffffff;

// Leading dimension of the column-major prefix P: nn + 1 rows rounded up to 4.
inline int64_t fix_ld(int64_t nn) { return (nn + 1 + 3) & ~int64_t(3); }

// f * 2^k for |k| <= 252 in two exact power-of-two steps.
__device__ __forceinline__ float scale_pow2(float f, int k) {
    const int a = k / 2, b = k - a;
    return __fmul_rn(__fmul_rn(f, __int_as_float((a + 127) << 23)), __int_as_float((b + 127) << 23));
}

// Column scale exponent from the bits of the column's largest |leaf moment|:
// every leaf moment is below 2^e, so with k = 61 - lg - e (nn < 2^lg) each
// scaled moment is below 2^(61 - lg) and any sum of nn of them below 2^61.
// Finite floats and nn < 2^31 keep k within [-99, 186].
__device__ __forceinline__ int fixed_exp(unsigned maxbits, int lg) {
    if (maxbits == 0u) return 0;
    if (maxbits >= 0x7f800000u) return kFixNonFinite;
    const int e = (int)(maxbits >> 23) - 126;
    return min(max(61 - lg - e, -200), 200);
}

// v 2^k rounded to the nearest integer (ties to even), in integer arithmetic
// (the 64-bit conversion instructions run at the FP64 rate).  The scale keeps
// the result below 2^61, so the left shift is at most 37.
__device__ __forceinline__ long long to_fixed(float v, int k) {
    if (k == kFixNonFinite) return 0ll;
    const uint32_t u = __float_as_uint(v);
    const uint32_t ex = (u >> 23) & 0xffu;
    const uint32_t mant = ex ? ((u & 0x7fffffu) | 0x800000u) : (u & 0x7fffffu);
    const int sh = (ex ? (int)ex : 1) - 150 + k;  // v = mant 2^(max(ex, 1) - 150)
    uint64_t r;
    if (sh >= 0) {
        r = (uint64_t)mant << sh;
    } else if (sh < -24) {
        r = 0;  // below 1/4
    } else {
        const int rs = -sh;
        const uint32_t q = mant >> rs, rem = mant & ((1u << rs) - 1u), half = 1u << (rs - 1);
        r = q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
    }
    return (u >> 31) ? -(long long)r : (long long)r;
}

// d 2^-k rounded to float (ties to even), in integer arithmetic.
__device__ __forceinline__ float from_fixed(long long d, int k) {
    if (k == kFixNonFinite) return __int_as_float(0x7fffffff);
    if (d == 0) return 0.0f;
    const uint64_t a = d < 0 ? (uint64_t)(-d) : (uint64_t)d;
    const int msb = 63 - __clzll((long long)a);
    uint32_t q = (uint32_t)a;
    int e = 0;
    if (msb > 23) {
        const int rs = msb - 23;
        q = (uint32_t)(a >> rs);
        const uint64_t rem = a & ((1ull << rs) - 1ull), half = 1ull << (rs - 1);
        q += (rem > half || (rem == half && (q & 1u))) ? 1u : 0u;
        e = rs;
    }
    const float f = __uint2float_rn(q);  // exact: q <= 2^24
    return scale_pow2(d < 0 ? -f : f, e - k);
}

// Columns j0 .. j0 + V of row t of S (rows of SR floats, 16-byte aligned;
// j0 is a multiple of 12 or 0, and the float4s read stay inside the row).
template <int SR, int V>
__device__ __forceinline__ void load_cols(const float* __restrict__ S, int64_t t, int j0,
                                          float (&x)[V]) {
    const float4* p = reinterpret_cast<const float4*>(S + t * SR + j0);
#pragma unroll
    for (int i = 0; i < (V + 3) / 4; ++i) {
        const float4 q = p[i];
        if (4 * i < V) x[4 * i] = q.x;
        if (4 * i + 1 < V) x[4 * i + 1] = q.y;
        if (4 * i + 2 < V) x[4 * i + 2] = q.z;
        if (4 * i + 3 < V) x[4 * i + 3] = q.w;
    }
}

__device__ __forceinline__ int bits_of(int64_t nn) {
    return 64 - __clzll((long long)nn);
}

// Leaves, one thread per point (Morton order): the thread gathers its point's
// attributes into mu and stages them with A_m n_m in shared memory; the
// thread at each leaf's first point sums the leaf's moments in float, point by
// point (a leaf running past the block's points reads the rest from global
// memory).  The largest |moment| of each column goes to cmax.
constexpr int kLeafThreads = 256;

template <int CP, typename AT>
__global__ void __launch_bounds__(kLeafThreads) k_refit_leaves(
    int64_t n, const PointRec* __restrict__ pts, const uint32_t* __restrict__ perm,
    const int32_t* __restrict__ leaf_of, const int32_t* __restrict__ count,
    const AT* __restrict__ attrs, int C, int G, AT* __restrict__ mu, float* __restrict__ S,
    unsigned* __restrict__ cmax) {
    constexpr int SR = srow(CP);
    constexpr int CH = CP < 4 ? CP : 4;  // channels per chunk
    constexpr int RW = CH + 4;           // staged row: CH attributes, then A n, A
    __shared__ float row[kLeafThreads * RW];
    __shared__ unsigned smax[3 * CP];
    for (int j = threadIdx.x; j < 3 * CP; j += blockDim.x) smax[j] = 0u;
    const int tid = threadIdx.x;
    for (int64_t m0 = (int64_t)blockIdx.x * kLeafThreads; m0 < n;
         m0 += (int64_t)gridDim.x * kLeafThreads) {
        const int64_t m = m0 + tid;
        const bool valid = m < n;
        const int64_t o = valid ? (int64_t)perm[m] : 0;
        const float4 w = valid ? pts[m].w : make_float4(0.f, 0.f, 0.f, 0.f);
        const int32_t leaf = valid ? leaf_of[m] : -1;
        const bool head = valid && (m == 0 || leaf_of[m - 1] != leaf);
        const int k = head ? count[leaf] : 0;
#pragma unroll 1
        for (int c0 = 0; c0 < CP; c0 += CH) {
            __syncthreads();  // the previous chunk's sums have read the rows
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const AT a = (valid && c0 + c < C) ? attrs[o * C + c0 + c] : from_f<AT>(0.0f);
                if (valid) mu[m * CP + c0 + c] = a;
                row[tid * RW + c] = to_f<AT>(a);
            }
            row[tid * RW + CH] = w.x;
            row[tid * RW + CH + 1] = w.y;
            row[tid * RW + CH + 2] = w.z;
            row[tid * RW + CH + 3] = w.w;
            __syncthreads();
            if (head) {
                float sacc[3 * CH];
#pragma unroll
                for (int j = 0; j < 3 * CH; ++j) sacc[j] = 0.0f;
                for (int i = 0; i < k; ++i) {
                    float v[CH], wx, wy, wz, wa;
                    if (tid + i < kLeafThreads) {
                        const float* r = row + (tid + i) * RW;
#pragma unroll
                        for (int c = 0; c < CH; ++c) v[c] = r[c];
                        wx = r[CH]; wy = r[CH + 1]; wz = r[CH + 2]; wa = r[CH + 3];
                    } else {  // past the block's points
                        const int64_t mi = m + i;
                        const int64_t oi = perm[mi];
#pragma unroll
                        for (int c = 0; c < CH; ++c)
                            v[c] = c0 + c < C ? to_f<AT>(attrs[oi * C + c0 + c]) : 0.0f;
                        const float4 wi = pts[mi].w;
                        wx = wi.x; wy = wi.y; wz = wi.z; wa = wi.w;
                    }
#pragma unroll
                    for (int c = 0; c < CH; ++c) {
                        if (c0 + c < G) {  // S^c = sum A n mu^c (eq. farfield_dipole_features)
                            sacc[3 * c] = fmaf(wx, v[c], sacc[3 * c]);
                            sacc[3 * c + 1] = fmaf(wy, v[c], sacc[3 * c + 1]);
                            sacc[3 * c + 2] = fmaf(wz, v[c], sacc[3 * c + 2]);
                        } else {  // no foreshortening term: M^c = sum A mu^c in the first slot
                            sacc[3 * c] = fmaf(wa, v[c], sacc[3 * c]);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < 3 * CH; ++j) {
                    S[(int64_t)leaf * SR + 3 * c0 + j] = sacc[j];
                    const unsigned bits = __float_as_uint(fabsf(sacc[j]));
                    if (bits) atomicMax(&smax[3 * c0 + j], bits);
                }
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < 3 * CP; j += blockDim.x)
        if (smax[j]) atomicMax(&cmax[j], smax[j]);
}

// Sum of V int64 values over the block (kRefitThreads threads); the totals
// land in tot[] of thread 0 only.  red must hold kRefitThreads / 32 * V.
template <int V>
__device__ __forceinline__ void block_sum_i64(long long (&v)[V], long long* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < V; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < V; ++j) red[warp * V + j] = v[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < V; ++j) {
            long long s = 0;
            for (int w = 0; w < kRefitThreads / 32; ++w) s += red[w * V + j];
            v[j] = s;
        }
    }
    __syncthreads();
}

// Exclusive prefix of V int64 values over the block's threads in order.
template <int V>
__device__ __forceinline__ void block_exclusive_i64(long long (&v)[V], long long* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long inc[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        inc[j] = v[j];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, inc[j], o);
            if (lane >= o) inc[j] += u;
        }
    }
    if (lane == 31) {
#pragma unroll
        for (int j = 0; j < V; ++j) red[warp * V + j] = inc[j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < V; ++j) {
        long long before = 0;
        for (int w = 0; w < warp; ++w) before += red[w * V + j];
        v[j] = before + inc[j] - v[j];
    }
    __syncthreads();
}

// Leaf flags of nodes base .. base + kRefitPer (base a multiple of 4; false
// past nn).
__device__ __forceinline__ void leaf_flags(const int32_t* __restrict__ is_leaf, int64_t nn,
                                           int64_t base, bool (&lf)[kRefitPer]) {
    static_assert(kRefitPer == 4, "one int4 per thread");
    if (base + 3 < nn) {
        const int4 q = *reinterpret_cast<const int4*>(is_leaf + base);
        lf[0] = q.x != 0; lf[1] = q.y != 0; lf[2] = q.z != 0; lf[3] = q.w != 0;
    } else {
#pragma unroll
        for (int r = 0; r < kRefitPer; ++r) lf[r] = base + r < nn && is_leaf[base + r] != 0;
    }
}

// Sum over the thread's kRefitPer nodes of their fixed-point leaf moments,
// columns j0 .. j0 + V.
template <int SR, int V>
__device__ __forceinline__ void thread_fixed_sum(const float* __restrict__ S, int64_t base,
                                                 const bool (&lf)[kRefitPer], int j0,
                                                 const int* sk, long long (&v)[V]) {
#pragma unroll
    for (int j = 0; j < V; ++j) v[j] = 0;
#pragma unroll
    for (int r = 0; r < kRefitPer; ++r) {
        if (!lf[r]) continue;
        float x[V];
        load_cols<SR, V>(S, base + r, j0, x);
#pragma unroll
        for (int j = 0; j < V; ++j) v[j] += to_fixed(x[j], sk[j0 + j]);
    }
}

// Tile b = nodes [b kRefitTile, (b + 1) kRefitTile), kRefitPer consecutive
// nodes per thread: the fixed-point sum of its leaf moments per column.  The
// last tile to finish (an arrival counter; no block waits for another) scans
// the tile sums into tile offsets, publishes the column exponents and clears
// cmax and the counter for the next refit.
template <int CP>
__global__ void __launch_bounds__(kRefitThreads) k_refit_tiles(
    int64_t nn, const int32_t* __restrict__ is_leaf, const float* __restrict__ S,
    unsigned* __restrict__ cmax, int* __restrict__ kexp, long long* __restrict__ tsum,
    unsigned* __restrict__ done) {
    constexpr int SR = srow(CP), NC = 3 * CP;
    constexpr int V = NC < kFixChunk ? NC : kFixChunk;
    __shared__ int sk[NC];
    __shared__ long long red[kRefitThreads / 32 * V];
    __shared__ bool last;
    const int lg = bits_of(nn);
    for (int j = threadIdx.x; j < NC; j += blockDim.x) sk[j] = fixed_exp(cmax[j], lg);
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRefitTile + (int64_t)threadIdx.x * kRefitPer;
    const int ntiles = gridDim.x;
    bool lf[kRefitPer];
    leaf_flags(is_leaf, nn, base, lf);
#pragma unroll 1
    for (int j0 = 0; j0 < NC; j0 += V) {
        long long v[V];
        thread_fixed_sum<SR, V>(S, base, lf, j0, sk, v);
        block_sum_i64<V>(v, red);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int j = 0; j < V; ++j) tsum[(int64_t)blockIdx.x * NC + j0 + j] = v[j];
        }
    }
    if (threadIdx.x == 0) {  // the only writer of this block's sums
        __threadfence();
        last = atomicAdd(done, 1u) == (unsigned)ntiles - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // exclusive scan of the tile sums: thread i takes a run of seg tiles
    const int seg = (ntiles + kRefitThreads - 1) / kRefitThreads;
    const int b0 = threadIdx.x * seg, b1 = min(b0 + seg, ntiles);
#pragma unroll 1
    for (int j0 = 0; j0 < NC; j0 += V) {
        long long v[V];
#pragma unroll
        for (int j = 0; j < V; ++j) v[j] = 0;
        for (int b = b0; b < b1; ++b) {
#pragma unroll
            for (int j = 0; j < V; ++j) v[j] += __ldcg(tsum + (int64_t)b * NC + j0 + j);
        }
        block_exclusive_i64<V>(v, red);
        for (int b = b0; b < b1; ++b) {
            long long* e = tsum + (int64_t)b * NC + j0;
            long long x[V];
#pragma unroll
            for (int j = 0; j < V; ++j) x[j] = __ldcg(e + j);  // all loads before the stores
#pragma unroll
            for (int j = 0; j < V; ++j) {
                e[j] = v[j];
                v[j] += x[j];
            }
        }
    }
    for (int j = threadIdx.x; j < NC; j += blockDim.x) {
        kexp[j] = sk[j];
        cmax[j] = 0u;
    }
    if (threadIdx.x == 0) *done = 0u;
}

// P for the tile's nodes (and P[nn], the total): the tile's offset plus the
// exclusive prefix inside the tile.  P is column-major with leading dimension
// ldP (a multiple of 4), so a thread's four nodes are 32 contiguous bytes of
// each column.
template <int CP>
__global__ void __launch_bounds__(kRefitThreads) k_refit_prefix(
    int64_t nn, int64_t ldP, const int32_t* __restrict__ is_leaf, const float* __restrict__ S,
    const int* __restrict__ kexp, const long long* __restrict__ toff, long long* __restrict__ P) {
    constexpr int SR = srow(CP), NC = 3 * CP;
    constexpr int V = NC < kFixChunk ? NC : kFixChunk;
    __shared__ int sk[NC];
    __shared__ long long red[kRefitThreads / 32 * V];
    for (int j = threadIdx.x; j < NC; j += blockDim.x) sk[j] = kexp[j];
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRefitTile + (int64_t)threadIdx.x * kRefitPer;
    bool lf[kRefitPer];
    leaf_flags(is_leaf, nn, base, lf);
#pragma unroll 1
    for (int j0 = 0; j0 < NC; j0 += V) {
        long long v[V];
        thread_fixed_sum<SR, V>(S, base, lf, j0, sk, v);
        block_exclusive_i64<V>(v, red);
        if (base >= nn) continue;
#pragma unroll
        for (int j = 0; j < V; ++j) {
            long long own[kRefitPer];
#pragma unroll
            for (int r = 0; r < kRefitPer; ++r)  // rows read above: L1 hits
                own[r] = lf[r] ? to_fixed(S[(base + r) * SR + j0 + j], sk[j0 + j]) : 0ll;
            long long* col = P + (int64_t)(j0 + j) * ldP;
            long long q0 = v[j] + toff[(int64_t)blockIdx.x * NC + j0 + j];
            const long long q1 = q0 + own[0], q2 = q1 + own[1], q3 = q2 + own[2];
            if (base + 3 < nn) {
                reinterpret_cast<longlong2*>(col + base)[0] = make_longlong2(q0, q1);
                reinterpret_cast<longlong2*>(col + base)[1] = make_longlong2(q2, q3);
            } else {
                const long long q[4] = {q0, q1, q2, q3};
#pragma unroll
                for (int r = 0; r < kRefitPer; ++r)
                    if (base + r < nn) col[base + r] = q[r];
            }
            const int64_t lastr = nn - 1 - base;  // the thread holding node nn - 1 writes P[nn]
            if (lastr >= 0 && lastr < kRefitPer)
                col[nn] = lastr == 0 ? q1 : lastr == 1 ? q2 : lastr == 2 ? q3 : q3 + own[3];
        }
    }
}

// Internal nodes: S_t = P[skip[t]] - P[t], back to float.
template <int CP>
__global__ void __launch_bounds__(128) k_refit_internal(
    int64_t nn, int64_t ldP, const int32_t* __restrict__ is_leaf, const int32_t* __restrict__ skip,
    const int* __restrict__ kexp, const long long* __restrict__ P, float* __restrict__ S) {
    constexpr int SR = srow(CP), NC = 3 * CP;
    __shared__ int sk[NC];
    for (int j = threadIdx.x; j < NC; j += blockDim.x) sk[j] = kexp[j];
    __syncthreads();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (is_leaf[t]) continue;
        int64_t e = skip[t];
        if (e < t || e > nn) e = t;  // only an imported, corrupt tree gets here
#pragma unroll 4
        for (int j = 0; j < NC; ++j) {
            const long long* col = P + (int64_t)j * ldP;
            S[t * SR + j] = from_fixed(col[e] - col[t], sk[j]);
        }
    }
}

// The bf16 copy of the moments (DIPOLE_BF16_MOMENTS): every value rounded to
// nearest even, padding columns 0.  Four values per thread, so that a warp
// reads and writes consecutive 16- and 8-byte pieces of the rows.
template <int CP>
__global__ void __launch_bounds__(256) k_moments_bf16(int64_t nn, const float* __restrict__ S,
                                                      uint16_t* __restrict__ S16) {
    constexpr int SR = srow(CP), SR16 = srow16(CP), NC = 3 * CP, QR = SR16 / 4;
    const int64_t total = nn * QR;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / QR;
        const int j = 4 * (int)(i - t * QR);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < SR) v = __ldg(reinterpret_cast<const float4*>(S + t * SR + j));
        const float f[4] = {v.x, v.y, v.z, v.w};
        unsigned short h[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            h[k] = j + k < NC ? __bfloat16_as_ushort(__float2bfloat16_rn(f[k])) : (unsigned short)0;
        uint2 out;
        out.x = (unsigned)h[0] | ((unsigned)h[1] << 16);
        out.y = (unsigned)h[2] | ((unsigned)h[3] << 16);
        *reinterpret_cast<uint2*>(S16 + t * SR16 + j) = out;
    }
}

// Stage 2 (eq. farfield_features_gradient): for each leaf, D^c = sum of dS^c
// over the leaf and its ancestors; each point of the leaf gets
// (A_m n_m) . D^c plus its opened-leaf term, written in the caller's order.
template <int CP>
__global__ void __launch_bounds__(128) k_stage2(
    int64_t nn, const PointRec* __restrict__ pts, const uint32_t* __restrict__ perm,
    const int32_t* __restrict__ first, const int32_t* __restrict__ count,
    const int32_t* __restrict__ is_leaf, const int32_t* __restrict__ parent,
    const float* __restrict__ dS, const float* __restrict__ dmu, int C, int G, int accumulate,
    float* __restrict__ grad) {
    constexpr int SR = srow(CP);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (!is_leaf[t]) continue;
        const int64_t f = first[t], k = count[t];
#pragma unroll 1
        for (int c0 = 0; c0 < CP; c0 += 4) {
            float D[12];
#pragma unroll
            for (int j = 0; j < 12; ++j) D[j] = 0.0f;
            for (int64_t u = t; u >= 0; u = parent[u]) {
#pragma unroll
                for (int j = 0; j < 12; ++j) {
                    if (3 * c0 + j >= 3 * CP) break;
                    D[j] += dS[u * SR + 3 * c0 + j];
                }
            }
            for (int64_t m = f; m < f + k; ++m) {
                const float4 w = pts[m].w;
                const int64_t o = perm[m];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int ch = c0 + c;
                    if (ch >= CP) break;
                    if (ch >= C) continue;
                    // channels without the foreshortening term: M^c = sum A mu^c
                    float v = ch < G ? fmaf(w.x, D[3 * c], fmaf(w.y, D[3 * c + 1], w.z * D[3 * c + 2]))
                                     : w.w * D[3 * c];
                    v += dmu[m * CP + ch];
                    float* dst = grad + o * C + ch;
                    *dst = accumulate ? *dst + v : v;
                }
            }
        }
    }
}

// Stage 2 for the normals and radii (reading of the paper's training of n and
// eps, Sec. 7 with App. C).  Per leaf, over the nodes u holding it:
//   dL/dn_m   = A_m sum_c mu_m^c sum_u dS_u^c + opened-leaf terms,
//   dL/deps_m = A_m sum_u dE_u / A~_u       + opened-leaf terms,
// since S_u^c = sum A_m mu_m^c n_m and eps~_u = sum A_m eps_m / A~_u.
template <int CP, typename AT>
__global__ void __launch_bounds__(128) k_stage2_geom(
    int64_t nn, const PointRec* __restrict__ pts, const uint32_t* __restrict__ perm,
    const int32_t* __restrict__ first, const int32_t* __restrict__ count,
    const int32_t* __restrict__ is_leaf, const int32_t* __restrict__ parent,
    const double* __restrict__ agg64, const float* __restrict__ dS, const float* __restrict__ dE,
    const AT* __restrict__ mu, const float* __restrict__ dgeo, int accumulate,
    float* __restrict__ grad_n, float* __restrict__ grad_eps) {
    constexpr int SR = srow(CP);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (!is_leaf[t]) continue;
        const int64_t f = first[t], k = count[t];
        if (grad_eps) {
            float E = 0.0f;
            for (int64_t u = t; u >= 0; u = parent[u])
                E = fmaf(dE[u], __frcp_rn((float)agg64[5 * u]), E);
            for (int64_t m = f; m < f + k; ++m) {
                const float v = fmaf(pts[m].w.w, E, dgeo[4 * m + 3]);
                float* dst = grad_eps + perm[m];
                *dst = accumulate ? *dst + v : v;
            }
        }
        if (!grad_n) continue;
#pragma unroll 1
        for (int c0 = 0; c0 < CP; c0 += 4) {
            float D[12];
#pragma unroll
            for (int j = 0; j < 12; ++j) D[j] = 0.0f;
            for (int64_t u = t; u >= 0; u = parent[u]) {
#pragma unroll
                for (int j = 0; j < 12; ++j) {
                    if (3 * c0 + j >= 3 * CP) break;
                    D[j] += dS[u * SR + 3 * c0 + j];
                }
            }
            for (int64_t m = f; m < f + k; ++m) {
                float v[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (c0 + c >= CP) break;
                    const float mc = to_f<AT>(mu[m * CP + c0 + c]);
#pragma unroll
                    for (int j = 0; j < 3; ++j) v[j] = fmaf(mc, D[3 * c + j], v[j]);
                }
                const float A = pts[m].w.w;
                float* dst = grad_n + 3 * (int64_t)perm[m];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float x = A * v[j];
                    if (c0 == 0) {
                        x += dgeo[4 * m + j];
                        dst[j] = accumulate ? dst[j] + x : x;
                    } else {
                        dst[j] += x;
                    }
                }
            }
        }
    }
}

template <int CP, typename AT>
void launch_stage2_geom(const dipole_tree* t, float* grad_n, float* grad_eps, int accumulate,
                        cudaStream_t s) {
    int64_t blocks = (t->nn + 127) / 128;
    int64_t cap = (int64_t)num_sms() * 16;
    note_launch();
    k_stage2_geom<CP, AT><<<(unsigned)(blocks < cap ? blocks : cap), 128, 0, s>>>(
        t->nn, t->pts, t->perm, t->first, t->count, t->is_leaf, t->parent, t->agg64, t->dS, t->dE,
        (const AT*)t->mu, t->dgeo, accumulate, grad_n, grad_eps);
}

template <int CP, typename AT>
void launch_refit(dipole_tree* t, const void* attrs, cudaStream_t s) {
    int64_t blocks = (t->nn + 127) / 128;
    int64_t cap = (int64_t)num_sms() * 16;
    const unsigned grid = (unsigned)(blocks < cap ? blocks : cap);
    const unsigned ntiles = (unsigned)((t->nn + kRefitTile - 1) / kRefitTile);
    const int64_t pblocks = (t->n + kLeafThreads - 1) / kLeafThreads, pcap = (int64_t)num_sms() * 8;
    note_launch();
    k_refit_leaves<CP, AT><<<(unsigned)(pblocks < pcap ? pblocks : pcap), kLeafThreads, 0, s>>>(
        t->n, t->pts, t->perm, t->leaf_of, t->count, (const AT*)attrs, t->C, t->G, (AT*)t->mu,
        t->S, t->fix_cmax);
    note_launch();
    k_refit_tiles<CP><<<ntiles, kRefitThreads, 0, s>>>(t->nn, t->is_leaf, t->S, t->fix_cmax,
                                                       t->fix_kexp, t->fix_tsum, t->fix_done);
    const int64_t ldP = fix_ld(t->nn);
    note_launch();
    k_refit_prefix<CP><<<ntiles, kRefitThreads, 0, s>>>(t->nn, ldP, t->is_leaf, t->S, t->fix_kexp,
                                                        t->fix_tsum, t->fix_P);
    note_launch();
    k_refit_internal<CP><<<grid, 128, 0, s>>>(t->nn, ldP, t->is_leaf, t->skip, t->fix_kexp,
                                              t->fix_P, t->S);
    if (t->S16) {
        const int64_t total = t->nn * (srow16(CP) / 4);
        const int64_t mblocks = (total + 255) / 256, mcap = (int64_t)num_sms() * 8;
        note_launch();
        k_moments_bf16<CP><<<(unsigned)(mblocks < mcap ? mblocks : mcap), 256, 0, s>>>(t->nn, t->S,
                                                                                     t->S16);
    }
}

template <int CP>
void launch_stage2(const dipole_tree* t, const float* dS, const float* dmu, float* grad,
                   int accumulate, cudaStream_t s) {
    int64_t blocks = (t->nn + 127) / 128;
    int64_t cap = (int64_t)num_sms() * 16;
    note_launch(); k_stage2<CP><<<(unsigned)(blocks < cap ? blocks : cap), 128, 0, s>>>(
        t->nn, t->pts, t->perm, t->first, t->count, t->is_leaf, t->parent, dS, dmu, t->C, t->G,
        accumulate, grad);
}

}  // namespace

int padded_channels(int C) {
    if (C <= 1) return 1;
    if (C <= 2) return 2;
    if (C <= 4) return 4;
    if (C <= 8) return 8;
    if (C <= 16) return 16;
    if (C <= 32) return 32;
    if (C <= 36) return 36;  // 32 appearance channels plus geometry, in chunks of 4
    return 64;
}

int refit(dipole_tree* t, const void* attrs, int C, int dtype, int G, cudaStream_t s) {
    const int Cp = padded_channels(C);
    const int SR = srow(Cp);
    const bool m16 = dtype == 2;  // bf16 attributes and a bf16 copy of the moments
    const int adt = m16 ? 1 : dtype;
    if (t->attr_Cp_alloc != Cp || t->attr_dtype_alloc != dtype) {
        // (re)allocate the attribute state in one block; the previous one is freed in stream order
        if (t->attr_block) cudaFreeAsync(t->attr_block, s);
        t->attr_block = nullptr;
        const int64_t NC = 3 * (int64_t)Cp;
        const int64_t ntiles = (t->nn + kRefitTile - 1) / kRefitTile;
        auto take = [&](Carve& c) {
            unsigned char* mu = nullptr;
            c.take(&mu, (adt == 1 ? 2 : 4) * t->n * Cp);
            t->mu = mu;
            c.take(&t->S, t->nn * SR);
            if (m16) c.take(&t->S16, t->nn * srow16(Cp));
            else t->S16 = nullptr;
            c.take(&t->dS, t->nn * SR);
            c.take(&t->dmu, t->n * Cp);
            c.take(&t->fix_P, fix_ld(t->nn) * NC);
            c.take(&t->fix_tsum, ntiles * NC);
            c.take(&t->fix_cmax, NC + 1);  // the column maxima, then the arrival counter
            t->fix_done = t->fix_cmax ? t->fix_cmax + NC : nullptr;
            c.take(&t->fix_kexp, NC);
        };
        Carve c;
        take(c);
        DIP_CUDA_TRY(dev_alloc((void**)&t->attr_block, c.off, s));
        c = Carve{static_cast<char*>(t->attr_block), 0};
        take(c);
        // (the moment rows' padding columns are never read)
        DIP_CUDA_TRY(cudaMemsetAsync(t->fix_cmax, 0, sizeof(unsigned) * (NC + 1), s));
        t->attr_Cp_alloc = Cp;
        t->attr_dtype_alloc = dtype;
    }
    t->C = C;
    t->G = G;
    t->Cp = Cp;
    t->dtype = adt;
#define DIP_REFIT_CASE(K)                                                          \
    case K:                                                                        \
        if (adt == 1) launch_refit<K, __nv_bfloat16>(t, attrs, s);                 \
        else launch_refit<K, float>(t, attrs, s);                                  \
        break;
    switch (Cp) {
        DIP_REFIT_CASE(1)
        DIP_REFIT_CASE(2)
        DIP_REFIT_CASE(4)
        DIP_REFIT_CASE(8)
        DIP_REFIT_CASE(16)
        DIP_REFIT_CASE(32)
        DIP_REFIT_CASE(36)
        DIP_REFIT_CASE(64)
        default:
            return dip_fail(-1, "dipole_refit: unsupported channel count");
    }
#undef DIP_REFIT_CASE
    DIP_CUDA_TRY(cudaGetLastError());
    return 0;
}

int64_t adjoint_acc_floats(const dipole_tree* t) {
    return t->nn * (int64_t)srow(t->Cp) + t->n * (int64_t)t->Cp;
}

int stage2(const dipole_tree* t, const float* dS, const float* dmu, float* grad, int accumulate,
           cudaStream_t s) {
    switch (t->Cp) {
        case 1: launch_stage2<1>(t, dS, dmu, grad, accumulate, s); break;
        case 2: launch_stage2<2>(t, dS, dmu, grad, accumulate, s); break;
        case 4: launch_stage2<4>(t, dS, dmu, grad, accumulate, s); break;
        case 8: launch_stage2<8>(t, dS, dmu, grad, accumulate, s); break;
        case 16: launch_stage2<16>(t, dS, dmu, grad, accumulate, s); break;
        case 32: launch_stage2<32>(t, dS, dmu, grad, accumulate, s); break;
        case 36: launch_stage2<36>(t, dS, dmu, grad, accumulate, s); break;
        case 64: launch_stage2<64>(t, dS, dmu, grad, accumulate, s); break;
        default: return dip_fail(-1, "dipole_adjoint: unsupported channel count");
    }
    DIP_CUDA_TRY(cudaGetLastError());
    return 0;
}

int ensure_geom_scratch(dipole_tree* t, cudaStream_t s) {
    if (!t->dE) DIP_CUDA_TRY(dev_alloc((void**)&t->dE, sizeof(float) * (size_t)t->nn, s));
    if (!t->dgeo) DIP_CUDA_TRY(dev_alloc((void**)&t->dgeo, sizeof(float) * 4 * (size_t)t->n, s));
    return 0;
}

int stage2_geom(const dipole_tree* t, float* grad_n, float* grad_eps, int accumulate,
                cudaStream_t s) {
    if (!grad_n && !grad_eps) return 0;
#define DIP_S2G_CASE(K)                                                                   \
    case K:                                                                               \
        if (t->dtype == 1) launch_stage2_geom<K, __nv_bfloat16>(t, grad_n, grad_eps, accumulate, s); \
        else launch_stage2_geom<K, float>(t, grad_n, grad_eps, accumulate, s);            \
        break;
    switch (t->Cp) {
        DIP_S2G_CASE(1)
        DIP_S2G_CASE(2)
        DIP_S2G_CASE(4)
        DIP_S2G_CASE(8)
        DIP_S2G_CASE(16)
        DIP_S2G_CASE(32)
        DIP_S2G_CASE(36)
        DIP_S2G_CASE(64)
        default:
            return dip_fail(-1, "stage2_geom: unsupported channel count");
    }
#undef DIP_S2G_CASE
    DIP_CUDA_TRY(cudaGetLastError());
    return 0;
}

}  // namespace dip
