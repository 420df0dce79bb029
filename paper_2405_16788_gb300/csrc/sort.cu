// Device-wide primitives: exclusive scan, stable LSD radix sort of (key, value)
// pairs, and Morton codes of query points.  The octree of Sec. 6.1 is built
// over points sorted by 30-bit Morton code (ties kept in input order); the
// queries are sorted the same way so that a warp holds nearby points.
#include "common.cuh"

namespace dip {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan of one tile in place; the tile total goes to totals[blockIdx].
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(uint32_t* data, int64_t n,
                                                            uint32_t* totals) {
    __shared__ uint32_t warp_sums[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)tid * kScanItems;
    uint32_t v[kScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? data[base + k] : 0u;
        sum += v[k];
    }
    uint32_t incl = warp_incl_scan(sum, lane);
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_sums[lane];
        uint32_t wi = warp_incl_scan(w, lane);
        warp_sums[lane] = wi - w;
    }
    __syncthreads();
    uint32_t run = warp_sums[warp] + incl - sum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) data[base + k] = run;
        run += v[k];
    }
    if (tid == kScanThreads - 1 && totals) totals[blockIdx.x] = run;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(uint32_t* data, int64_t n,
                                                           const uint32_t* offsets) {
    const uint32_t add = offsets[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
        int64_t i = base + k;
        if (i < n) data[i] += add;
    }
}

// ------------------------------------------------------------- radix sort
constexpr int kSortThreads = 256;
constexpr int kSortItems = 4;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortWarps = kSortThreads / 32;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* keys, int64_t n,
                                                             int shift, uint32_t mask,
                                                             uint32_t* hist, int nblocks) {
    __shared__ uint32_t cnt[kRadix];
    const int tid = threadIdx.x, lane = tid & 31;
    cnt[tid] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = base + (int64_t)r * kSortThreads + tid;
        uint32_t d = (i < n) ? ((keys[i] >> shift) & mask) : (uint32_t)kRadix;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (d < (uint32_t)kRadix && lane == __ffs(peers) - 1) atomicAdd(&cnt[d], __popc(peers));
    }
    __syncthreads();
    hist[(int64_t)tid * nblocks + blockIdx.x] = cnt[tid];
}

// Stable scatter: keys are ranked round by round (256 consecutive keys per
// round), warp by warp, lane by lane, which is input order.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, int shift, uint32_t mask,
    const uint32_t* __restrict__ offsets, int nblocks) {
    __shared__ uint32_t wcnt[kSortWarps][kRadix];
    __shared__ uint32_t running[kRadix];
    __shared__ uint32_t gbase[kRadix];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    running[tid] = 0;
    gbase[tid] = offsets[(int64_t)tid * nblocks + blockIdx.x];
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        int64_t i = base + (int64_t)r * kSortThreads + tid;
        bool valid = i < n;
        uint32_t key = valid ? kin[i] : 0u;
        uint32_t val = valid ? vin[i] : 0u;
        uint32_t d = valid ? ((key >> shift) & mask) : (uint32_t)kRadix;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt_mask);
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {   // per digit: exclusive prefix over warps, continuing earlier rounds
            uint32_t run = running[tid];
#pragma unroll
            for (int w = 0; w < kSortWarps; ++w) {
                uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = run;
                run += c;
            }
            running[tid] = run;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = gbase[d] + wcnt[warp][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

__global__ void k_query_codes(const float* __restrict__ q, int64_t nq, const float* __restrict__ bbox,
                              int shift, uint32_t* __restrict__ codes, uint32_t* __restrict__ idx,
                              int* status, int hilbert) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float x = q[3 * i], y = q[3 * i + 1], z = q[3 * i + 2];
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) atomicOr(status, kStatusNonFinite);
        uint32_t qx, qy, qz;
        cube_cell(x, y, z, bbox, qx, qy, qz);
        codes[i] = (hilbert ? hilbert30(qx, qy, qz) : morton30(qx, qy, qz)) >> shift;
        idx[i] = (uint32_t)i;
    }
}

// Bandwidth probe: every thread reads its grid-stride share of `buf` `passes`
// times with L2-only loads and writes one value so the loads stay live.
__global__ void k_probe_l2(const float4* __restrict__ buf, int64_t n4, int passes,
                           float* __restrict__ sink) {
    float acc = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int p = 0; p < passes; ++p)
        for (int64_t i = t; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc += (v.x + v.y) + (v.z + v.w);
        }
    sink[t] = acc;
}

}  // namespace

void probe_l2(const void* buf, int64_t bytes, int passes, float* sink, cudaStream_t s) {
    note_launch();
    k_probe_l2<<<4 * num_sms(), 256, 0, s>>>(static_cast<const float4*>(buf), bytes / 16, passes,
                                             sink);
}

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

int64_t scan_tmp_entries(int64_t n) {
    int64_t total = 0;
    int64_t m = n;
    while (m > kScanTile) {
        m = (m + kScanTile - 1) / kScanTile;
        total += m + 32;
    }
    return total + 32;
}

void exclusive_scan_u32(uint32_t* data, int64_t n, uint32_t* tmp, cudaStream_t s) {
    if (n <= 0) return;
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        note_launch(); k_scan_tile<<<1, kScanThreads, 0, s>>>(data, n, nullptr);
        return;
    }
    uint32_t* totals = tmp;
    note_launch(); k_scan_tile<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, totals);
    exclusive_scan_u32(totals, nb, tmp + nb + 32, s);
    note_launch(); k_scan_add<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, totals);
}

int64_t radix_hist_entries(int64_t n) {
    int64_t nb = (n + kSortTile - 1) / kSortTile;
    if (nb < 1) nb = 1;
    int64_t h = nb * kRadix;
    return h + scan_tmp_entries(h);
}

void radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                      uint32_t* hist, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1) return;
    int nb = (int)((n + kSortTile - 1) / kSortTile);
    int64_t h = (int64_t)nb * kRadix;
    uint32_t* scan_tmp = hist + h;
    uint32_t *ki = keys, *vi = vals, *ko = keys_tmp, *vo = vals_tmp;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += kRadixBits) {
        int w = bits - shift < kRadixBits ? bits - shift : kRadixBits;
        uint32_t mask = (1u << w) - 1u;
        note_launch(); k_radix_hist<<<nb, kSortThreads, 0, s>>>(ki, n, shift, mask, hist, nb);
        exclusive_scan_u32(hist, h, scan_tmp, s);
        note_launch(); k_radix_scatter<<<nb, kSortThreads, 0, s>>>(ki, vi, ko, vo, n, shift, mask, hist, nb);
        uint32_t* t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
        ++passes;
    }
    if (passes & 1) {
        cudaMemcpyAsync(keys, ki, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, vi, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
    }
}

void query_codes(const float* queries, int64_t q, const float* bbox, int shift, uint32_t* codes,
                 uint32_t* idx, int* status, cudaStream_t s, bool hilbert) {
    if (q <= 0) return;
    int64_t blocks = (q + 255) / 256;
    int64_t cap = (int64_t)num_sms() * 8;
    note_launch(); k_query_codes<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(
        queries, q, bbox, shift, codes, idx, status, hilbert ? 1 : 0);
}

}  // namespace dip
