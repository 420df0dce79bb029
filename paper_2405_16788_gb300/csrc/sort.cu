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
static_assert(kScanTile == kScanTileSize, "the tile-local scan's tile");

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan in one launch, for consumers that add the tile offsets
// themselves: the tiles write their local exclusive scans and totals, and the
// last tile to finish (an arrival counter; no block waits for another) turns
// the totals into exclusive tile offsets in place, 4,096 at a time, writes the
// sum of all values to *grand (if given) and clears the counter.  The scan's
// value at i is then data[i] + totals[i / kScanTile].
__global__ void __launch_bounds__(kScanThreads) k_scan_tile_last(uint32_t* data, int64_t n,
                                                                 uint32_t* totals, unsigned* done,
                                                                 uint32_t* grand) {
    __shared__ uint32_t warp_sums[32];
    __shared__ bool last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto block_exclusive = [&](uint32_t* a, int64_t m, int64_t base0, uint32_t carry) {
        // exclusive scan of a[base0 .. base0 + kScanTile) (bounded by m) plus carry;
        // returns the chunk's total through warp_sums[31] + last partial
        const int64_t base = base0 + (int64_t)tid * kScanItems;
        uint32_t v[kScanItems];
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            v[k] = (base + k < m) ? __ldcg(a + base + k) : 0u;
            sum += v[k];
        }
        const uint32_t incl = warp_incl_scan(sum, lane);
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = warp_sums[lane];
            const uint32_t wi = warp_incl_scan(w, lane);
            warp_sums[lane] = wi - w;
        }
        __syncthreads();
        uint32_t run = carry + warp_sums[warp] + incl - sum;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (base + k < m) a[base + k] = run;
            run += v[k];
        }
        __syncthreads();  // warp_sums is reused
        return run;       // the running total after this thread's items
    };
    const uint32_t tot = block_exclusive(data, n, (int64_t)blockIdx.x * kScanTile, 0u);
    if (tid == kScanThreads - 1) {
        totals[blockIdx.x] = tot;
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ uint32_t carry_s;
    uint32_t carry = 0;
    for (int64_t c0 = 0; c0 < gridDim.x; c0 += kScanTile) {
        const uint32_t r = block_exclusive(totals, gridDim.x, c0, carry);
        if (tid == kScanThreads - 1) carry_s = r;
        __syncthreads();
        carry = carry_s;
        __syncthreads();
    }
    if (tid == 0) {
        *done = 0u;
        if (grand) *grand = carry;  // the sum of all n values
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
    const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ tile_off, int nblocks) {
    __shared__ uint32_t wcnt[kSortWarps][kRadix];
    __shared__ uint32_t running[kRadix];
    __shared__ uint32_t gbase[kRadix];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    running[tid] = 0;
    {   // offsets: tile-local exclusive scan plus the tile's offset (k_scan_tile_last)
        const int64_t i = (int64_t)tid * nblocks + blockIdx.x;
        gbase[tid] = offsets[i] + tile_off[i / kScanTile];
    }
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

int64_t scan_local_entries(int64_t n) { return (n + kScanTile - 1) / kScanTile + 4; }

void exclusive_scan_local(uint32_t* data, int64_t n, uint32_t* ws, uint32_t* grand,
                          cudaStream_t s, unsigned* done_zero) {
    if (n <= 0) return;
    const unsigned st = (unsigned)((n + kScanTile - 1) / kScanTile);
    unsigned* done = done_zero;
    if (!done) {
        done = reinterpret_cast<unsigned*>(ws + st);
        cudaMemsetAsync(done, 0, sizeof(unsigned), s);
    }
    note_launch(); k_scan_tile_last<<<st, kScanThreads, 0, s>>>(data, n, ws, done, grand);
}

int64_t radix_hist_entries(int64_t n) {
    int64_t nb = (n + kSortTile - 1) / kSortTile;
    if (nb < 1) nb = 1;
    const int64_t h = nb * kRadix;
    return h + (h + kScanTile - 1) / kScanTile + 4;  // counts, tile totals, arrival counter
}

// Three launches per 8-bit pass: digit counts per tile of keys, their scan
// (tile-local, the last tile scanning the tile totals), the stable scatter.
void radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                      uint32_t* hist, int64_t n, int bits, cudaStream_t s, unsigned* done_zero) {
    if (n <= 1) return;
    int nb = (int)((n + kSortTile - 1) / kSortTile);
    int64_t h = (int64_t)nb * kRadix;
    const unsigned st = (unsigned)((h + kScanTile - 1) / kScanTile);
    uint32_t* totals = hist + h;  // st entries
    unsigned* done = done_zero;   // arrival counter of the scans, zero between passes
    if (!done) {
        done = reinterpret_cast<unsigned*>(totals + st);
        cudaMemsetAsync(done, 0, sizeof(unsigned), s);
    }
    uint32_t *ki = keys, *vi = vals, *ko = keys_tmp, *vo = vals_tmp;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += kRadixBits) {
        int w = bits - shift < kRadixBits ? bits - shift : kRadixBits;
        uint32_t mask = (1u << w) - 1u;
        note_launch(); k_radix_hist<<<nb, kSortThreads, 0, s>>>(ki, n, shift, mask, hist, nb);
        note_launch(); k_scan_tile_last<<<st, kScanThreads, 0, s>>>(hist, h, totals, done, nullptr);
        note_launch(); k_radix_scatter<<<nb, kSortThreads, 0, s>>>(ki, vi, ko, vo, n, shift, mask, hist,
                                                                  totals, nb);
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
