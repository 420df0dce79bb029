// Octree construction and node geometry (Sec. 6.1, eq. farfield_dipole;
// Sec. 6.3: the tree is built once because positions are not optimized).
//
// Tree definition (the paper says only "octree"): 30-bit Morton codes over
// the bounding cube, points sorted stably by code; a node at level l is a
// maximal run of sorted codes sharing their top 3l bits; a run of at most
// leaf_size points, or at level max_depth, is a leaf; a run whose points all
// share the next digit is the same node as its only child.  Nodes are stored
// in depth-first preorder with skip[t] = the index just past t's subtree.
//
// GPU construction: preorder is the order of (first point, level), so every
// sorted point i enumerates the runs that start at i level by level (their
// ends found by galloping search over the sorted codes), keeps the ones the
// definition keeps, and an exclusive scan of the per-point node counts gives
// every node its preorder index.  No recursion, no per-level launches.
#include "tree.cuh"

#include <float.h>

#include <algorithm>
#include <cstring>

namespace dip {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Bounding cube from the per-block boxes: lo = per-axis minimum; ext = largest
// per-axis extent (float subtraction), 1 if 0; scale = 1024 / ext (correctly
// rounded division).  One warp reduces the partials.
__device__ void bbox_final(const float* partial, int nb, float* bbox) {
    const int lane = threadIdx.x & 31;
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int b = lane; b < nb; b += 32)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], __ldcg(partial + b * 6 + a));
            hi[a] = fmaxf(hi[a], __ldcg(partial + b * 6 + 3 + a));
        }
    for (int a = 0; a < 3; ++a) { lo[a] = warp_min(lo[a]); hi[a] = warp_max(hi[a]); }
    if (lane != 0) return;
    float ext = 0.0f;
    for (int a = 0; a < 3; ++a) {
        float e = __fsub_rn(hi[a], lo[a]);
        if (e > ext) ext = e;
    }
    if (!(ext > 0.0f)) ext = 1.0f;
    bbox[0] = lo[0]; bbox[1] = lo[1]; bbox[2] = lo[2];
    bbox[3] = ext;
    bbox[4] = __fdiv_rn(1024.0f, ext);
}

// Input validation and per-block bounding boxes; the last block to finish
// (an arrival counter, zero on entry; no block waits for another) reduces them
// into the bounding cube.
__global__ void __launch_bounds__(kThreads) k_bbox(const float* __restrict__ p,
                                                   const float* __restrict__ nrm,
                                                   const float* __restrict__ A,
                                                   const float* __restrict__ eps, int64_t n,
                                                   float* partial, int* status, unsigned* done,
                                                   float* bbox) {
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float x = p[3 * i], y = p[3 * i + 1], z = p[3 * i + 2];
        float a = A[i];
        float e = eps ? eps[i] : 0.0f;
        bool fin = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(nrm[3 * i]) &&
                   isfinite(nrm[3 * i + 1]) && isfinite(nrm[3 * i + 2]) && isfinite(a) &&
                   isfinite(e);
        if (!fin) bad |= kStatusNonFinite;
        if (!(a > 0.0f)) bad |= kStatusBadArea;
        if (e < 0.0f) bad |= kStatusBadRadius;
        lo[0] = fminf(lo[0], x); hi[0] = fmaxf(hi[0], x);
        lo[1] = fminf(lo[1], y); hi[1] = fmaxf(hi[1], y);
        lo[2] = fminf(lo[2], z); hi[2] = fmaxf(hi[2], z);
    }
    if (bad) atomicOr(status, bad);
    __shared__ float sh[6][kThreads / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float l = warp_min(lo[a]), h = warp_max(hi[a]);
        if (lane == 0) { sh[a][warp] = l; sh[3 + a][warp] = h; }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        float v = sh[threadIdx.x][0];
        for (int w = 1; w < kThreads / 32; ++w)
            v = threadIdx.x < 3 ? fminf(v, sh[threadIdx.x][w]) : fmaxf(v, sh[threadIdx.x][w]);
        partial[blockIdx.x * 6 + threadIdx.x] = v;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1u;
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    bbox_final(partial, (int)gridDim.x, bbox);
}

// Point record of sorted point i (input point perm[i]).
__device__ __forceinline__ void pack_point(int64_t i, const uint32_t* __restrict__ perm,
                                           const float* __restrict__ p,
                                           const float* __restrict__ nrm,
                                           const float* __restrict__ A,
                                           const float* __restrict__ eps,
                                           PointRec* __restrict__ pts, float* __restrict__ eps_sorted) {
    int64_t m = perm[i];
    float a = A[m];
    float e = eps ? eps[m] : 0.0f;
    PointRec r;
    r.geo = make_float4(p[3 * m], p[3 * m + 1], p[3 * m + 2], __frcp_rn(e));
    r.w = make_float4(__fmul_rn(a, nrm[3 * m]), __fmul_rn(a, nrm[3 * m + 1]),
                      __fmul_rn(a, nrm[3 * m + 2]), a);
    pts[i] = r;
    eps_sorted[i] = e;
}

__global__ void k_pack(const uint32_t* __restrict__ perm, const float* __restrict__ p,
                       const float* __restrict__ nrm, const float* __restrict__ A,
                       const float* __restrict__ eps, int64_t n, PointRec* __restrict__ pts,
                       float* __restrict__ eps_sorted) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        pack_point(i, perm, p, nrm, A, eps, pts, eps_sorted);
}

// ------------------------------------------------------------- topology
__device__ __forceinline__ int lcp_digits(uint32_t a, uint32_t b) {
    uint32_t x = a ^ b;
    return x ? (__clz(x) - 2) / 3 : kMaxLevel;
}

__device__ __forceinline__ bool same_run(uint32_t a, uint32_t b, int l) {
    return l == 0 || ((a ^ b) >> (30 - 3 * l)) == 0u;
}

// First index >= lb whose code leaves the level-l run of code ci (every index
// in (i, lb) is known to be inside it).  Galloping, then bisection.
__device__ int64_t run_end(const uint32_t* __restrict__ c, int64_t n, uint32_t ci, int l,
                           int64_t lb) {
    if (lb >= n || !same_run(ci, c[lb], l)) return lb;
    int64_t lo = lb, hi, step = 1;
    for (;;) {
        hi = lo + step;
        if (hi >= n) { hi = n; break; }
        if (!same_run(ci, c[hi], l)) break;
        lo = hi;
        step <<= 1;
    }
    while (hi - lo > 1) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (same_run(ci, c[mid], l)) lo = mid; else hi = mid;
    }
    return hi;
}

// Runs starting at sorted point i that are nodes.  Bit l of the returned mask:
// the level-l run starting at i is a node; bit l of *imask: it is internal.
// e[l] receives the end of the level-l run holding i, for the levels visited.
// The loops run over all kMaxLevel + 1 levels with the bounds as guards, so
// that they unroll and e stays in registers.
__device__ __forceinline__ uint32_t analyze_point(const uint32_t* __restrict__ c, int64_t n,
                                                  int64_t i, int leaf_size, int max_depth,
                                                  int64_t (&e)[kMaxLevel + 2], uint32_t* imask) {
    const uint32_t ci = c[i];
    const int s = (i == 0) ? 0 : lcp_digits(c[i - 1], ci) + 1;
    *imask = 0;
    if (s > max_depth) return 0;
    const int lmin = s > 0 ? s - 1 : 0;
    int64_t lb = i + 1;
#pragma unroll
    for (int l = kMaxLevel; l >= 0; --l) {
        if (l > max_depth || l < lmin) continue;
        lb = run_end(c, n, ci, l, lb);
        e[l] = lb;
    }
    uint32_t mask = 0;
#pragma unroll
    for (int l = 0; l <= kMaxLevel; ++l) {
        if (l < s || l > max_depth) continue;
        const int64_t cnt = e[l] - i;
        if (l < max_depth && cnt > leaf_size && e[l + 1] < e[l]) {  // branches at digit l
            mask |= 1u << l;
            *imask |= 1u << l;
            continue;
        }
        if (!(cnt <= leaf_size || l == max_depth)) continue;  // single child: collapsed
        bool parent_open = true;                               // root
        if (l > 0) {
            // the level-(l-1) run holding i has more than leaf_size points?
            const int64_t pe = e[l - 1];
            if (pe - i <= leaf_size) {
                const int64_t k = pe - leaf_size - 1;
                parent_open = (k >= 0) && same_run(c[k], ci, l - 1);
            }
        }
        if (parent_open) mask |= 1u << l;
    }
    return mask;
}

// Per sorted point: the number of nodes whose runs start there (into cnt), the
// node/internal masks (mask | imask << 16) and, for every level with a node,
// the end of its run (estage[11 i + l]), so that the emit pass need not search
// again.
// Also packs the point records (one launch for two per-point passes) and
// sets the count after the last point, cnt[n], to 0.
__global__ void k_topo_count(const uint32_t* __restrict__ c, int64_t n, int leaf_size,
                             int max_depth, uint32_t* __restrict__ cnt, uint32_t* __restrict__ tmask,
                             int32_t* __restrict__ estage, const uint32_t* __restrict__ perm,
                             const float* __restrict__ p, const float* __restrict__ nrm,
                             const float* __restrict__ A, const float* __restrict__ eps,
                             PointRec* __restrict__ pts, float* __restrict__ eps_sorted) {
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt[n] = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        pack_point(i, perm, p, nrm, A, eps, pts, eps_sorted);
        int64_t e[kMaxLevel + 2];
        uint32_t im;
        const uint32_t mask = analyze_point(c, n, i, leaf_size, max_depth, e, &im);
        cnt[i] = __popc(mask);
        tmask[i] = mask | (im << 16);
#pragma unroll
        for (int l = 0; l <= kMaxLevel; ++l)  // no bit above max_depth is set
            if (mask & (1u << l)) estage[i * (kMaxLevel + 1) + l] = (int32_t)e[l];
    }
}

// off: the tile-local exclusive scan of the per-point node counts, completed
// by tile_off (exclusive_scan_local).
// It also sets what the node pass expects cleared: parent[t] = -1 and
// rbits[t] = 0 for the nn nodes, and the level counters.
__global__ void k_topo_emit(int64_t n, int64_t nn, int max_depth, const uint32_t* __restrict__ off,
                            const uint32_t* __restrict__ tile_off, int32_t* __restrict__ parent,
                            unsigned int* __restrict__ rbits, unsigned int* __restrict__ lvl_cnt,
                            const uint32_t* __restrict__ tmask, const int32_t* __restrict__ estage,
                            int32_t* __restrict__ first, int32_t* __restrict__ count,
                            int32_t* __restrict__ level, int32_t* __restrict__ skip,
                            int32_t* __restrict__ is_leaf, int32_t* __restrict__ leaf_of) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t t = g; t < nn; t += stride) {
        parent[t] = -1;
        rbits[t] = 0u;
    }
    if (g < 2 * (kMaxLevel + 1)) lvl_cnt[g] = 0u;
    for (int64_t i = g; i < n; i += stride) {
        const uint32_t mk = tmask[i];
        const uint32_t mask = mk & 0xffffu, im = mk >> 16;
        if (!mask) continue;
        uint32_t t = off[i] + tile_off[i / kScanTileSize];
        for (int l = 0; l <= max_depth; ++l) {
            if (!(mask & (1u << l))) continue;
            const int64_t e = estage[i * (kMaxLevel + 1) + l];
            first[t] = (int32_t)i;
            count[t] = (int32_t)(e - i);
            level[t] = l;
            skip[t] = (int32_t)(off[e] + tile_off[e / kScanTileSize]);
            const bool leaf = !(im & (1u << l));
            is_leaf[t] = leaf ? 1 : 0;
            if (leaf)
                for (int64_t m = i; m < e; ++m) leaf_of[m] = (int32_t)t;
            ++t;
        }
    }
}

// Children of internal node t: t+1, skip[t+1], ... below skip[t].
__global__ void k_children(int64_t nn, const int32_t* __restrict__ skip,
                           const int32_t* __restrict__ is_leaf, int32_t* __restrict__ parent,
                           int32_t* __restrict__ nchild, int* status) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (is_leaf[t]) { nchild[t] = 0; continue; }
        int k = 0;
        int32_t end = skip[t];
        for (int32_t ch = (int32_t)t + 1; ch < end;) {
            parent[ch] = (int32_t)t;
            ++k;
            int32_t nx = skip[ch];
            if (nx <= ch || k > 8) { atomicOr(status, kStatusTraversal); break; }
            ch = nx;
        }
        nchild[t] = k;
    }
}

// Internal nodes grouped by level (the order inside a level is arbitrary):
// count, offsets, then one slot per node.  Bottom-up passes process the leaves
// first, then the internal levels from the deepest to the root, one launch per
// level, so a node's children are always complete before it is summed.
__global__ void k_level_count(int64_t nn, const int32_t* __restrict__ level,
                              const int32_t* __restrict__ is_leaf, unsigned int* lvl_cnt) {
    __shared__ unsigned int sc[kMaxLevel + 1];
    if (threadIdx.x <= kMaxLevel) sc[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn;
         t += (int64_t)gridDim.x * blockDim.x)
        if (!is_leaf[t]) atomicAdd(&sc[level[t]], 1u);
    __syncthreads();
    if (threadIdx.x <= kMaxLevel && sc[threadIdx.x]) atomicAdd(&lvl_cnt[threadIdx.x], sc[threadIdx.x]);
}

__global__ void k_level_offsets(const unsigned int* lvl_cnt, int32_t* lvl_off, unsigned int* lvl_fill) {
    if (threadIdx.x != 0) return;
    int32_t run = 0;
    for (int l = 0; l <= kMaxLevel; ++l) {
        lvl_off[l] = run;
        lvl_fill[l] = 0;
        run += (int32_t)lvl_cnt[l];
    }
    lvl_off[kMaxLevel + 1] = run;
}

// Each block reserves one range per level, then hands out slots inside it.
// The grid-stride loop runs the same number of rounds in every thread of a
// block so that the barriers are uniform.
__global__ void k_level_fill(int64_t nn, const int32_t* __restrict__ level,
                             const int32_t* __restrict__ is_leaf, const int32_t* __restrict__ lvl_off,
                             unsigned int* lvl_fill, int32_t* __restrict__ lvl_list) {
    __shared__ unsigned int sc[kMaxLevel + 1];
    __shared__ unsigned int sb[kMaxLevel + 1];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nn; base += stride) {
        if (threadIdx.x <= kMaxLevel) sc[threadIdx.x] = 0;
        __syncthreads();
        const int64_t t = base + threadIdx.x;
        int l = -1;
        unsigned int r = 0;
        if (t < nn && !is_leaf[t]) {
            l = level[t];
            r = atomicAdd(&sc[l], 1u);
        }
        __syncthreads();
        if (threadIdx.x <= kMaxLevel && sc[threadIdx.x])
            sb[threadIdx.x] = atomicAdd(&lvl_fill[threadIdx.x], sc[threadIdx.x]);
        __syncthreads();
        if (l >= 0) lvl_list[lvl_off[l] + (int32_t)(sb[l] + r)] = (int32_t)t;
        __syncthreads();
    }
}

// Node sums: in float point by point inside a leaf, in double child by child
// inside an internal node, both in Morton order, so that the float centroid is
// the same on any machine and double precision serves only the upper levels.  The ratios use one correctly rounded reciprocal of
// the area: p~ = (sum A p) * (1 / sum A), eps~ = (sum A eps) * (1 / sum A).
__device__ __forceinline__ void finalize_geom(int64_t t, const double* s, float4* cen4,
                                              float* eps_node) {
    const double r = __drcp_rn(s[0]);
    const double cx = __dmul_rn(s[1], r), cy = __dmul_rn(s[2], r), cz = __dmul_rn(s[3], r);
    cen4[t] = make_float4(__double2float_rn(cx), __double2float_rn(cy), __double2float_rn(cz),
                          0.0f);
    eps_node[t] = __double2float_rn(__dmul_rn(s[4], r));
}

__global__ void k_geom_leaves(int64_t nn, const PointRec* __restrict__ pts,
                              const float* __restrict__ eps_sorted,
                              const int32_t* __restrict__ first, const int32_t* __restrict__ count,
                              const int32_t* __restrict__ is_leaf, double* __restrict__ agg,
                              float4* __restrict__ cen4, float* __restrict__ eps_node) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (!is_leaf[t]) continue;
        // float inside a leaf, one rounding per product and per sum (no fused
        // multiply-add), point by point in Morton order
        float fs[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        const int64_t f = first[t], k = count[t];
        for (int64_t m = f; m < f + k; ++m) {
            const float4 g = pts[m].geo;
            const float a = pts[m].w.w;
            fs[0] = __fadd_rn(fs[0], a);
            fs[1] = __fadd_rn(fs[1], __fmul_rn(a, g.x));
            fs[2] = __fadd_rn(fs[2], __fmul_rn(a, g.y));
            fs[3] = __fadd_rn(fs[3], __fmul_rn(a, g.z));
            fs[4] = __fadd_rn(fs[4], __fmul_rn(a, eps_sorted[m]));
        }
        double s[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) s[j] = (double)fs[j];
#pragma unroll
        for (int j = 0; j < 5; ++j) agg[t * 5 + j] = s[j];
        finalize_geom(t, s, cen4, eps_node);
    }
}

// Levels l_hi down to l_lo; a launch over several levels must be one block
// (its threads order the levels with __syncthreads).
__global__ void __launch_bounds__(kTopThreads) k_geom_level(int l_hi, int l_lo,
                             const int32_t* __restrict__ lvl_off,
                             const int32_t* __restrict__ lvl_list, const int32_t* __restrict__ skip,
                             double* __restrict__ agg, float4* __restrict__ cen4,
                             float* __restrict__ eps_node) {
    for (int l = l_hi; l >= l_lo; --l) {
        const int32_t b = lvl_off[l], e = lvl_off[l + 1];
        for (int64_t i = b + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < e;
             i += (int64_t)gridDim.x * blockDim.x) {
            const int32_t p = lvl_list[i];
            double q[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
            int k = 0;
            for (int32_t ch = p + 1; ch < skip[p] && k < 8; ++k) {
#pragma unroll
                for (int j = 0; j < 5; ++j) q[j] = __dadd_rn(q[j], agg[(int64_t)ch * 5 + j]);
                const int32_t nx = skip[ch];
                if (nx <= ch) break;  // only an imported, corrupt tree gets here
                ch = nx;
            }
#pragma unroll
            for (int j = 0; j < 5; ++j) agg[(int64_t)p * 5 + j] = q[j];
            finalize_geom(p, q, cen4, eps_node);
        }
        if (l > l_lo) __syncthreads();
    }
}

// r~_t = max over the node's points of the float distance to the float
// centroid (fixed operation order).  One thread per point walks its ancestors;
// lanes at the same node combine with a warp max before one atomicMax, which is
// skipped when the node already holds as much: the values only grow, so a
// stale read can only cost an atomic, and the upper nodes (the root takes one
// candidate per warp of the whole cloud) stop serialising on one address.
__global__ void k_radius(int64_t n, const PointRec* __restrict__ pts,
                         const int32_t* __restrict__ leaf_of, const int32_t* __restrict__ parent,
                         const float4* __restrict__ cen4, unsigned int* __restrict__ rbits) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < n;
        int32_t t = valid ? leaf_of[i] : -1;
        float px = 0.f, py = 0.f, pz = 0.f;
        if (valid) { const float4 g = pts[i].geo; px = g.x; py = g.y; pz = g.z; }
        while (__any_sync(0xffffffffu, t >= 0)) {
            unsigned int bits = 0u;
            if (t >= 0) {
                const float4 c = cen4[t];
                const float ex = __fsub_rn(px, c.x), ey = __fsub_rn(py, c.y), ez = __fsub_rn(pz, c.z);
                const float d2 = __fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex)));
                bits = __float_as_uint(__fsqrt_rn(d2));
            }
            const unsigned int peers = __match_any_sync(0xffffffffu, (unsigned int)t);
            const unsigned int m = __reduce_max_sync(peers, bits);
            if (t >= 0 && lane == __ffs(peers) - 1 && m > rbits[t]) atomicMax(&rbits[t], m);
            if (t >= 0) t = parent[t];
        }
    }
}

__global__ void k_finalize_nodes(int64_t nn, const float4* __restrict__ cen4,
                                 const unsigned int* __restrict__ rbits,
                                 const int32_t* __restrict__ skip, const int32_t* __restrict__ first,
                                 const int32_t* __restrict__ count,
                                 const int32_t* __restrict__ is_leaf,
                                 const float* __restrict__ eps_node, NodeRec* __restrict__ nodes) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn;
         t += (int64_t)gridDim.x * blockDim.x) {
        const float4 c = cen4[t];
        NodeRec r;
        r.geo = make_float4(c.x, c.y, c.z, __uint_as_float(rbits[t]));
        r.meta = make_int4(skip[t], first[t], is_leaf[t] ? count[t] : 0,
                           __float_as_int(__frcp_rn(eps_node[t])));
        nodes[t] = r;
    }
}

__global__ void k_leaf_of(int64_t nn, const int32_t* __restrict__ first,
                          const int32_t* __restrict__ count, const int32_t* __restrict__ is_leaf,
                          int32_t* __restrict__ leaf_of) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (!is_leaf[t]) continue;
        for (int64_t m = first[t]; m < (int64_t)first[t] + count[t]; ++m) leaf_of[m] = (int32_t)t;
    }
}

unsigned grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}


// Point arrays, status word and bounding box of a new tree (one block).
int alloc_point_state(dipole_tree* t, cudaStream_t s) {
    const int64_t n = t->n;
    auto take = [&](Carve& c) {
        c.take(&t->pts, n);
        c.take(&t->code, n);
        c.take(&t->perm, n);
        c.take(&t->leaf_of, n);
        // small[0..5) bbox, [8] status word, [9] the build's node count, [10..13)
        // arrival counters of the build's one-launch reductions; [8..16) zeroed at
        // once, [0..10) read back at once
        float* small = nullptr;
        c.take(&small, 16);
        t->bbox = small;
        t->status = reinterpret_cast<int*>(small + 8);
    };
    Carve c;
    take(c);
    DIP_CUDA_TRY(dev_alloc((void**)&t->point_block, c.off, s));
    c = Carve{static_cast<char*>(t->point_block), 0};
    take(c);
    DIP_CUDA_TRY(cudaMemsetAsync(t->bbox + 8, 0, 8 * sizeof(float), s));
    return 0;
}

// The small area's arrival counters (zero from alloc_point_state).
unsigned* build_counter(dipole_tree* t, int k) { return reinterpret_cast<unsigned*>(t->bbox + 10 + k); }

// The node ranges, levels, skip indices and leaf flags (one block).
int alloc_topology(dipole_tree* t, int64_t nn, cudaStream_t s) {
    auto take = [&](Carve& c) {
        c.take(&t->first, nn);
        c.take(&t->count, nn);
        c.take(&t->level, nn);
        c.take(&t->skip, nn);
        c.take(&t->is_leaf, nn);
    };
    Carve c;
    take(c);
    DIP_CUDA_TRY(dev_alloc((void**)&t->topo_block, c.off, s));
    c = Carve{static_cast<char*>(t->topo_block), 0};
    take(c);
    return 0;
}

int status_error(int status_host, const char* who) {
    if (status_host & kStatusNonFinite)
        return dip_fail(-4, std::string(who) + ": non-finite point, normal, area or radius");
    if (status_host & kStatusBadArea)
        return dip_fail(-1, std::string(who) + ": every area weight must be > 0");
    if (status_host & kStatusBadRadius) return dip_fail(-1, std::string(who) + ": radii must be >= 0");
    return 0;
}

// Everything that follows from the node ranges (first, count, level, skip,
// is_leaf, already on the device) and leaf_of: parents, level lists, node
// geometry (eq. farfield_dipole), radius, node records.
// The node arrays (one block) and the node pass's scratch (another).
struct NodeScratch {
    float4* cen4 = nullptr;
    unsigned int* rbits = nullptr;
    unsigned int* lvl_cnt = nullptr;  // [kMaxLevel + 1] counts, [kMaxLevel + 1] fill cursors
    void* tmp = nullptr;
};

int alloc_nodes(dipole_tree* t, NodeScratch& ns, cudaStream_t s) {
    const int64_t nn = t->nn;
    auto take = [&](Carve& c) {
        c.take(&t->nodes, nn);
        c.take(&t->parent, nn);
        c.take(&t->nchild, nn);
        c.take(&t->agg64, nn * 5);
        c.take(&t->eps_node, nn);
        c.take(&t->lvl_list, nn);
        c.take(&t->lvl_off, kMaxLevel + 2);
    };
    auto take_tmp = [&](Carve& c) {
        c.take(&ns.cen4, nn);
        c.take(&ns.rbits, nn);
        c.take(&ns.lvl_cnt, 2 * (kMaxLevel + 1));
    };
    Carve c, ct;
    take(c);
    take_tmp(ct);
    DIP_CUDA_TRY(dev_alloc((void**)&t->node_block, c.off, s));
    DIP_CUDA_TRY(dev_alloc((void**)&ns.tmp, ct.off, s));
    c = Carve{static_cast<char*>(t->node_block), 0};
    ct = Carve{static_cast<char*>(ns.tmp), 0};
    take(c);
    take_tmp(ct);
    return 0;
}

// inited: parent (-1), rbits and lvl_cnt (0) were set by the topology pass.
int derive_nodes(dipole_tree* t, const float* eps_sorted, NodeScratch& ns, bool inited,
                 cudaStream_t s) {
    const int64_t n = t->n, nn = t->nn;
    float4* cen4 = ns.cen4;
    unsigned int *rbits = ns.rbits, *lvl_cnt = ns.lvl_cnt;
    void* tmp = ns.tmp;
    if (!inited) {
        DIP_CUDA_TRY(cudaMemsetAsync(t->parent, 0xff, sizeof(int32_t) * nn, s));
        DIP_CUDA_TRY(cudaMemsetAsync(lvl_cnt, 0, sizeof(unsigned int) * 2 * (kMaxLevel + 1), s));
        DIP_CUDA_TRY(cudaMemsetAsync(rbits, 0, sizeof(unsigned int) * nn, s));
    }
    note_launch(); k_children<<<grid_for(nn, kThreads), kThreads, 0, s>>>(nn, t->skip, t->is_leaf, t->parent,
                                                           t->nchild, t->status);
    note_launch(); k_level_count<<<grid_for(nn, kThreads), kThreads, 0, s>>>(nn, t->level, t->is_leaf,
                                                                            lvl_cnt);
    note_launch(); k_level_offsets<<<1, 32, 0, s>>>(lvl_cnt, t->lvl_off, lvl_cnt + kMaxLevel + 1);
    note_launch(); k_level_fill<<<grid_for(nn, kThreads), kThreads, 0, s>>>(
        nn, t->level, t->is_leaf, t->lvl_off, lvl_cnt + kMaxLevel + 1, t->lvl_list);
    note_launch(); k_geom_leaves<<<grid_for(nn, kThreads), kThreads, 0, s>>>(
        nn, t->pts, eps_sorted, t->first, t->count, t->is_leaf, t->agg64, cen4, t->eps_node);
    for (int l = t->max_depth - 1; l > kTopLevel; --l) {
        note_launch();
        k_geom_level<<<2u * (unsigned)num_sms(), kThreads, 0, s>>>(l, l, t->lvl_off, t->lvl_list,
                                                                 t->skip, t->agg64, cen4, t->eps_node);
    }
    note_launch();
    k_geom_level<<<1, kTopThreads, 0, s>>>(min(kTopLevel, t->max_depth - 1), 0, t->lvl_off,
                                          t->lvl_list, t->skip, t->agg64, cen4, t->eps_node);
    note_launch(); k_radius<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, t->pts, t->leaf_of, t->parent, cen4,
                                                        rbits);
    note_launch(); k_finalize_nodes<<<grid_for(nn, kThreads), kThreads, 0, s>>>(nn, cen4, rbits, t->skip,
                                                                 t->first, t->count, t->is_leaf,
                                                                 t->eps_node, t->nodes);
    cudaFreeAsync(tmp, s);
    DIP_CUDA_TRY(cudaGetLastError());
    return 0;
}

}  // namespace

int build_tree(dipole_tree* t, const float* points, const float* normals, const float* areas,
               const float* radii, cudaStream_t s) {
    const int64_t n = t->n;
    int rc = alloc_point_state(t, s);
    if (rc) return rc;

    // temporaries
    uint32_t *ktmp = nullptr, *vtmp = nullptr, *hist = nullptr, *off = nullptr, *scan_ws = nullptr;
    float* partial = nullptr;
    const unsigned nbb = grid_for(n, kThreads) < 2u * (unsigned)num_sms() ? grid_for(n, kThreads)
                                                                          : 2u * (unsigned)num_sms();
    float* eps_sorted = nullptr;
    uint32_t* tmask = nullptr;
    int32_t* estage = nullptr;
    auto take_tmp = [&](Carve& c) {
        c.take(&ktmp, n);
        c.take(&vtmp, n);
        c.take(&hist, radix_hist_entries(n));
        c.take(&off, n + 1);
        c.take(&scan_ws, scan_local_entries(n + 1));
        c.take(&partial, (int64_t)nbb * 6);
        c.take(&eps_sorted, n);
        c.take(&tmask, n);
        c.take(&estage, n * (kMaxLevel + 1));
    };
    Carve ct;
    take_tmp(ct);
    void* tmp = nullptr;
    DIP_CUDA_TRY(dev_alloc((void**)&tmp, ct.off, s));
    ct = Carve{static_cast<char*>(tmp), 0};
    take_tmp(ct);

    note_launch(); k_bbox<<<nbb, kThreads, 0, s>>>(points, normals, areas, radii, n, partial, t->status,
                                                   build_counter(t, 0), t->bbox);
    query_codes(points, n, t->bbox, 0, t->code, t->perm, t->status, s);
    radix_sort_pairs(t->code, t->perm, ktmp, vtmp, hist, n, 30, s, build_counter(t, 1));
    note_launch(); k_topo_count<<<grid_for(n, kThreads), kThreads, 0, s>>>(
        t->code, n, t->leaf_size, t->max_depth, off, tmask, estage, t->perm, points, normals, areas,
        radii, t->pts, eps_sorted);
    exclusive_scan_local(off, n + 1, scan_ws, reinterpret_cast<uint32_t*>(t->bbox + 9), s,
                         build_counter(t, 2));
    // one read: bbox (5 floats), the status word (float 8), the node count (float 9)
    float hs[10];
    DIP_CUDA_TRY(cudaMemcpyAsync(hs, t->bbox, sizeof(hs), cudaMemcpyDeviceToHost, s));
    DIP_CUDA_TRY(cudaStreamSynchronize(s));
    std::memcpy(t->bbox_host, hs, 5 * sizeof(float));
    int status_host = 0;
    uint32_t nn_host = 0;
    std::memcpy(&status_host, hs + 8, sizeof(int));
    std::memcpy(&nn_host, hs + 9, sizeof(uint32_t));
    DIP_CUDA_TRY(cudaGetLastError());

    auto free_tmp = [&]() { cudaFreeAsync(tmp, s); };
    rc = status_error(status_host, "dipole_build_tree");
    if (rc) {
        free_tmp();
        return rc;
    }
    const int64_t nn = nn_host;
    t->nn = nn;
    rc = alloc_topology(t, nn, s);
    NodeScratch ns;
    if (rc == 0) rc = alloc_nodes(t, ns, s);
    if (rc) {
        free_tmp();
        return rc;
    }
    note_launch(); k_topo_emit<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, nn, t->max_depth, off, scan_ws,
                                                           t->parent, ns.rbits, ns.lvl_cnt, tmask, estage,
                                                           t->first, t->count, t->level,
                                                           t->skip, t->is_leaf, t->leaf_of);
    rc = derive_nodes(t, eps_sorted, ns, true, s);
    free_tmp();
    return rc;
}

int import_tree(dipole_tree* t, const float* points, const float* normals, const float* areas,
                const float* radii, const uint32_t* codes_h, const uint32_t* perm_h,
                const int32_t* first_h, const int32_t* count_h, const int32_t* level_h,
                const int32_t* skip_h, const int32_t* is_leaf_h, cudaStream_t s) {
    const int64_t n = t->n, nn = t->nn;
    int rc = alloc_point_state(t, s);
    if (rc) return rc;
    float* partial = nullptr;
    float* eps_sorted = nullptr;
    const unsigned nbb = grid_for(n, kThreads) < 2u * (unsigned)num_sms() ? grid_for(n, kThreads)
                                                                          : 2u * (unsigned)num_sms();
    auto take_tmp = [&](Carve& c) {
        c.take(&partial, (int64_t)nbb * 6);
        c.take(&eps_sorted, n);
    };
    Carve ct;
    take_tmp(ct);
    void* tmp = nullptr;
    DIP_CUDA_TRY(dev_alloc((void**)&tmp, ct.off, s));
    ct = Carve{static_cast<char*>(tmp), 0};
    take_tmp(ct);
    rc = alloc_topology(t, nn, s);
    if (rc) {
        cudaFreeAsync(tmp, s);
        return rc;
    }
    DIP_CUDA_TRY(cudaMemcpyAsync(t->perm, perm_h, 4 * n, cudaMemcpyHostToDevice, s));
    if (codes_h) DIP_CUDA_TRY(cudaMemcpyAsync(t->code, codes_h, 4 * n, cudaMemcpyHostToDevice, s));
    else DIP_CUDA_TRY(cudaMemsetAsync(t->code, 0, 4 * n, s));
    DIP_CUDA_TRY(cudaMemcpyAsync(t->first, first_h, 4 * nn, cudaMemcpyHostToDevice, s));
    DIP_CUDA_TRY(cudaMemcpyAsync(t->count, count_h, 4 * nn, cudaMemcpyHostToDevice, s));
    DIP_CUDA_TRY(cudaMemcpyAsync(t->level, level_h, 4 * nn, cudaMemcpyHostToDevice, s));
    DIP_CUDA_TRY(cudaMemcpyAsync(t->skip, skip_h, 4 * nn, cudaMemcpyHostToDevice, s));
    DIP_CUDA_TRY(cudaMemcpyAsync(t->is_leaf, is_leaf_h, 4 * nn, cudaMemcpyHostToDevice, s));
    note_launch(); k_bbox<<<nbb, kThreads, 0, s>>>(points, normals, areas, radii, n, partial, t->status,
                                                   build_counter(t, 0), t->bbox);
    note_launch(); k_pack<<<grid_for(n, kThreads), kThreads, 0, s>>>(t->perm, points, normals, areas, radii, n,
                                                      t->pts, eps_sorted);
    DIP_CUDA_TRY(cudaMemsetAsync(t->leaf_of, 0xff, sizeof(int32_t) * n, s));
    note_launch(); k_leaf_of<<<grid_for(nn, kThreads), kThreads, 0, s>>>(nn, t->first, t->count, t->is_leaf,
                                                          t->leaf_of);
    int status_host = 0;
    DIP_CUDA_TRY(cudaMemcpyAsync(&status_host, t->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    DIP_CUDA_TRY(cudaMemcpyAsync(t->bbox_host, t->bbox, 5 * sizeof(float), cudaMemcpyDeviceToHost, s));
    DIP_CUDA_TRY(cudaStreamSynchronize(s));
    DIP_CUDA_TRY(cudaGetLastError());
    rc = status_error(status_host, "dipole_tree_import");
    NodeScratch ns;
    if (rc == 0) rc = alloc_nodes(t, ns, s);
    if (rc == 0) rc = derive_nodes(t, eps_sorted, ns, false, s);
    cudaFreeAsync(tmp, s);
    return rc;
}

}  // namespace dip
