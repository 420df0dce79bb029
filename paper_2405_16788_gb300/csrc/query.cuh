// Pieces shared by the query kernels of traverse.cu (dipole sum and its
// adjoint) and traverse_grad.cu (spatial gradient and its adjoint): the
// kernel arguments, attribute row loads and the persistent grid size.
#pragma once

#include "kernels.cuh"
#include "tree.cuh"

namespace dip {

constexpr int kQThreads = 256;

// A dense grid of query points lo + h (i, j, k), 0 <= i < dim[0] etc., walked
// as 4x4x2 bricks (one 32-query packet each); nb[0] = 0 means no grid.
struct GridSpec {
    float lo[3] = {0.f, 0.f, 0.f};
    float h = 0.f;
    int64_t dim[3] = {0, 0, 0};
    int64_t nb[3] = {0, 0, 0};
};

struct QueryArgs {
    const NodeRec* nodes;
    const PointRec* pts;
    unsigned nn;
    int* status;
    const float* q;
    int64_t nq;
    const uint32_t* qperm;
    float beta;
    int kernel;         // dipole_kernel of the tree
    int C;
    int G;              // channels [0, G) with the foreshortening term, [G, C) without
    int Cp;
    const void* mu;
    const float* S;
    const uint16_t* S16;  // S rounded to bf16, [nn, srow16(Cp)] (bf16 attributes), or NULL
    float* out;         // D [q, C]
    float* gout;        // grad D [q, C, 3]
    const float* g;     // dL/dD [q, C]
    const float* gg;    // dL/d(grad D) [q, C, 3]
    float* dS;
    float* dmu;
    float* dE;          // [nn] d eps~_t sums (kAdjointGeom)
    float* dgeo;        // [n, 4] opened-leaf normal (xyz) and radius (w) terms (kAdjointGeom)
    float* gq;          // dL/dx [q, 3] (kForwardGradDot)
    int accumulate;     // gq: add to it (non-ranged; ranged items always add)
    int32_t* counts;
    int32_t* ucounts;   // [packets, 4] warp steps, far steps, opened-leaf point loads, lanes (kCount)
    unsigned long long* work;
    int64_t npts;            // points of the tree (leaf point ranges lie in [0, npts))
    int64_t n_slots;         // entries of items (ranged work)
    // treelet: the top levels of the tree staged in shared memory (forward, up to
    // 4 channels); walk states are keys (node << kTLSlotBits | slot hint)
    const void* tl;             // TLRec [kTLMax]
    const uint32_t* tl_node;    // [kTLMax] treelet node ids, ascending
    const NodeRec* nodes_k;     // node records with meta.x = the packed key of the skip
    const uint32_t* porder;  // packet (or item) order, or NULL for sorted order
    GridSpec grid;           // dense-grid queries instead of q / qperm
    uint32_t* plan;          // query plan being written (forward): kPlanWords per packet
    const uint4* items;      // ranged work items {packet, lo, hi, part}, read in porder if set
    const unsigned* n_items; // number of valid items
    const int32_t* parent;   // node parents (ranged items)
};

// Query plan, kPlanWords words per 32-query packet: [0] the packet's warp
// steps (all its items together); [1..3] the nodes its lower forward item
// visited at its steps 128, 256, 384; [4] the node where the forward split
// the walk; [5..7] the same as [1..3] for the upper item (0 = none).  Any
// increasing subsequence of [1..7] inside (0, nn) partitions the walk, so a
// stale or foreign plan changes only the balance of an adjoint, never a result.
constexpr unsigned kCutSteps = 128u;
constexpr unsigned kPartCuts = 3u;
constexpr unsigned kPlanWords = 8u;

// n attribute values (n = 1, 2 or 4; p aligned to n elements) as floats.
template <typename AT>
__device__ __forceinline__ void load_row(const AT* p, float* v, int n);

template <>
__device__ __forceinline__ void load_row<float>(const float* p, float* v, int n) {
    if (n == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else if (n == 2) {
        const float2 a = __ldg(reinterpret_cast<const float2*>(p));
        v[0] = a.x; v[1] = a.y;
    } else {
        v[0] = __ldg(p);
    }
}

template <>
__device__ __forceinline__ void load_row<__nv_bfloat16>(const __nv_bfloat16* p, float* v, int n) {
    if (n == 4) {
        const uint2 a = __ldg(reinterpret_cast<const uint2*>(p));
        v[0] = __uint_as_float(a.x << 16); v[1] = __uint_as_float(a.x & 0xffff0000u);
        v[2] = __uint_as_float(a.y << 16); v[3] = __uint_as_float(a.y & 0xffff0000u);
    } else if (n == 2) {
        const unsigned a = __ldg(reinterpret_cast<const unsigned*>(p));
        v[0] = __uint_as_float(a << 16); v[1] = __uint_as_float(a & 0xffff0000u);
    } else {
        v[0] = __bfloat162float(p[0]);
    }
}

// Blocks of a persistent query grid: enough for one warp per 32-query packet,
// at most what stays resident on all SMs (per_sm caches the occupancy).
template <typename Kernel>
inline unsigned query_grid(Kernel kernel, int64_t nq, int& per_sm) {
    if (per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kQThreads, 0);
        if (per_sm < 1) per_sm = 1;
    }
    const int64_t need = (nq + 31) / 32;
    const int64_t blocks = (need + (kQThreads / 32) - 1) / (kQThreads / 32);
    const int64_t cap = (int64_t)num_sms() * per_sm;
    return (unsigned)(blocks < cap ? blocks : cap);
}

// Launch the gradient query kernels (traverse_grad.cu) for mode kForwardGrad
// or kAdjointGrad.
int dispatch_grad(const dipole_tree* t, int mode, const QueryArgs& a, cudaStream_t s);

}  // namespace dip
