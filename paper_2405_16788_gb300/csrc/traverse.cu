// Barnes-Hut primal and adjoint queries (Alg. 1; Sec. 6.1, eq. farfield;
// Sec. 6.2 and App. C, eq. farfield_gradient).
//
// Persistent, warp-cooperative, stackless traversal.  Queries are sorted
// along a Hilbert curve, so the 32 queries of a warp are neighbours.  The tree is in
// depth-first preorder with skip indices: a query at node t moves to skip[t]
// when t is far or a leaf, else to t+1 (its first child).  Every lane keeps
// its own next node; the warp visits the smallest of them, so all lanes that
// need a node read it in the same instruction (one 32-byte broadcast from L2
// instead of up to 32 scattered reads), and lanes whose next node lies
// further on wait.  Each lane therefore takes exactly the decisions of its
// own depth-first traversal (Alg. 1), in the same order.
//
// The adjoint (stage 1) recomputes the traversal rather than storing
// interaction lists.  The lanes taking a far node are all at that node in the
// same step, so their contributions to dS_t are summed inside the warp before
// one set of atomics; the same holds for the points of an opened leaf.
#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

#include "query.cuh"

namespace dip {
namespace {

// Value v (0..23) of a group of 24 bf16 values held in three 16-byte vectors,
// as a float (v is a compile-time index after unrolling).
__device__ __forceinline__ float bf16_in_group(const uint4* g, int v) {
    const uint4 q = g[v >> 3];
    const int w = (v >> 1) & 3;
    const unsigned u = w == 0 ? q.x : w == 1 ? q.y : w == 2 ? q.z : q.w;
    return __uint_as_float((v & 1) ? (u & 0xffff0000u) : (u << 16));
}

// Treelet (the upper tree in shared memory): nodes of depth < kTLDepth in
// preorder, at most kTLMax, with their records, the packed keys of their skip
// and first child and the first moment chunk (up to 4 channels).
constexpr int kTLDepth = 3;
constexpr int kTLMax = 80;
constexpr unsigned kTLSlotBits = 7, kTLInv = 127u;
struct __align__(16) TLRec {
    float4 geo;
    int4 meta;      // meta.x: the packed key of the skip
    uint4 ext;      // ext.x: the packed key of the first child
    float4 mom[3];  // the moment row's first 12 floats
};

// The slot of node u among the ascending treelet node ids, kTLInv if absent.
__device__ __forceinline__ unsigned tl_slot_of(const uint32_t* ids, int cnt, unsigned u) {
    int lo = 0, hi = cnt;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ids[mid] < u) lo = mid + 1; else hi = mid;
    }
    return (lo < cnt && ids[lo] == u) ? (unsigned)lo : kTLInv;
}

// RANGED: each work item is a preorder range [lo, hi) of one packet's walk; a
// lane enters it in the state its depth-first walk has at lo (decided by lo's
// ancestors alone) and stops at hi, so the items of a packet together visit
// exactly the packet's nodes, each once.  The forward splits every packet in
// two (k_fwd_items) and its two parts add into the zeroed output (a sum of two
// floats does not depend on their order); the adjoint with a plan cuts every
// walk at the nodes the forward recorded (k_plan_items).
//
// KERN: 0 the regularized kernel, 1 the desingularized one, 2 the regularized
// kernel with channels [a.G, C) interpolated without the foreshortening term
// (a point adds A rho(r/eps)/(4 pi r^2) mu, a far node rho(d/eps~)/(4 pi d^2)
// M with M = sum A mu in the first slot of the channel's moment row).
//
// M16: far-node moments from the bf16 copy (DIPOLE_BF16_MOMENTS).  TL: the
// treelet (dipole_set_treelet): walk states are packed keys, node << 7 | the
// node's treelet slot (127 outside it), carried by every skip and child key,
// so a treelet node is read from shared memory without a lookup.
template <int CP, typename AT, int MODE, int KERN, bool RANGED, bool M16, bool TL>
__global__ void __launch_bounds__(kQThreads, (MODE == kForward && CP <= 4) ? 6
                                          : (MODE == kForward && CP <= 32) ? 3 : (MODE == kForward && CP <= 36) ? 2 : 1)
k_query(const QueryArgs a) {
    constexpr bool NF = KERN == 2;       // some channels skip the foreshortening term
    constexpr int KR = NF ? 0 : KERN;    // the radial factor's kernel
    constexpr int SR = srow(CP);
    constexpr int SR16 = srow16(CP);
    constexpr bool kS16 = MODE == kForward && M16;  // far-node moments from the bf16 copy
    constexpr bool kTL = TL && MODE == kForward && CP <= 4 && !M16;
    constexpr int CH = CP < 4 ? CP : 4;  // channels per chunk
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const NodeRec* __restrict__ nodes = kTL ? a.nodes_k : a.nodes;
    const PointRec* __restrict__ pts = a.pts;
    const unsigned nn = a.nn;

    // the treelet, staged once per block by one bulk copy (no multicast)
    __shared__ TLRec sh_tl[kTL ? kTLMax : 1];
    __shared__ __align__(16) uint32_t sh_tln[kTL ? kTLMax : 4];
    __shared__ __align__(8) unsigned long long sh_bar;
    __shared__ int sh_tl_ok;
    if (kTL) {
        const unsigned bar = (unsigned)__cvta_generic_to_shared(&sh_bar);
        constexpr unsigned kBytes = (unsigned)(sizeof(TLRec) * kTLMax + sizeof(uint32_t) * kTLMax);
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            sh_tl_ok = 1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}"
                         ::"r"(bar), "r"(kBytes) : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                ::"r"((unsigned)__cvta_generic_to_shared(sh_tl)), "l"(a.tl),
                "r"((unsigned)(sizeof(TLRec) * kTLMax)), "r"(bar) : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                ::"r"((unsigned)__cvta_generic_to_shared(sh_tln)), "l"(a.tl_node),
                "r"((unsigned)(sizeof(uint32_t) * kTLMax)), "r"(bar) : "memory");
        }
        // bounded wait for phase 0
        unsigned done = 0;
        for (int it = 0; it < (1 << 22) && !done; ++it) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                : "=r"(done) : "r"(bar) : "memory");
        }
        if (!done) {
            atomicOr(a.status, kStatusTraversal);
            sh_tl_ok = 0;  // (benign race: every failing thread writes 0)
            // the copies may still be in flight: wait for them again, bounded
            for (int it = 0; it < (1 << 22) && !done; ++it) {
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                    : "=r"(done) : "r"(bar) : "memory");
            }
        }
        __syncthreads();
        if (!sh_tl_ok) return;
    }
    auto key_of = [&](unsigned u) -> unsigned {  // packed key of node u (treelet search)
        return kTL ? ((u << kTLSlotBits) | tl_slot_of(sh_tln, kTLMax, u)) : u;
    };

    for (;;) {
        unsigned long long pk = 0;
        if (lane == 0) pk = atomicAdd(a.work, 1ull);
        pk = __shfl_sync(FULL, pk, 0);
        int64_t pm;
        unsigned lo = 0u, hi = nn;
        unsigned half = 0u;  // forward item: 0 lower, 1 upper part of the walk
        if (RANGED) {
            if (pk >= *a.n_items) break;
            const uint64_t slot = a.porder ? a.porder[pk] : pk;
            if (!in_bounds(slot < (uint64_t)a.n_slots, a.status)) continue;
            const uint4 it = a.items[slot];
            pm = (int64_t)it.x;
            lo = it.y;
            hi = it.z;
            half = it.w;
            if (!in_bounds(lo <= hi && hi <= nn && pm * 32 < a.nq, a.status)) continue;
        } else {
            if ((int64_t)pk * 32 >= a.nq) break;
            pm = (int64_t)(a.porder ? a.porder[pk] : pk);  // packet index in sorted order
            if (!in_bounds(pm * 32 < a.nq, a.status)) continue;
        }
        bool valid;
        int64_t qo;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f;
        if (a.grid.nb[0] > 0) {
            // dense grid: packet pm is the 4x4x2 brick pm (bricks x-fastest);
            // the lane's point is lo + h * (i, j, k), one rounding per operation
            const int64_t bx = pm % a.grid.nb[0], r = pm / a.grid.nb[0];
            const int64_t by = r % a.grid.nb[1], bz = r / a.grid.nb[1];
            const int64_t i = 4 * bx + (lane & 3), j = 4 * by + ((lane >> 2) & 3), k = 2 * bz + (lane >> 4);
            valid = i < a.grid.dim[0] && j < a.grid.dim[1] && k < a.grid.dim[2];
            qo = valid ? i + a.grid.dim[0] * (j + a.grid.dim[1] * k) : 0;
            if (valid) {
                x0 = __fadd_rn(a.grid.lo[0], __fmul_rn((float)i, a.grid.h));
                x1 = __fadd_rn(a.grid.lo[1], __fmul_rn((float)j, a.grid.h));
                x2 = __fadd_rn(a.grid.lo[2], __fmul_rn((float)k, a.grid.h));
            }
        } else {
            const int64_t qi = pm * 32 + lane;
            valid = qi < a.nq;
            qo = valid ? (a.qperm ? (int64_t)a.qperm[qi] : qi) : 0;
            if (valid && !in_bounds(qo >= 0 && qo < a.nq, a.status)) {
                valid = false;
                qo = 0;
            }
            if (valid) { x0 = a.q[3 * qo]; x1 = a.q[3 * qo + 1]; x2 = a.q[3 * qo + 2]; }
        }

        // Forward sums: plain float partial sums (part), folded every kFoldSteps
        // warp steps into a Kahan-compensated sum (acc, cmp) for up to 36
        // channels; per-term Kahan for more (register budget).  From 4 channels
        // on the Kahan pairs live in shared memory (one column per thread, read
        // and written only at a fold), which leaves the registers to the walk:
        // six blocks per SM without spills in the walk at 4 channels, three from
        // 8 to 32, two at 36.
        constexpr bool kBlocked = CP <= 36;
        constexpr unsigned kFoldSteps = 32;
        constexpr bool kSmem = MODE == kForward && CP >= 4 && CP <= 36;
        constexpr int kRegSums = (MODE == kForward && !kSmem) ? CP : 1;
        __shared__ float sh_acc[kSmem ? CP : 1][kQThreads], sh_cmp[kSmem ? CP : 1][kQThreads];
        float acc[kRegSums], cmp[kRegSums];
        float part[MODE == kForward && kBlocked ? CP : 1];
        float g[MODE == kAdjoint ? CP : 1];
        auto kahan_into = [&](int c, float v) {  // channel c's Kahan sum += v
            if (kSmem) kahan_add(sh_acc[kSmem ? c : 0][threadIdx.x], sh_cmp[kSmem ? c : 0][threadIdx.x], v);
            else kahan_add(acc[kSmem ? 0 : c], cmp[kSmem ? 0 : c], v);
        };
        auto kahan_total = [&](int c) -> float {
            return kSmem ? __fsub_rn(sh_acc[kSmem ? c : 0][threadIdx.x], sh_cmp[kSmem ? c : 0][threadIdx.x])
                         : __fsub_rn(acc[kSmem ? 0 : c], cmp[kSmem ? 0 : c]);
        };
        if (MODE == kForward) {
#pragma unroll
            for (int c = 0; c < CP; ++c) {
                if (kSmem) {
                    sh_acc[kSmem ? c : 0][threadIdx.x] = 0.f;
                    sh_cmp[kSmem ? c : 0][threadIdx.x] = 0.f;
                } else {
                    acc[kSmem ? 0 : c] = 0.f;
                    cmp[kSmem ? 0 : c] = 0.f;
                }
            }
            if (kBlocked) {
#pragma unroll
                for (int c = 0; c < CP; ++c) part[c] = 0.f;
            }
        }
        // adjoint: the upstream gradient, scaled by 1/(4 pi) and put into each
        // chunk's lane_channel_order (see adjoint_far_reduce)
        int ord[CH];
        lane_channel_order<CH>(lane, ord);
        if (MODE == kAdjoint) {
#pragma unroll
            for (int c0 = 0; c0 < CP; c0 += CH) {
                float gc[CH];
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    gc[c] = (valid && c0 + c < a.C) ? a.g[qo * a.C + c0 + c] * kInv4Pi : 0.f;
#pragma unroll
                for (int i = 0; i < CH; ++i) {
                    float v = gc[0];
#pragma unroll
                    for (int c = 1; c < CH; ++c) v = (ord[i] == c) ? gc[c] : v;
                    g[c0 + i] = v;
                }
            }
        }
        auto add_term = [&](int c, float v) {
            if (MODE == kForward) {
                if (kBlocked) part[c] += v;
                else kahan_into(c, v);
            }
        };
        int n_tested = 0, n_far = 0, n_pts = 0;
        unsigned u_far = 0, u_pts = 0;  // warp counts (kCount with a.ucounts)

        unsigned next = key_of(valid ? lo : nn);
        if (RANGED && lo > 0u && lo < nn) {
            // the walk reaches lo unless an ancestor of lo is far; it then
            // resumes at the topmost far ancestor's skip, the largest of them
            const unsigned start = kTL ? (next >> kTLSlotBits) : next;
            int32_t u = a.parent[lo];
            for (int up = 0; up <= kMaxLevel + 1 && u >= 0; ++up) {
                if (!in_bounds(u < (int32_t)nn, a.status)) break;
                const float4 geo = __ldg(&nodes[u].geo);
                const int4 meta = __ldg(&nodes[u].meta);
                const float dx = __fsub_rn(x0, geo.x);
                const float dy = __fsub_rn(x1, geo.y);
                const float dz = __fsub_rn(x2, geo.z);
                const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                const float R = __fmul_rn(a.beta, geo.w);
                if (start == lo && d2 > __fmul_rn(R, R)) next = max(next, (unsigned)meta.x);  // packed with kTL
                u = a.parent[u];
            }
        }
        unsigned steps = 0;
        // bf16 moments (bf16 attributes, forward): a row is read in groups of up
        // to 8 channels, 24 bf16 values in three 16-byte loads
        auto load_group16 = [&](unsigned node, int c0, uint4* gp) {
            const uint4* p = reinterpret_cast<const uint4*>(a.S16 + (size_t)node * SR16 + 3 * c0);
            const int nv = 3 * ((CP - c0) < 8 ? (CP - c0) : 8);
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (8 * j < nv) gp[j] = __ldg(p + j);
        };
        // one warp step of the walk; false once the walk is over
        auto walk_step = [&](const bool fold_here) -> bool {
            const unsigned key = __reduce_min_sync(FULL, next);
            const unsigned n = kTL ? key >> kTLSlotBits : key;
            if (MODE == kForward) {
                if (n >= hi) return false;
            } else if ((n >= hi) | (steps >= nn)) {  // a well-formed tree needs at most nn steps
                if (n < hi && lane == 0) atomicOr(a.status, kStatusTraversal);
                return false;
            }
            ++steps;
            const unsigned slot = kTL ? (key & kTLInv) : kTLInv;
            float4 geo;
            int4 meta;
            unsigned ckey;
            // forward: the node's first moment chunk is loaded before the far test
            // so that its latency overlaps the test (most visited nodes are far
            // for some lane)
            float4 s_first[MODE == kForward && !kS16 ? (3 * CH + 3) / 4 : 1];
            uint4 grp[kS16 ? 3 : 1];  // bf16 moments: the row's current group of 8 channels
            if (kTL && slot != kTLInv) {
                const TLRec& r = sh_tl[kTL ? slot : 0];
                geo = r.geo;
                meta = r.meta;
                ckey = r.ext.x;
#pragma unroll
                for (int j = 0; j < (3 * CH + 3) / 4; ++j) s_first[j] = r.mom[j];
            } else {
                geo = __ldg(&nodes[n].geo);
                meta = __ldg(&nodes[n].meta);
                ckey = kTL ? key + (1u << kTLSlotBits) : n + 1u;
                if (MODE == kForward && kS16) {
                    load_group16(n, 0, grp);
                } else if (MODE == kForward) {
                    const float4* sp = reinterpret_cast<const float4*>(a.S + (size_t)n * SR);
#pragma unroll
                    for (int j = 0; j < (3 * CH + 3) / 4; ++j) s_first[j] = __ldg(sp + j);
                }
            }
            const bool act = next == key;
            // far test of Alg. 1 in a fixed float operation order
            const float dx = __fsub_rn(x0, geo.x);
            const float dy = __fsub_rn(x1, geo.y);
            const float dz = __fsub_rn(x2, geo.z);
            const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
            const float R = __fmul_rn(a.beta, geo.w);
            const bool far = act && (d2 > __fmul_rn(R, R));
            const bool leaf = meta.z > 0;
            const bool open_leaf = act && !far && leaf;
            if (act) next = (far || leaf) ? (unsigned)meta.x : ckey;

            if (MODE == kCount) {
                if (act) {
                    ++n_tested;
                    if (far) ++n_far;
                    else if (leaf) n_pts += meta.z;
                }
                if (a.ucounts) {
                    // the warp's own fetches: the moment row of a node some lane
                    // takes as far, the points of a leaf some lane opens
                    if (__any_sync(FULL, far)) ++u_far;
                    if (__any_sync(FULL, open_leaf)) u_pts += (unsigned)meta.z;
                }
            } else {
                if (__any_sync(FULL, far)) {
                    // far field, eq. farfield: rho(d/eps~) S.(p~ - x) / d^3 (1/4pi applied at the end)
                    float k = 0.f, wf = 0.f;
                    if (far) {
                        k = radial_over_d3(d2, __int_as_float(meta.w), KR);
                        if (NF) wf = k * (d2 * rsqrtf(d2));  // rho(d/eps~)/d^2
                    }
                    const float vx = -k * dx, vy = -k * dy, vz = -k * dz;
                    if (MODE == kForward) {
                        const float* Sr = a.S + (size_t)n * SR;
#pragma unroll
                        for (int c0 = 0; c0 < CP; c0 += CH) {
                            float s[3 * CH + 3];
                            if (kS16) {
                                if (c0 > 0 && c0 % 8 == 0) load_group16(n, c0, grp);
#pragma unroll
                                for (int j = 0; j < 3 * CH; ++j) s[j] = bf16_in_group(grp, 3 * (c0 % 8) + j);
                            } else {
#pragma unroll
                                for (int j = 0; j < (3 * CH + 3) / 4; ++j) {
                                    const float4 q4 = c0 == 0 ? s_first[j] : __ldg(reinterpret_cast<const float4*>(Sr + 3 * c0) + j);
                                    s[4 * j] = q4.x; s[4 * j + 1] = q4.y; s[4 * j + 2] = q4.z; s[4 * j + 3] = q4.w;
                                }
                            }
#pragma unroll
                            for (int c = 0; c < CH; ++c) {
                                const bool nf = NF && c0 + c >= a.G;
                                // blocked sums: k = wf = 0 on lanes that did not take the
                                // node, whose term is an exact zero
                                if (CP <= 4 && kBlocked) {
                                    // -k (S.(x - p~)) = k S.(p~ - x): the kernel factor folded
                                    // into the accumulation (fewer instructions; from 8
                                    // channels, latency bound, the scaled vector is faster)
                                    const float dot =
                                        fmaf(dx, s[3 * c], fmaf(dy, s[3 * c + 1], dz * s[3 * c + 2]));
                                    part[c0 + c] =
                                        nf ? fmaf(s[3 * c], wf, part[c0 + c]) : fmaf(-k, dot, part[c0 + c]);
                                } else {
                                    float term = fmaf(vx, s[3 * c], fmaf(vy, s[3 * c + 1], vz * s[3 * c + 2]));
                                    if (nf) term = s[3 * c] * wf;
                                    if (kBlocked) part[c0 + c] += term;
                                    else if (far) add_term(c0 + c, term);
                                }
                            }
                        }
                    } else if (MODE == kAdjoint && !NF) {
                        // eq. farfield_gradient: dS_t^c += rho (p~ - x)/d^3 g^c
                        float* dst = a.dS + (size_t)n * SR;
#pragma unroll
                        for (int c0 = 0; c0 < CP; c0 += CH)
                            adjoint_far_reduce<CH>(vx, vy, vz, g + c0, dst + 3 * c0, ord[0], lane);
                    } else if (MODE == kAdjoint) {
                        // channels without the foreshortening term add rho/d^2 g^c to
                        // the first slot of their row; the lanes' channel order
                        // (ord) decides which vector each slot of v gets
                        float* dst = a.dS + (size_t)n * SR;
#pragma unroll
                        for (int c0 = 0; c0 < CP; c0 += CH) {
                            float v[3 * CH];
#pragma unroll
                            for (int i = 0; i < CH; ++i) {
                                const bool geo = c0 + ord[i] < a.G;
                                const float gi = g[c0 + i];
                                v[3 * i] = (geo ? vx : wf) * gi;
                                v[3 * i + 1] = geo ? vy * gi : 0.f;
                                v[3 * i + 2] = geo ? vz * gi : 0.f;
                            }
                            adjoint_vec_reduce<CH>(v, dst + 3 * c0, ord[0], lane);
                        }
                    }
                }

                // opened-leaf point term: the dipole kernel times A_m n_m . (p_m - x);
                // kn: without the foreshortening term, rho(r/eps) A_m / r^2
                auto point_k2 = [&](const PointRec& pr, float& kn) {
                    float k = 0.f;
                    kn = 0.f;
                    if (open_leaf) {
                        const float ex = pr.geo.x - x0, ey = pr.geo.y - x1, ez = pr.geo.z - x2;
                        const float r2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
                        if (r2 > 0.f) {
                            const float kr = radial_over_d3(r2, pr.geo.w, KR);
                            k = kr * fmaf(pr.w.x, ex, fmaf(pr.w.y, ey, pr.w.z * ez));
                            if (NF) kn = kr * pr.w.w * (r2 * rsqrtf(r2));
                        }
                    }
                    return k;
                };
                auto point_k = [&](const PointRec& pr) {
                    float kn;
                    return point_k2(pr, kn);
                };
                if (MODE == kAdjoint && NF && __any_sync(FULL, open_leaf)) {
                    // opened leaf, one point at a time: each channel takes the
                    // kernel of its kind
                    const int f = meta.y;
                    const int cnt =
                        in_bounds(f >= 0 && meta.z >= 0 && (int64_t)f + meta.z <= a.npts, a.status) ? meta.z : 0;
                    for (int j = 0; j < cnt; ++j) {
                        float kn;
                        const float kd = point_k2(pts[f + j], kn);
                        float* dst = a.dmu + (size_t)(f + j) * CP;
#pragma unroll
                        for (int c0 = 0; c0 < CP; c0 += CH) {
                            float v[CH];
#pragma unroll
                            for (int i = 0; i < CH; ++i) v[i] = (c0 + ord[i] < a.G ? kd : kn) * g[c0 + i];
                            adjoint_scalar_reduce<CH>(v, dst + c0, ord[0], lane);
                        }
                    }
                } else if (MODE == kAdjoint && __any_sync(FULL, open_leaf)) {
                    // opened leaf, points in pairs (adjoint_point_pair_reduce)
                    const int f = meta.y;
                    const int cnt =
                        in_bounds(f >= 0 && meta.z >= 0 && (int64_t)f + meta.z <= a.npts, a.status) ? meta.z : 0;
                    for (int j = 0; j < cnt; j += 2) {
                        const bool two = j + 1 < cnt;
                        const float ka = point_k(pts[f + j]);
                        const float kb = two ? point_k(pts[f + j + 1]) : 0.f;
                        float* dst = a.dmu + (size_t)(f + j) * CP;
#pragma unroll
                        for (int c0 = 0; c0 < CP; c0 += CH)
                            adjoint_point_pair_reduce<CH>(ka, kb, g + c0, dst + c0, CP, two, ord[0],
                                                          lane);
                    }
                } else if (MODE != kAdjoint && __any_sync(FULL, open_leaf)) {
                    // opened leaf: exact sum over its points (eq. dipole_sum)
                    const int f = meta.y;
                    const int cnt =
                        in_bounds(f >= 0 && meta.z >= 0 && (int64_t)f + meta.z <= a.npts, a.status) ? meta.z : 0;
                    if (MODE == kForward) {
                        prefetch_l1(pts + f, cnt * (int)sizeof(PointRec), lane);
                        prefetch_l1(reinterpret_cast<const AT*>(a.mu) + (size_t)f * CP,
                                    cnt * CP * (int)sizeof(AT), lane);
                    }
                    for (int j = 0; j < cnt; ++j) {
                        float kn;
                        const float k = point_k2(pts[f + j], kn);
                        if (MODE == kForward) {
                            const AT* mrow = reinterpret_cast<const AT*>(a.mu) + (size_t)(f + j) * CP;
#pragma unroll
                            for (int c0 = 0; c0 < CP; c0 += CH) {
                                float m[CH];
                                load_row<AT>(mrow + c0, m, CH);
#pragma unroll
                                for (int c = 0; c < CH; ++c) {
                                    const float kk = NF && c0 + c >= a.G ? kn : k;
                                    if (kBlocked) part[c0 + c] = fmaf(kk, m[c], part[c0 + c]);  // k = kn = 0 off the leaf
                                    else if (open_leaf) add_term(c0 + c, kk * m[c]);
                                }
                            }
                        }
                    }
                }
                if (MODE == kForward && fold_here && (steps % kFoldSteps) == 0u) {
                    if (steps > nn) {  // the forward checks the bound every kFoldSteps steps
                        if (lane == 0) atomicOr(a.status, kStatusTraversal);
                        return false;
                    }
                    if (kBlocked) {
#pragma unroll
                        for (int c = 0; c < CP; ++c) {
                            kahan_into(c, part[c]);
                            part[c] = 0.f;
                        }
                    }
                    // plan record: the node of every kCutSteps-th step of this part
                    if (RANGED && a.plan && lane == 0 && (steps & (kCutSteps - 1u)) == 0u &&
                        steps <= kCutSteps * kPartCuts)
                        a.plan[(size_t)pm * kPlanWords + 1u + 4u * half + steps / kCutSteps - 1u] = n;
                }
            }
            return true;
        };
        if (MODE == kForward) {
            // two steps per turn: the fold (every kFoldSteps steps, an even count)
            // is only tested after the second
            for (;;) {
                if (!walk_step(false)) break;
                if (!walk_step(true)) break;
            }
        } else {
            while (walk_step(true)) {
            }
        }
        if (MODE == kForward && kBlocked) {
#pragma unroll
            for (int c = 0; c < CP; ++c) kahan_into(c, part[c]);
        }

        if (RANGED && MODE == kForward && a.plan && lane == 0)
            atomicAdd(a.plan + (size_t)pm * kPlanWords, steps);
        if (valid) {
            if (MODE == kForward) {
#pragma unroll
                for (int c = 0; c < CP; ++c) {
                    if (c >= a.C) continue;
                    const float v = kahan_total(c) * kInv4Pi;
                    if (RANGED) atomicAdd(a.out + qo * a.C + c, v);  // the two parts of a packet
                    else a.out[qo * a.C + c] = v;
                }
            } else if (MODE == kCount && a.counts) {
                a.counts[3 * qo] = n_tested;
                a.counts[3 * qo + 1] = n_far;
                a.counts[3 * qo + 2] = n_pts;
            }
        }
        if (MODE == kCount && a.ucounts) {
            const unsigned lanes = __popc(__ballot_sync(FULL, valid));
            if (lane == 0) {
                int32_t* u = a.ucounts + 4 * pm;
                u[0] = (int32_t)steps;
                u[1] = (int32_t)u_far;
                u[2] = (int32_t)u_pts;
                u[3] = (int32_t)lanes;
            }
        }
    }
}

// ------------------------------------------------------------------ item order
// Work items run in decreasing order of an estimated cost, so that the long
// ones start first and the queue's tail is short.  The order only needs to be
// coarse: an item goes to one of 256 buckets of its cost on a log scale (16 per
// octave; bucket 0 holds the most costly).  The kernel that makes the items
// counts them per bucket; the last of its blocks to finish (an arrival
// counter: no block waits for another) turns the counts into bucket starts,
// and k_order_place puts every item into its bucket.  The order inside a
// bucket is that of arrival, which changes no result: the forward's two parts
// of a query add into its zeroed output (a sum of two floats, either order),
// and the adjoint's node sums are atomic adds in any case.
// ostate: [0, 256) counts, [256, 512) bucket cursors, [512] arrivals; zeroed
// before the item kernel.
constexpr int kOrderBuckets = 256;
constexpr int kOrderStateWords = 2 * kOrderBuckets + 1;
constexpr uint32_t kNoBucket = 0xffffffffu;

__device__ __forceinline__ uint32_t cost_bucket(uint32_t c) {
    const uint32_t x = min(c, 0x7fffffffu) + 1u;
    const int e = 31 - __clz(x);
    const uint32_t frac = e >= 4 ? (x >> (e - 4)) & 15u : (x << (4 - e)) & 15u;
    const uint32_t f = min(16u * (uint32_t)e + frac, (uint32_t)kOrderBuckets - 1u);
    return (uint32_t)kOrderBuckets - 1u - f;
}

// End of an item kernel: add the block's bucket counts (sh, shared) to ostate;
// the last block writes the exclusive bucket starts.  Called by every thread.
__device__ __forceinline__ void order_counts_flush(const uint32_t* sh, uint32_t* ostate) {
    __shared__ bool last;
    __syncthreads();
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x)
        if (sh[b]) atomicAdd(ostate + b, sh[b]);
    __threadfence();
    if (threadIdx.x == 0) last = atomicAdd(ostate + 2 * kOrderBuckets, 1u) == gridDim.x - 1u;
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    const int lane = threadIdx.x;
    constexpr int K = kOrderBuckets / 32;
    uint32_t c[K], sum = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        c[k] = __ldcg(ostate + K * lane + k);
        sum += c[k];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    uint32_t run = inc - sum;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        ostate[kOrderBuckets + K * lane + k] = run;
        run += c[k];
    }
}

__global__ void k_order_place(const uint32_t* __restrict__ ibucket, int64_t ni,
                              uint32_t* __restrict__ ostate, uint32_t* __restrict__ porder) {
    const int lane = threadIdx.x & 31;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < ni; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        const uint32_t b = i < ni ? ibucket[i] : kNoBucket;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (b != kNoBucket && lane == leader) base = atomicAdd(ostate + kOrderBuckets + b, __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (b != kNoBucket) porder[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
    }
}

// Work items of the ranged adjoint: packet p's walk is cut at the increasing
// nodes of plan words [1..7] inside (0, nn); item k of p goes to slot
// p * kPlanWords + k, in the bucket of its estimated steps (the packet's steps
// shared evenly); unused slots get no bucket.
__global__ void k_plan_items(const uint32_t* plan, int64_t np, unsigned nn, uint4* items,
                             uint32_t* ibucket, unsigned* n_items, uint32_t* ostate) {
    __shared__ uint32_t sh[kOrderBuckets];
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t* w = plan + p * kPlanWords;
        unsigned cut[kPlanWords - 1];
        unsigned ncut = 0, prev = 0;
        for (unsigned k = 1; k < kPlanWords; ++k) {
            const unsigned c = w[k];
            if (c > prev && c < nn) {
                cut[ncut++] = c;
                prev = c;
            }
        }
        const unsigned est = max(1u, w[0] / (ncut + 1u));
        const uint32_t bk = cost_bucket(est);
        unsigned lo = 0;
        for (unsigned k = 0; k < kPlanWords; ++k) {
            const int64_t slot = p * kPlanWords + k;
            if (k <= ncut) {
                const unsigned hi = k < ncut ? cut[k] : nn;
                items[slot] = make_uint4((unsigned)p, lo, hi, 0u);
                ibucket[slot] = bk;
                lo = hi;
            } else {
                items[slot] = make_uint4((unsigned)p, nn, nn, 0u);
                ibucket[slot] = kNoBucket;
            }
        }
        atomicAdd(&sh[bk], ncut + 1u);
        atomicAdd(n_items, ncut + 1u);
    }
    order_counts_flush(sh, ostate);
}

// First index i in [0, n) with v[i] >= x (n if none), v sorted, found by
// the 32 lanes of a warp together: each round every lane probes one of 32
// evenly spaced positions and a ballot keeps the interval between the last
// probe below x and the first at or above it (a 32-ary search: four rounds of
// one load each for a million entries).  Must be called by all 32 lanes with
// the same x; every lane gets the result.
__device__ __forceinline__ int64_t warp_lower_bound_u32(const uint32_t* v, int64_t n, uint32_t x,
                                                        int lane) {
    int64_t lo = 0, hi = n;  // the answer lies in [lo, hi]
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t p = lo + (int64_t)(lane + 1) * step - 1;
        const bool below = p < hi && v[p] < x;
        const int k = __popc(__ballot_sync(0xffffffffu, below));
        const int64_t nlo = lo + (int64_t)k * step;
        hi = min(nlo + step - 1, hi);  // v[lo + (k + 1) step - 1] >= x, or hi
        lo = min(nlo, hi);
    }
    const int64_t p = lo + lane;
    const bool below = p < hi && v[p] < x;
    return lo + __popc(__ballot_sync(0xffffffffu, below));
}

// The forward's two items per packet (one warp per packet): the walk is cut
// at the leaf holding the middle point (Morton order) of those whose codes lie
// between the smallest and largest Morton code of the packet's queries, which
// puts about half of the packet's near-field work on each side.  Both items go
// to the bucket of that point count (a proxy of the walk's length).  The cut
// is also written to the plan (word 4) when one is recorded.
__global__ void k_fwd_items(const float* q, const uint32_t* qperm, int64_t nq, int64_t np,
                            const float* bbox, const uint32_t* pcode, int64_t n,
                            const int32_t* leaf_of, unsigned nn, uint4* items, unsigned* n_items,
                            uint32_t* plan, uint32_t* ibucket, uint32_t* ostate) {
    __shared__ uint32_t sh[kOrderBuckets];
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < np; p += warps) {
        const int64_t i = p * 32 + lane;
        uint32_t cmin = 0xffffffffu, cmax = 0u;
        if (i < nq) {
            const int64_t o = qperm[i];
            uint32_t qx, qy, qz;
            cube_cell(q[3 * o], q[3 * o + 1], q[3 * o + 2], bbox, qx, qy, qz);
            cmin = cmax = morton30(qx, qy, qz);
        }
        cmin = __reduce_min_sync(0xffffffffu, cmin);
        cmax = __reduce_max_sync(0xffffffffu, cmax);
        const int64_t ilo = warp_lower_bound_u32(pcode, n, cmin, lane);
        const int64_t ihi = warp_lower_bound_u32(pcode, n, cmax + 1u, lane);
        if (lane != 0) continue;
        const int64_t imid = min((ilo + ihi) / 2, n - 1);
        unsigned cut = (unsigned)leaf_of[imid];
        if (cut == 0u || cut >= nn) cut = nn;  // one item holds the whole walk
        items[2 * p] = make_uint4((unsigned)p, 0u, cut, 0u);
        items[2 * p + 1] = make_uint4((unsigned)p, cut, nn, 1u);
        const uint32_t bk = cost_bucket((uint32_t)min(ihi - ilo, (int64_t)0x7fffffff));
        ibucket[2 * p] = bk;
        ibucket[2 * p + 1] = bk;
        atomicAdd(&sh[bk], 2u);
        if (plan) plan[p * kPlanWords + 4] = cut < nn ? cut : 0u;
        if (p == 0) *n_items = (unsigned)(2 * np);
    }
    order_counts_flush(sh, ostate);
}

void order_place(const uint32_t* ibucket, int64_t ni, uint32_t* ostate, uint32_t* porder,
                 cudaStream_t s) {
    const int64_t blocks = (ni + 255) / 256, cap = (int64_t)num_sms() * 8;
    note_launch();
    k_order_place<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(ibucket, ni, ostate, porder);
}

// Packets below this count are too few for the queue's tail to matter.
constexpr int64_t kOrderMinPackets = 2048;

// The treelet: nodes of depth < kTLDepth in preorder (one thread walks them),
// their records with packed keys, and the moment rows' first 12 floats.
__global__ void k_tl_build(unsigned nn, const NodeRec* __restrict__ nodes, const float* __restrict__ S,
                           int SR, TLRec* __restrict__ tl, uint32_t* __restrict__ tl_node) {
    __shared__ uint32_t ids[kTLMax];
    __shared__ int dep[kTLMax];
    __shared__ int cnt;
    if (threadIdx.x == 0) {
        int c = 0;
        uint32_t st_node[kTLDepth], st_next[kTLDepth];
        int sp = 0;
        ids[c] = 0; dep[c] = 0; ++c;
        if (__ldg(&nodes[0].meta).z == 0 && kTLDepth > 1 && nn > 1) { st_node[0] = 0; st_next[0] = 1; sp = 1; }
        bool bad = false;
        while (sp > 0 && !bad) {
            const uint32_t top = st_node[sp - 1], ch = st_next[sp - 1];
            const uint32_t end = (uint32_t)__ldg(&nodes[top].meta).x;
            if (ch >= end || ch >= nn) { --sp; continue; }
            const int4 m = __ldg(&nodes[ch].meta);
            if ((uint32_t)m.x <= ch || c >= kTLMax) { bad = true; break; }
            st_next[sp - 1] = (uint32_t)m.x;
            ids[c] = ch; dep[c] = sp; ++c;
            if (m.z == 0 && sp + 1 < kTLDepth) { st_node[sp] = ch; st_next[sp] = ch + 1; ++sp; }
        }
        cnt = bad ? 0 : c;
    }
    __syncthreads();
    const int n_tl = cnt;
    for (int i = threadIdx.x; i < kTLMax; i += blockDim.x) tl_node[i] = i < n_tl ? ids[i] : 0xffffffffu;
    for (int i = threadIdx.x; i < kTLMax; i += blockDim.x) {
        TLRec r;
        r.geo = make_float4(0.f, 0.f, 0.f, 0.f);
        r.meta = make_int4(0, 0, 0, 0);
        r.ext = make_uint4(0u, 0u, 0u, 0u);
        for (int j = 0; j < 3; ++j) r.mom[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < n_tl) {
            const uint32_t v = ids[i];
            r.geo = __ldg(&nodes[v].geo);
            r.meta = __ldg(&nodes[v].meta);
            const uint32_t sk = (uint32_t)r.meta.x;
            r.meta.x = (int)((sk << kTLSlotBits) | tl_slot_of(ids, n_tl, sk));
            r.ext.x = ((v + 1u) << kTLSlotBits) | (r.meta.z == 0 && dep[i] + 1 < kTLDepth ? tl_slot_of(ids, n_tl, v + 1u) : kTLInv);
            float m[12];
            for (int j = 0; j < 12; ++j) m[j] = j < SR ? S[(size_t)v * SR + j] : 0.f;
            for (int j = 0; j < 3; ++j) r.mom[j] = make_float4(m[4 * j], m[4 * j + 1], m[4 * j + 2], m[4 * j + 3]);
        }
        tl[i] = r;
    }
}

// Node records for the treelet walk: meta.x = the packed key of the skip.
__global__ void k_tl_keys(unsigned nn, const NodeRec* __restrict__ nodes, const uint32_t* __restrict__ tl_node,
                          NodeRec* __restrict__ out) {
    __shared__ uint32_t ids[kTLMax];
    for (int i = threadIdx.x; i < kTLMax; i += blockDim.x) ids[i] = tl_node[i];
    __syncthreads();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (int64_t)gridDim.x * blockDim.x) {
        NodeRec r = nodes[t];
        const uint32_t sk = (uint32_t)r.meta.x;
        r.meta.x = (int)((sk << kTLSlotBits) | tl_slot_of(ids, kTLMax, sk));
        out[t] = r;
    }
}

template <int CP, typename AT, int MODE, int KERN, bool RANGED, bool M16, bool TL = false>
void launch_query_m(const QueryArgs& a, cudaStream_t s) {
    static int per_sm = 0;
    const unsigned grid = query_grid(k_query<CP, AT, MODE, KERN, RANGED, M16, TL>, a.nq, per_sm);
    note_launch(); k_query<CP, AT, MODE, KERN, RANGED, M16, TL><<<grid, kQThreads, 0, s>>>(a);
}

// bf16 node moments (a.S16) only in the forward with bf16 attributes
template <int CP, typename AT, int MODE, int KERN, bool RANGED>
void launch_query_k(const QueryArgs& a, cudaStream_t s) {
    if constexpr (MODE == kForward && std::is_same<AT, __nv_bfloat16>::value) {
        if (a.S16) {
            launch_query_m<CP, AT, MODE, KERN, RANGED, true>(a, s);
            return;
        }
    }
    if constexpr (MODE == kForward && CP <= 4) {
        if (a.tl) {
            launch_query_m<CP, AT, MODE, KERN, RANGED, false, true>(a, s);
            return;
        }
    }
    launch_query_m<CP, AT, MODE, KERN, RANGED, false>(a, s);
}

// The kernel choice, ranged items and the moment type are template
// parameters: runtime branches cost the plain kernels registers.
template <int CP, typename AT, int MODE>
void launch_query(const QueryArgs& a, cudaStream_t s) {
    // kernel 2: the regularized kernel with channels that skip the foreshortening term
    const int kern = (MODE != kCount && a.G < a.C) ? 2 : a.kernel;
    if constexpr (MODE == kAdjoint || MODE == kForward) {
        if (a.items) {
            if (kern == 0) launch_query_k<CP, AT, MODE, 0, true>(a, s);
            else if (kern == 1) launch_query_k<CP, AT, MODE, 1, true>(a, s);
            else launch_query_k<CP, AT, MODE, 2, true>(a, s);
            return;
        }
    }
    if (MODE == kCount || kern == 0) launch_query_k<CP, AT, MODE, 0, false>(a, s);
    else if (kern == 1) launch_query_k<CP, AT, MODE, 1, false>(a, s);
    else if constexpr (MODE != kCount) launch_query_k<CP, AT, MODE, 2, false>(a, s);
}

template <int MODE>
int dispatch(const dipole_tree* t, const QueryArgs& a, cudaStream_t s) {
    if constexpr (MODE == kCount) {
        launch_query<1, float, kCount>(a, s);
        return 0;
    } else {
#define DIP_Q_CASE(K)                                                                    \
    case K:                                                                              \
        if constexpr (MODE == kAdjoint) launch_query<K, float, MODE>(a, s);              \
        else if (t->dtype == 0) launch_query<K, float, MODE>(a, s);                      \
        else launch_query<K, __nv_bfloat16, MODE>(a, s);                                 \
        break;
    switch (t->Cp) {
        DIP_Q_CASE(1)
        DIP_Q_CASE(2)
        DIP_Q_CASE(4)
        DIP_Q_CASE(8)
        DIP_Q_CASE(16)
        DIP_Q_CASE(32)
        DIP_Q_CASE(36)
        DIP_Q_CASE(64)
        default:
            return dip_fail(-1, "unsupported channel count");
    }
#undef DIP_Q_CASE
    return 0;
    }
}

// ---------------------------------------------------------------- no-alloc forward
// Scratch of dipole_forward_noalloc: the query sort (codes, indices, their
// ping-pong copies, the radix histograms with their scan space) and the work
// counter, for at most kNoAllocMaxQueries queries.  A file-scope device array:
// every GPU that loads this library holds it (about 4.5 MB) until the process
// exits; nothing is allocated per call.
constexpr int64_t kNoAllocMaxQueries = int64_t(1) << 18;
constexpr int64_t kNoAllocHistEntries = (kNoAllocMaxQueries / 1024) * 256 + 4096;
constexpr size_t kNoAllocBytes =
    4 * sizeof(uint32_t) * (size_t)kNoAllocMaxQueries + sizeof(uint32_t) * (size_t)kNoAllocHistEntries + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mutex;

// Device address of g_noalloc_scratch on the current device, looked up once per
// device (host code must not use the symbol itself: it names a host stand-in).
int noalloc_scratch(void** out) {
    int dev = 0;
    DIP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return dip_fail(-1, "dipole_forward_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        DIP_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return 0;
}

// ------------------------------------------------------------ traversal timer
constexpr int kTimerModes = 8;
struct TimerState {
    std::mutex m;
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[kTimerModes];
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spare;
};
TimerState g_timer;

// Event pair for one launch of `mode`, or {nullptr, nullptr} when the timer is off.
std::pair<cudaEvent_t, cudaEvent_t> timer_pair(int mode) {
    std::lock_guard<std::mutex> lock(g_timer.m);
    if (!g_timer.on || mode < 0 || mode >= kTimerModes) return {nullptr, nullptr};
    std::pair<cudaEvent_t, cudaEvent_t> p{nullptr, nullptr};
    if (!g_timer.spare.empty()) {
        p = g_timer.spare.back();
        g_timer.spare.pop_back();
    } else if (cudaEventCreate(&p.first) != cudaSuccess || cudaEventCreate(&p.second) != cudaSuccess) {
        return {nullptr, nullptr};
    }
    g_timer.pending[mode].push_back(p);
    return p;
}

}  // namespace

void timer_enable(bool on) {
    std::lock_guard<std::mutex> lock(g_timer.m);
    g_timer.on = on;
}

int timer_elapsed(int mode, float* total_ms, int64_t* launches) {
    if (mode < 0 || mode >= kTimerModes) return dip_fail(-1, "dipole_traversal_elapsed: bad mode");
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ps;
    {
        std::lock_guard<std::mutex> lock(g_timer.m);
        ps.swap(g_timer.pending[mode]);
    }
    float sum = 0.f;
    cudaError_t err = cudaSuccess;
    for (auto& p : ps) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(p.second);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.first, p.second);
        if (e != cudaSuccess && err == cudaSuccess) err = e;
        sum += ms;
    }
    {
        std::lock_guard<std::mutex> lock(g_timer.m);
        g_timer.spare.insert(g_timer.spare.end(), ps.begin(), ps.end());
    }
    DIP_CUDA_TRY(err);
    *total_ms = sum;
    *launches = (int64_t)ps.size();
    return 0;
}

int64_t noalloc_max_queries() { return kNoAllocMaxQueries; }

int query_noalloc(const dipole_tree* t, const float* queries, int64_t q, float beta, float* out,
                  cudaStream_t s) {
    if (q > kNoAllocMaxQueries || radix_hist_entries(q) > kNoAllocHistEntries)
        return dip_fail(-1, "dipole_forward_noalloc: q exceeds the static scratch limit of "
                            "262144 queries; split the queries or use dipole_forward");
    void* base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc) return rc;
    uint32_t* codes = static_cast<uint32_t*>(base);
    uint32_t* idx = codes + kNoAllocMaxQueries;
    uint32_t* ktmp = idx + kNoAllocMaxQueries;
    uint32_t* vtmp = ktmp + kNoAllocMaxQueries;
    uint32_t* hist = vtmp + kNoAllocMaxQueries;
    unsigned long long* work = reinterpret_cast<unsigned long long*>(hist + kNoAllocHistEntries);
    // the previous call's contents stay in the array: only the counter must start at 0
    DIP_CUDA_TRY(cudaMemsetAsync(work, 0, sizeof(unsigned long long), s));
    query_codes(queries, q, t->bbox, 30 - kQueryKeyBits, codes, idx, t->status, s, true);
    radix_sort_pairs(codes, idx, ktmp, vtmp, hist, q, kQueryKeyBits, s);
    QueryArgs a;
    a.nodes = t->nodes;
    a.pts = t->pts;
    a.nn = (unsigned)t->nn;
    a.status = t->status;
    a.q = queries;
    a.nq = q;
    a.qperm = idx;
    a.beta = beta;
    a.kernel = t->kernel;
    a.C = t->C;
    a.G = t->G;
    a.Cp = t->Cp;
    a.mu = t->mu;
    a.S = t->S;
    a.S16 = t->S16;
    a.out = out;
    a.gout = nullptr;
    a.g = nullptr;
    a.gg = nullptr;
    a.dS = nullptr;
    a.dmu = nullptr;
    a.dE = nullptr;
    a.dgeo = nullptr;
    a.gq = nullptr;
    a.accumulate = 0;
    a.counts = nullptr;
    a.ucounts = nullptr;
    a.work = work;
    a.npts = t->n;
    a.n_slots = 0;
    a.tl = nullptr;
    a.tl_node = nullptr;
    a.nodes_k = nullptr;
    a.porder = nullptr;  // packets in sorted order
    a.plan = nullptr;
    a.items = nullptr;
    a.n_items = nullptr;
    a.parent = t->parent;
    a.grid = GridSpec{};
    rc = dispatch<kForward>(t, a, s);
    if (rc) return rc;
    DIP_CUDA_TRY(cudaGetLastError());
    return 0;
}

int query(const dipole_tree* t, const QueryCall& call, cudaStream_t s) {
    const int mode = call.mode;
    const int64_t q = call.q;
    uint32_t* plan_perm = call.plan_perm;
    uint32_t* plan_cost = call.plan_cost;
    const bool plan_in = call.plan_in;
    const bool adjoint = mode == kAdjoint || mode == kAdjointGrad || mode == kAdjointGeom;
    const int SR = srow(t->Cp > 0 ? t->Cp : 1);
    const int64_t np = (q + 31) / 32;
    uint32_t *codes = nullptr, *idx = nullptr, *ktmp = nullptr, *vtmp = nullptr, *hist = nullptr;
    uint32_t* own_idx = nullptr;
    uint4* items = nullptr;
    uint32_t *ibucket = nullptr, *iorder = nullptr;
    uint32_t* small = nullptr;  // work counter (two words), item order state, item count
    const bool grid = call.grid_dim[0] > 0;
    const bool sorted = q > 0 && !grid;
    const bool big = sorted && np >= kOrderMinPackets;
    const bool adj_items = big && adjoint && plan_in && plan_cost;
    const bool fwd_items = big && mode != kCount && !plan_in;
    const int64_t ni = adj_items ? np * kPlanWords : fwd_items ? 2 * np : 0;
    // treelet: the value forward with up to 4 float moments, nodes below 2^25 (packed keys)
    const bool use_tl = t->treelet && mode == kForward && t->Cp <= 4 && !t->S16 &&
                        t->nn < (int64_t(1) << 25);
    // one allocation for the call's scratch (each API call costs the host microseconds)
    auto take = [&](Carve& c) {
        c.take(&small, 2 + kOrderStateWords + 1);
        if (sorted) {
            c.take(&codes, q);
            c.take(&ktmp, q);
            c.take(&vtmp, q);
            c.take(&hist, radix_hist_entries(q));
            if (!plan_in && !plan_perm) c.take(&own_idx, q);
        }
        if (ni) {
            c.take(&items, ni);
            c.take(&ibucket, ni);
            c.take(&iorder, ni);
        }
    };
    Carve cs;
    take(cs);
    void* block = nullptr;
    DIP_CUDA_TRY(dev_alloc((void**)&block, cs.off, s));
    cs = Carve{static_cast<char*>(block), 0};
    take(cs);
    unsigned long long* work = reinterpret_cast<unsigned long long*>(small);
    uint32_t* ostate = small + 2;
    unsigned* n_items = ostate + kOrderStateWords;
    DIP_CUDA_TRY(cudaMemsetAsync(small, 0, sizeof(uint32_t) * (2 + kOrderStateWords + 1), s));
    if (sorted) {
        if (plan_in) {
            idx = plan_perm;  // the query order computed by the forward on these queries
        } else {
            // query order: Hilbert indices of the cells in the tree's cube, sorted with the
            // query indices (runs of the Hilbert curve are compact, so packets are too)
            idx = plan_perm ? plan_perm : own_idx;
            query_codes(call.queries, q, t->bbox, 30 - kQueryKeyBits, codes, idx, t->status, s, true);
            radix_sort_pairs(codes, idx, ktmp, vtmp, hist, q, kQueryKeyBits, s);
        }
    }
    // Scheduling.  Packets run in sorted order, each recording its warp steps
    // into the plan when one is given; a call that reads a plan runs the
    // packets longest first from those records.  The record only changes the
    // order of the packets, never a result.
    const uint32_t* porder = nullptr;
    uint32_t* plan_w = nullptr;  // the plan this forward records
    if (adj_items) {
        // ranged items from the walk cuts recorded by the forward, longest first
        note_launch();
        k_plan_items<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(plan_cost, np, (unsigned)t->nn,
                                                                  items, ibucket, n_items, ostate);
        order_place(ibucket, ni, ostate, iorder, s);
        porder = iorder;
    }
    if (big && !plan_in && plan_cost && (mode == kForward || mode == kForwardGrad)) {
        plan_w = plan_cost;  // items add their steps and record their cuts
        DIP_CUDA_TRY(cudaMemsetAsync(plan_w, 0, sizeof(uint32_t) * kPlanWords * (size_t)np, s));
    }
    if (fwd_items) {
        // every packet's walk in two ranged items (the forward's add into the
        // zeroed outputs), longest predicted first
        if (call.out) DIP_CUDA_TRY(cudaMemsetAsync(call.out, 0, sizeof(float) * (size_t)q * t->C, s));
        if (call.gout)
            DIP_CUDA_TRY(cudaMemsetAsync(call.gout, 0, sizeof(float) * 3 * (size_t)q * t->C, s));
        if (call.gq && !call.accumulate)
            DIP_CUDA_TRY(cudaMemsetAsync(call.gq, 0, sizeof(float) * 3 * (size_t)q, s));
        note_launch();
        k_fwd_items<<<(unsigned)((np + 7) / 8), 256, 0, s>>>(
            call.queries, idx, q, np, t->bbox, t->code, t->n, t->leaf_of, (unsigned)t->nn, items,
            n_items, plan_w, ibucket, ostate);
        order_place(ibucket, ni, ostate, iorder, s);
        porder = iorder;
    }
    // stage-1 sums: the tree's scratch, or the caller's accumulator
    float* dS = call.acc ? call.acc : t->dS;
    float* dmu = call.acc ? call.acc + (size_t)t->nn * SR : t->dmu;
    if (adjoint && !(call.acc && call.accumulate)) {
        DIP_CUDA_TRY(cudaMemsetAsync(dS, 0, sizeof(float) * (size_t)t->nn * SR, s));
        DIP_CUDA_TRY(cudaMemsetAsync(dmu, 0, sizeof(float) * (size_t)t->n * t->Cp, s));
    }
    if (mode == kAdjointGeom) {
        DIP_CUDA_TRY(cudaMemsetAsync(t->dE, 0, sizeof(float) * (size_t)t->nn, s));
        DIP_CUDA_TRY(cudaMemsetAsync(t->dgeo, 0, sizeof(float) * 4 * (size_t)t->n, s));
    }
    int rc = 0;
    if (q > 0) {
        QueryArgs a;
        a.nodes = t->nodes;
        a.pts = t->pts;
        a.nn = (unsigned)t->nn;
        a.status = t->status;
        a.q = call.queries;
        a.nq = q;
        a.qperm = idx;
        a.beta = call.beta;
        a.kernel = t->kernel;
        a.C = t->C;
        a.G = t->G;
        a.Cp = t->Cp;
        a.mu = t->mu;
        a.S = t->S;
        a.S16 = t->S16;
        a.out = call.out;
        a.gout = call.gout;
        a.g = call.g;
        a.gg = call.gg;
        a.dS = dS;
        a.dmu = dmu;
        a.dE = t->dE;
        a.dgeo = t->dgeo;
        a.gq = call.gq;
        a.accumulate = call.accumulate;
        a.counts = call.counts;
        a.ucounts = call.ucounts;
        a.work = work;
        a.npts = t->n;
        a.n_slots = ni;
        a.tl = nullptr;
        a.tl_node = nullptr;
        a.nodes_k = nullptr;
        if (use_tl) {
            // the block and the keyed node copy are made once per tree (geometry
            // only); the records, which carry the moments, at every call
            auto take_tl = [&](Carve& c, TLRec** r, uint32_t** ids, NodeRec** nk) {
                c.take(r, kTLMax);
                c.take(ids, kTLMax);
                c.take(nk, t->nn);
            };
            TLRec* tl_rec = nullptr;
            uint32_t* tl_ids = nullptr;
            NodeRec* nodes_k = nullptr;
            const bool fresh = t->tl_block == nullptr;
            if (fresh) {
                Carve ct;
                take_tl(ct, &tl_rec, &tl_ids, &nodes_k);
                void* blk = nullptr;
                DIP_CUDA_TRY(dev_alloc(&blk, ct.off, s));
                t->tl_block = blk;  // cached state of the tree (mutable)
            }
            Carve ct{static_cast<char*>(t->tl_block), 0};
            take_tl(ct, &tl_rec, &tl_ids, &nodes_k);
            note_launch();
            k_tl_build<<<1, 128, 0, s>>>((unsigned)t->nn, t->nodes, t->S, srow(t->Cp), tl_rec, tl_ids);
            if (fresh) {
                const int64_t kb = (t->nn + 255) / 256, kcap = (int64_t)num_sms() * 8;
                note_launch();
                k_tl_keys<<<(unsigned)(kb < kcap ? kb : kcap), 256, 0, s>>>((unsigned)t->nn, t->nodes,
                                                                            tl_ids, nodes_k);
            }
            a.tl = tl_rec;
            a.tl_node = tl_ids;
            a.nodes_k = nodes_k;
        }
        a.porder = porder;
        a.plan = plan_w;
        a.items = items;
        a.n_items = n_items;
        a.parent = t->parent;
        a.grid = GridSpec{};
        if (grid) {
            for (int d = 0; d < 3; ++d) {
                a.grid.lo[d] = call.grid_lo[d];
                a.grid.dim[d] = call.grid_dim[d];
            }
            a.grid.h = call.grid_h;
            a.grid.nb[0] = (call.grid_dim[0] + 3) / 4;
            a.grid.nb[1] = (call.grid_dim[1] + 3) / 4;
            a.grid.nb[2] = (call.grid_dim[2] + 1) / 2;
            a.nq = 32 * a.grid.nb[0] * a.grid.nb[1] * a.grid.nb[2];  // one packet per brick
        }
        const auto ev = timer_pair(mode);
        if (ev.first) DIP_CUDA_TRY(cudaEventRecord(ev.first, s));
        if (mode == kForward) rc = dispatch<kForward>(t, a, s);
        else if (mode == kAdjoint) rc = dispatch<kAdjoint>(t, a, s);
        else if (mode == kCount) rc = dispatch<kCount>(t, a, s);
        else rc = dispatch_grad(t, mode, a, s);
        if (ev.second) DIP_CUDA_TRY(cudaEventRecord(ev.second, s));
    }
    if (rc == 0 && adjoint && call.grad && !call.acc)
        rc = stage2(t, t->dS, t->dmu, call.grad, call.accumulate, s);
    if (rc == 0 && mode == kAdjointGeom)
        rc = stage2_geom(t, call.grad_n, call.grad_eps, call.accumulate, s);
    cudaFreeAsync(block, s);
    if (rc) return rc;
    DIP_CUDA_TRY(cudaGetLastError());
    return 0;
}

}  // namespace dip
