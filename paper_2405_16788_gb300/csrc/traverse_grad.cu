// Spatial gradient of the Barnes-Hut dipole sum and its adjoint.
//
// The paper differentiates the sum only with respect to the point attributes
// (Sec. 6.2); the gradient with respect to the query position follows from
// the same kernel (Sec. 4.1, eq. regularized_poisson).  With u = p - x,
// r = |u|, a(r) = rho(r/eps)/r^3 and b(r) = a'(r)/r, the term
// A mu a(r) n.u/(4 pi) of eq. dipole_sum has the x-gradient
//   -A mu/(4 pi) [a n + b (n.u) u],
// and the far-field term rho(d/eps~) S.(p~ - x)/(4 pi d^3) of eq. farfield,
// with v = p~ - x, has the x-gradient -[a S + b (S.v) v]/(4 pi).
// The walk, the far test and the warp cooperation are those of traverse.cu
// (Alg. 1): a lane takes exactly the decisions of its own depth-first walk.
//
// A query needs four running sums per channel (D and its three derivatives),
// so the kernel handles CG <= 4 channels per walk and walks the tree once per
// group of CG channels.  The adjoint of both outputs (dL/dD = g and
// dL/d grad D = G) gives, for a far node,
//   dS^c += [a g^c v - a G^c - b (v.G^c) v]/(4 pi),
// and for a point of an opened leaf, with w = A n,
//   dmu^c += [a (w.u) g^c - a (w.G^c) - b (w.u)(u.G^c)]/(4 pi);
// stage 2 (eq. farfield_features_gradient) is unchanged.
//
// kAdjointGeom extends that adjoint to the normals and radii: a far node also
// sums dE_t = d L/d eps~_t over the warp (one atomic), and an opened leaf's
// point also gets its normal and radius terms (four values, one warp
// reduce-scatter); k_stage2_geom (refit.cu) sends both to the points.
#include "query.cuh"

namespace dip {
namespace {

// Series of (t rho'(t) - 3 rho(t))/t^5 in u = t^2, from the series of rho:
// coefficient k-1 = (-1)^k (4/sqrt(pi)) 2k/(k! (2k+3)), k >= 1.  Seven terms
// leave a relative error below 1e-8 at t = 0.5.
constexpr float kGSer0 = -0.9027033336764101f;
constexpr float kGSer1 = 0.6447880954831501f;
constexpr float kGSer2 = -0.250750926021225f;
constexpr float kGSer3 = 0.06838661618760682f;
constexpr float kGSer4 = -0.014466399578147597f;
constexpr float kGSer5 = 0.0025075092602122504f;
constexpr float kGSer6 = -0.00036875136179591913f;

// a = rho(d/eps)/d^3 and b = a'(d)/d = (t rho'(t) - 3 rho(t))/d^5, t = d/eps,
// rho'(t) = (4/sqrt(pi)) t^2 exp(-t^2); d^2 = d2 > 0, inv_eps = 1/eps (+inf
// for eps = 0).  Same branches as rho_over_d3.
__device__ __forceinline__ void grad_factors(float d2, float inv_eps, float& a, float& b) {
    const float inv_d = rsqrtf(d2);
    const float inv_d2 = inv_d * inv_d;
    const float inv_d3 = inv_d2 * inv_d;
    const float t = d2 * inv_d * inv_eps;
    if (t >= kTCut) {
        a = inv_d3;
        b = -3.0f * inv_d3 * inv_d2;
        return;
    }
    const float u = t * t;
    if (t < kTSeries) {
        float p = kSer6;
        p = fmaf(p, u, kSer5);
        p = fmaf(p, u, kSer4);
        p = fmaf(p, u, kSer3);
        p = fmaf(p, u, kSer2);
        p = fmaf(p, u, kSer1);
        p = fmaf(p, u, kSer0);
        float r = kGSer6;
        r = fmaf(r, u, kGSer5);
        r = fmaf(r, u, kGSer4);
        r = fmaf(r, u, kGSer3);
        r = fmaf(r, u, kGSer2);
        r = fmaf(r, u, kGSer1);
        r = fmaf(r, u, kGSer0);
        const float ie2 = inv_eps * inv_eps, ie3 = ie2 * inv_eps;
        a = p * ie3;
        b = r * (ie3 * ie2);
        return;
    }
    const float e = __expf(-u);
    const float rho = erff(t) - kTwoOverSqrtPi * t * e;
    const float trho1 = 2.0f * kTwoOverSqrtPi * u * t * e;  // t rho'(t)
    a = rho * inv_d3;
    b = (trho1 - 3.0f * rho) * (inv_d3 * inv_d2);
}

// grad_factors plus the eps-derivatives a_e = da/deps =
// -(4/sqrt(pi)) t^3 exp(-t^2)/(eps d^3) and b_e = db/deps =
// (8/sqrt(pi)) t^5 exp(-t^2)/(eps d^5), sharing the reciprocal square root and
// the exponential.  a_e, b_e have no cut at kTCut: far from every point these
// tiny values are the whole eps-gradient; they are 0 for eps = 0 (t = inf) and
// from t = 10, where exp(-t^2) leaves the float range.
__device__ __forceinline__ void geom_factors(float d2, float inv_eps, float& a, float& b, float& ae,
                                             float& be) {
    const float inv_d = rsqrtf(d2);
    const float inv_d2 = inv_d * inv_d;
    const float inv_d3 = inv_d2 * inv_d;
    const float t = d2 * inv_d * inv_eps;
    const float u = t * t;
    const float e = t < 10.0f ? __expf(-u) : 0.0f;
    if (t >= kTCut) {
        a = inv_d3;
        b = -3.0f * inv_d3 * inv_d2;
    } else if (t < kTSeries) {
        float p = kSer6;
        p = fmaf(p, u, kSer5);
        p = fmaf(p, u, kSer4);
        p = fmaf(p, u, kSer3);
        p = fmaf(p, u, kSer2);
        p = fmaf(p, u, kSer1);
        p = fmaf(p, u, kSer0);
        float r = kGSer6;
        r = fmaf(r, u, kGSer5);
        r = fmaf(r, u, kGSer4);
        r = fmaf(r, u, kGSer3);
        r = fmaf(r, u, kGSer2);
        r = fmaf(r, u, kGSer1);
        r = fmaf(r, u, kGSer0);
        const float ie2 = inv_eps * inv_eps, ie3 = ie2 * inv_eps;
        a = p * ie3;
        b = r * (ie3 * ie2);
    } else {
        const float rho = erff(t) - kTwoOverSqrtPi * t * e;
        const float trho1 = 2.0f * kTwoOverSqrtPi * u * t * e;
        a = rho * inv_d3;
        b = (trho1 - 3.0f * rho) * (inv_d3 * inv_d2);
    }
    if (t < 10.0f) {
        const float g = 2.0f * kTwoOverSqrtPi * e * t * u * inv_eps;
        ae = -g * inv_d3;
        be = 2.0f * g * u * (inv_d3 * inv_d2);
    } else {
        ae = 0.0f;
        be = 0.0f;
    }
}

// The desingularized kernel's factors (1/max(d, delta)^3, delta = 1/inv_eps):
// outside the cutoff a = 1/d^3, b = -3/d^5 and no delta-dependence; inside,
// a = 1/delta^3, b = 0, a_e = da/ddelta = -3/delta^4, b_e = 0.
__device__ __forceinline__ void desing_factors(float d2, float inv_eps, float& a, float& b, float& ae,
                                               float& be) {
    const float inv_d = rsqrtf(d2);
    const float t = d2 * inv_d * inv_eps;
    be = 0.0f;
    if (t >= 1.0f) {
        const float inv_d3 = inv_d * inv_d * inv_d;
        a = inv_d3;
        b = -3.0f * inv_d3 * inv_d * inv_d;
        ae = 0.0f;
    } else {
        const float ie3 = inv_eps * inv_eps * inv_eps;
        a = ie3;
        b = 0.0f;
        ae = -3.0f * ie3 * inv_eps;
    }
}

// Three resident blocks for the forward and the normal/radius adjoint (80
// registers, a few spilled bytes: -10% and -9% against two blocks at 100 and
// 109 registers); two for the gradient adjoint (72 registers fit three anyway).
// RANGED: work items are preorder ranges of a packet's walk, as in the value
// traversal (two per packet in the forward, the plan's cuts in the adjoints);
// the same range holds for every channel group, whose walks are identical.
template <int CG, typename AT, int MODE, bool RANGED>
__global__ void __launch_bounds__(kQThreads, (MODE == kForwardGrad || MODE == kForwardGradDot ||
                                               MODE == kAdjointGrad) ? 4
                                              : (MODE == kAdjointGeom) ? 3 : 2)
    k_query_grad(const QueryArgs a) {
    static_assert(CG == 1 || CG == 2 || CG == 4, "channel group");
    constexpr bool FWD = MODE == kForwardGrad || MODE == kForwardGradDot;
    constexpr bool DOT = MODE == kForwardGradDot;  // only sum_c g^c grad D^c
    constexpr bool GEOM = MODE == kAdjointGeom;  // also the normal and radius gradients
    constexpr unsigned FULL = 0xffffffffu;
    constexpr unsigned kFoldSteps = 32;
    constexpr int NV = FWD ? 4 * CG : 1;  // D and grad D per channel: [4c] D, [4c+1+k] d/dx_k
    const int lane = threadIdx.x & 31;
    const NodeRec* __restrict__ nodes = a.nodes;
    const PointRec* __restrict__ pts = a.pts;
    const unsigned nn = a.nn;
    const int Cp = a.Cp;
    const int SR = srow(Cp);

    for (;;) {
        unsigned long long pk = 0;
        if (lane == 0) pk = atomicAdd(a.work, 1ull);
        pk = __shfl_sync(FULL, pk, 0);
        int64_t pm;
        unsigned lo = 0u, hi = nn, half = 0u;
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
            pm = (int64_t)(a.porder ? a.porder[pk] : pk);
            if (!in_bounds(pm * 32 < a.nq, a.status)) continue;
        }
        const int64_t qi = pm * 32 + lane;
        bool valid = qi < a.nq;
        int64_t qo = valid ? (a.qperm ? (int64_t)a.qperm[qi] : qi) : 0;
        if (valid && !in_bounds(qo >= 0 && qo < a.nq, a.status)) {
            valid = false;
            qo = 0;
        }
        float x0 = 0.f, x1 = 0.f, x2 = 0.f;
        if (valid) { x0 = a.q[3 * qo]; x1 = a.q[3 * qo + 1]; x2 = a.q[3 * qo + 2]; }
        int ord[CG];
        lane_channel_order<CG>(lane, ord);
        unsigned steps = 0;
        float gq[DOT ? 3 : 1];  // kForwardGradDot: sum_c g^c grad D^c
#pragma unroll
        for (int k = 0; k < (DOT ? 3 : 1); ++k) gq[k] = 0.f;

        for (int c0 = 0; c0 < Cp; c0 += CG) {
            // forward: blocked Kahan sums, plain partial sums (registers) folded
            // every kFoldSteps warp steps into compensated ones (shared memory,
            // one column per thread, touched only at a fold: 32 KB per block at
            // CG = 4, which leaves the registers to the walk and four blocks per SM)
            __shared__ float sh_acc[FWD ? NV : 1][kQThreads], sh_cmp[FWD ? NV : 1][kQThreads];
            float part[NV];
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                part[i] = 0.f;
                if (FWD) {
                    sh_acc[FWD ? i : 0][threadIdx.x] = 0.f;
                    sh_cmp[FWD ? i : 0][threadIdx.x] = 0.f;
                }
            }
            auto kahan_into = [&](int i, float v) {
                kahan_add(sh_acc[FWD ? i : 0][threadIdx.x], sh_cmp[FWD ? i : 0][threadIdx.x], v);
            };
            auto total = [&](int i) -> float {
                return __fsub_rn(sh_acc[FWD ? i : 0][threadIdx.x], sh_cmp[FWD ? i : 0][threadIdx.x]);
            };
            // adjoint: upstream values and gradients of this group, scaled by
            // 1/(4 pi), in lane_channel_order
            float gl[FWD ? 1 : CG], Gl[FWD ? 1 : 3 * CG];
            float gN[GEOM ? CG : 1], GN[GEOM ? 3 * CG : 1];  // natural channel order
            if (!FWD) {
                float gc[CG], Gc[3 * CG];
#pragma unroll
                for (int c = 0; c < CG; ++c) {
                    const bool on = valid && c0 + c < a.C;
                    const int64_t o = qo * a.C + c0 + c;
                    gc[c] = (on && a.g) ? a.g[o] * kInv4Pi : 0.f;
#pragma unroll
                    for (int k = 0; k < 3; ++k) Gc[3 * c + k] = (on && a.gg) ? a.gg[3 * o + k] * kInv4Pi : 0.f;
                }
#pragma unroll
                for (int i = 0; i < CG; ++i) {
                    float v = gc[0], v0 = Gc[0], v1 = Gc[1], v2 = Gc[2];
#pragma unroll
                    for (int c = 1; c < CG; ++c) {
                        const bool m = ord[i] == c;
                        v = m ? gc[c] : v;
                        v0 = m ? Gc[3 * c] : v0;
                        v1 = m ? Gc[3 * c + 1] : v1;
                        v2 = m ? Gc[3 * c + 2] : v2;
                    }
                    gl[FWD ? 0 : i] = v;
                    Gl[FWD ? 0 : 3 * i] = v0;
                    Gl[FWD ? 0 : 3 * i + 1] = v1;
                    Gl[FWD ? 0 : 3 * i + 2] = v2;
                }
                if (GEOM) {
#pragma unroll
                    for (int c = 0; c < CG; ++c) {
                        gN[GEOM ? c : 0] = gc[c];
#pragma unroll
                        for (int k = 0; k < 3; ++k) GN[GEOM ? 3 * c + k : 0] = Gc[3 * c + k];
                    }
                }
            }

            unsigned next = valid ? lo : nn;
            if (RANGED && lo > 0u && lo < nn) {
                // the walk reaches lo unless an ancestor of lo is far; it then resumes
                // at the topmost far ancestor's skip, the largest of them
                const unsigned start = next;
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
                    if (start == lo && d2 > __fmul_rn(R, R)) next = max(next, (unsigned)meta.x);
                    u = a.parent[u];
                }
            }
            unsigned gsteps = 0;
            // one warp step of the walk; false once the walk is over
            auto walk_step = [&](const bool fold_here) -> bool {
                const unsigned n = __reduce_min_sync(FULL, next);
                if (FWD) {
                    if (n >= hi) return false;
                } else if ((n >= hi) | (gsteps >= nn)) {  // a well-formed tree needs at most nn steps
                    if (n < hi && lane == 0) atomicOr(a.status, kStatusTraversal);
                    return false;
                }
                ++gsteps;
                const float4 geo = __ldg(&nodes[n].geo);
                const int4 meta = __ldg(&nodes[n].meta);
                const bool act = next == n;
                float4 s_first[(FWD || GEOM) ? (3 * CG + 3) / 4 : 1];
                if (FWD || GEOM) {
                    const float4* sp = reinterpret_cast<const float4*>(a.S + (size_t)n * SR + 3 * c0);
#pragma unroll
                    for (int j = 0; j < (3 * CG + 3) / 4; ++j) s_first[j] = __ldg(sp + j);
                }
                // far test of Alg. 1 in the fixed float order of traverse.cu
                const float dx = __fsub_rn(x0, geo.x);
                const float dy = __fsub_rn(x1, geo.y);
                const float dz = __fsub_rn(x2, geo.z);
                const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                const float R = __fmul_rn(a.beta, geo.w);
                const bool far = act && (d2 > __fmul_rn(R, R));
                const bool leaf = meta.z > 0;
                const bool open_leaf = act && !far && leaf;
                if (act) next = (far || leaf) ? (unsigned)meta.x : n + 1u;

                if (__any_sync(FULL, far)) {
                    float fa = 0.f, fb = 0.f, fae = 0.f, fbe = 0.f;
                    if (far) {
                        if (a.kernel) desing_factors(d2, __int_as_float(meta.w), fa, fb, fae, fbe);
                        else if (GEOM) geom_factors(d2, __int_as_float(meta.w), fa, fb, fae, fbe);
                        else grad_factors(d2, __int_as_float(meta.w), fa, fb);
                    }
                    const float vx = -dx, vy = -dy, vz = -dz;  // v = p~ - x
                    if (FWD) {
                        float s[4 * ((3 * CG + 3) / 4)];
#pragma unroll
                        for (int j = 0; j < (3 * CG + 3) / 4; ++j) {
                            s[4 * j] = s_first[j].x; s[4 * j + 1] = s_first[j].y;
                            s[4 * j + 2] = s_first[j].z; s[4 * j + 3] = s_first[j].w;
                        }
                        // no per-lane predicate: a lane that did not take the node
                        // has fa = fb = 0 and adds exact zeros
#pragma unroll
                        for (int c = 0; c < CG; ++c) {
                            const float sx = s[3 * c], sy = s[3 * c + 1], sz = s[3 * c + 2];
                            const float sv = fmaf(sx, vx, fmaf(sy, vy, sz * vz));
                            const float bsv = fb * sv;
                            part[4 * c] = fmaf(fa, sv, part[4 * c]);
                            part[4 * c + 1] -= fmaf(fa, sx, bsv * vx);
                            part[4 * c + 2] -= fmaf(fa, sy, bsv * vy);
                            part[4 * c + 3] -= fmaf(fa, sz, bsv * vz);
                        }
                    } else {
                        float val[3 * CG];
#pragma unroll
                        for (int i = 0; i < CG; ++i) {
                            const float G0 = Gl[3 * i], G1 = Gl[3 * i + 1], G2 = Gl[3 * i + 2];
                            const float vG = fmaf(vx, G0, fmaf(vy, G1, vz * G2));
                            const float coef = fmaf(fa, gl[i], -fb * vG);
                            val[3 * i] = fmaf(coef, vx, -fa * G0);
                            val[3 * i + 1] = fmaf(coef, vy, -fa * G1);
                            val[3 * i + 2] = fmaf(coef, vz, -fa * G2);
                        }
                        adjoint_vec_reduce<CG>(val, a.dS + (size_t)n * SR + 3 * c0, ord[0], lane);
                        if (GEOM) {
                            // d eps~_t += sum_c [g^c a_e (S^c.v) - a_e (S^c.G^c) - b_e (S^c.v)(v.G^c)]
                            const float ae = fae, be = fbe;
                            float s[4 * ((3 * CG + 3) / 4)];
#pragma unroll
                            for (int j = 0; j < (3 * CG + 3) / 4; ++j) {
                                s[4 * j] = s_first[j].x; s[4 * j + 1] = s_first[j].y;
                                s[4 * j + 2] = s_first[j].z; s[4 * j + 3] = s_first[j].w;
                            }
                            float e = 0.f;
#pragma unroll
                            for (int c = 0; c < CG; ++c) {
                                const float G0 = GN[3 * c], G1 = GN[3 * c + 1], G2 = GN[3 * c + 2];
                                const float sx = s[3 * c], sy = s[3 * c + 1], sz = s[3 * c + 2];
                                const float sv = fmaf(sx, vx, fmaf(sy, vy, sz * vz));
                                const float sG = fmaf(sx, G0, fmaf(sy, G1, sz * G2));
                                const float vG = fmaf(vx, G0, fmaf(vy, G1, vz * G2));
                                e += fmaf(ae, fmaf(gN[c], sv, -sG), -be * sv * vG);
                            }
#pragma unroll
                            for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(FULL, e, off);
                            if (lane == 0 && e != 0.f) atomicAdd(a.dE + n, e);
                        }
                    }
                }

                if (__any_sync(FULL, open_leaf)) {
                    // opened leaf: exact terms of its points (eq. dipole_sum)
                    const int f = meta.y;
                    const int cnt =
                        in_bounds(f >= 0 && meta.z >= 0 && (int64_t)f + meta.z <= a.npts, a.status) ? meta.z : 0;
                    if (FWD) {
                        prefetch_l1(pts + f, cnt * (int)sizeof(PointRec), lane);
                        prefetch_l1(reinterpret_cast<const AT*>(a.mu) + (size_t)f * Cp + c0,
                                    cnt * Cp * (int)sizeof(AT), lane);
                    }
                    for (int j = 0; j < cnt; ++j) {
                        const PointRec pr = pts[f + j];
                        float fa = 0.f, fb = 0.f, wu = 0.f, pae = 0.f, pbe = 0.f;
                        const float ux = pr.geo.x - x0, uy = pr.geo.y - x1, uz = pr.geo.z - x2;
                        if (open_leaf) {
                            const float r2 = fmaf(uz, uz, fmaf(uy, uy, ux * ux));
                            if (r2 > 0.f) {
                                if (a.kernel) desing_factors(r2, pr.geo.w, fa, fb, pae, pbe);
                                else if (GEOM) geom_factors(r2, pr.geo.w, fa, fb, pae, pbe);
                                else grad_factors(r2, pr.geo.w, fa, fb);
                                wu = fmaf(pr.w.x, ux, fmaf(pr.w.y, uy, pr.w.z * uz));
                            }
                        }
                        const float bwu = fb * wu;
                        if (FWD) {
                            // per unit mu: value a (w.u), gradient -(a w + b (w.u) u)
                            const float kd = fa * wu;
                            const float g0 = -fmaf(fa, pr.w.x, bwu * ux);
                            const float g1 = -fmaf(fa, pr.w.y, bwu * uy);
                            const float g2 = -fmaf(fa, pr.w.z, bwu * uz);
                            float m[CG];
                            load_row<AT>(reinterpret_cast<const AT*>(a.mu) + (size_t)(f + j) * Cp + c0, m, CG);
#pragma unroll
                            for (int c = 0; c < CG; ++c) {  // kd = g = 0 off the leaf
                                part[4 * c] = fmaf(kd, m[c], part[4 * c]);
                                part[4 * c + 1] = fmaf(g0, m[c], part[4 * c + 1]);
                                part[4 * c + 2] = fmaf(g1, m[c], part[4 * c + 2]);
                                part[4 * c + 3] = fmaf(g2, m[c], part[4 * c + 3]);
                            }
                        } else {
                            float val[CG];
#pragma unroll
                            for (int i = 0; i < CG; ++i) {
                                const float G0 = Gl[3 * i], G1 = Gl[3 * i + 1], G2 = Gl[3 * i + 2];
                                const float wG = fmaf(pr.w.x, G0, fmaf(pr.w.y, G1, pr.w.z * G2));
                                const float uG = fmaf(ux, G0, fmaf(uy, G1, uz * G2));
                                val[i] = fmaf(fa, fmaf(wu, gl[i], -wG), -bwu * uG);
                            }
                            adjoint_scalar_reduce<CG>(val, a.dmu + (size_t)(f + j) * Cp + c0, ord[0], lane);
                            if (GEOM) {
                                // normal (A sum_c mu^c [g^c a u - a G^c - b (u.G^c) u]) and
                                // radius (sum_c mu^c [g^c a_e (w.u) - a_e (w.G^c) - b_e (w.u)(u.G^c)])
                                const float ae = pae, be = pbe;
                                float m[CG];
                                load_row<AT>(reinterpret_cast<const AT*>(a.mu) + (size_t)(f + j) * Cp + c0, m, CG);
                                float gv[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                                for (int c = 0; c < CG; ++c) {
                                    const float G0 = GN[3 * c], G1 = GN[3 * c + 1], G2 = GN[3 * c + 2];
                                    const float uG = fmaf(ux, G0, fmaf(uy, G1, uz * G2));
                                    const float wG = fmaf(pr.w.x, G0, fmaf(pr.w.y, G1, pr.w.z * G2));
                                    const float ga = fa * gN[c], bu = fb * uG;
                                    gv[0] = fmaf(m[c], fmaf(ga, ux, -fmaf(fa, G0, bu * ux)), gv[0]);
                                    gv[1] = fmaf(m[c], fmaf(ga, uy, -fmaf(fa, G1, bu * uy)), gv[1]);
                                    gv[2] = fmaf(m[c], fmaf(ga, uz, -fmaf(fa, G2, bu * uz)), gv[2]);
                                    gv[3] = fmaf(m[c], fmaf(ae, fmaf(gN[c], wu, -wG), -be * wu * uG), gv[3]);
                                }
                                gv[0] *= pr.w.w; gv[1] *= pr.w.w; gv[2] *= pr.w.w;
                                warp_reduce_add<4>(gv, a.dgeo + 4 * (size_t)(f + j), lane);
                            }
                        }
                    }
                }
                if (FWD && fold_here && (gsteps % kFoldSteps) == 0u) {
                    if (gsteps > nn) {  // checked every kFoldSteps steps
                        if (lane == 0) atomicOr(a.status, kStatusTraversal);
                        return false;
                    }
#pragma unroll
                    for (int i = 0; i < NV; ++i) {
                        kahan_into(i, part[i]);
                        part[i] = 0.f;
                    }
                    // plan record (first channel group): nodes of this part's steps 128, 256, 384
                    if (RANGED && a.plan && c0 == 0 && lane == 0 && (gsteps & (kCutSteps - 1u)) == 0u &&
                        gsteps <= kCutSteps * kPartCuts)
                        a.plan[(size_t)pm * kPlanWords + 1u + 4u * half + gsteps / kCutSteps - 1u] = n;
                }
                return true;
            };
            if (FWD) {
                // two steps per turn: the fold (every kFoldSteps steps, an even
                // count) is only tested after the second
                for (;;) {
                    if (!walk_step(false)) break;
                    if (!walk_step(true)) break;
                }
            } else {
                while (walk_step(true)) {
                }
            }
            steps += gsteps;
            if (FWD) {
#pragma unroll
                for (int i = 0; i < NV; ++i) kahan_into(i, part[i]);
                if (valid) {
#pragma unroll
                    for (int c = 0; c < CG; ++c) {
                        if (c0 + c >= a.C) continue;
                        const int64_t o = qo * a.C + c0 + c;
                        if constexpr (DOT) {
                            const float gc = a.g[o];
#pragma unroll
                            for (int k = 0; k < 3; ++k)
                                gq[k] = fmaf(gc, total(4 * c + 1 + k) * kInv4Pi, gq[k]);
                            continue;
                        }
                        // ranged: the two parts of a packet add into the zeroed outputs
                        const float d = total(4 * c) * kInv4Pi;
                        if (a.out) {
                            if (RANGED) atomicAdd(a.out + o, d);
                            else a.out[o] = d;
                        }
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float v = total(4 * c + 1 + k) * kInv4Pi;
                            if (RANGED) atomicAdd(a.gout + 3 * o + k, v);
                            else a.gout[3 * o + k] = v;
                        }
                    }
                }
            }
        }
        if (DOT && valid) {
            // dL/dx of the query; ranged: the two parts add into the output
#pragma unroll
            for (int k = 0; k < (DOT ? 3 : 0); ++k) {
                float* dst = a.gq + 3 * qo + k;
                if (RANGED) atomicAdd(dst, gq[k]);
                else *dst = a.accumulate ? *dst + gq[k] : gq[k];
            }
        }
        if (a.plan && lane == 0) atomicAdd(a.plan + (size_t)pm * kPlanWords, steps);
    }
}

template <int CG, typename AT, int MODE, bool RANGED>
void launch_grad_r(const QueryArgs& a, cudaStream_t s) {
    static int per_sm = 0;
    const unsigned grid = query_grid(k_query_grad<CG, AT, MODE, RANGED>, a.nq, per_sm);
    note_launch(); k_query_grad<CG, AT, MODE, RANGED><<<grid, kQThreads, 0, s>>>(a);
}

template <int CG, typename AT, int MODE>
void launch_grad(const QueryArgs& a, cudaStream_t s) {
    if (a.items) launch_grad_r<CG, AT, MODE, true>(a, s);
    else launch_grad_r<CG, AT, MODE, false>(a, s);
}

template <int CG, int MODE>
void launch_grad_dtype(const dipole_tree* t, const QueryArgs& a, cudaStream_t s) {
    if constexpr (MODE == kAdjointGrad) {
        launch_grad<CG, float, MODE>(a, s);  // reads no attributes
    } else {
        if (t->dtype == 0) launch_grad<CG, float, MODE>(a, s);
        else launch_grad<CG, __nv_bfloat16, MODE>(a, s);
    }
}

template <int MODE>
void launch_grad_cg(const dipole_tree* t, const QueryArgs& a, cudaStream_t s) {
    if (t->Cp == 1) launch_grad_dtype<1, MODE>(t, a, s);
    else if (t->Cp == 2) launch_grad_dtype<2, MODE>(t, a, s);
    else launch_grad_dtype<4, MODE>(t, a, s);
}

}  // namespace

int dispatch_grad(const dipole_tree* t, int mode, const QueryArgs& a, cudaStream_t s) {
    if (t->Cp != 1 && t->Cp != 2 && t->Cp % 4 != 0) return dip_fail(-1, "unsupported channel count");
    if (mode == kForwardGrad) launch_grad_cg<kForwardGrad>(t, a, s);
    else if (mode == kForwardGradDot) launch_grad_cg<kForwardGradDot>(t, a, s);
    else if (mode == kAdjointGrad) launch_grad_cg<kAdjointGrad>(t, a, s);
    else if (mode == kAdjointGeom) launch_grad_cg<kAdjointGeom>(t, a, s);
    else return dip_fail(-1, "dispatch_grad: not a gradient mode");
    return 0;
}

}  // namespace dip
