// The tree object behind the opaque dipole_tree handle, and the host launchers
// of the build, refit and query kernels.
#pragma once

#include <mutex>

#include "common.cuh"


struct dipole_tree {
    int device = 0;
    int64_t n = 0;
    int64_t nn = 0;
    int leaf_size = 8;
    int max_depth = 10;
    int kernel = 0;              // dipole_kernel: 0 regularized, 1 desingularized

    // points, Morton order
    dip::PointRec* pts = nullptr;
    uint32_t* code = nullptr;
    uint32_t* perm = nullptr;
    int32_t* leaf_of = nullptr;  // [n] leaf node holding each point

    // device memory is taken in a few blocks (one allocation each, the arrays
    // below point into them): points, topology, nodes, attribute state
    void* point_block = nullptr;
    void* topo_block = nullptr;
    void* node_block = nullptr;
    void* attr_block = nullptr;

    // nodes, depth-first preorder
    dip::NodeRec* nodes = nullptr;
    int32_t* first = nullptr;
    int32_t* count = nullptr;
    int32_t* level = nullptr;
    int32_t* parent = nullptr;
    int32_t* skip = nullptr;
    int32_t* is_leaf = nullptr;
    int32_t* nchild = nullptr;
    int32_t* lvl_list = nullptr; // internal nodes grouped by level
    int32_t* lvl_off = nullptr;  // [kMaxLevel + 2] start of each level in lvl_list
    double* agg64 = nullptr;     // [nn, 5] sum A, sum A p (3), sum A eps
    float* eps_node = nullptr;   // [nn]
    float* bbox = nullptr;       // device: lo.xyz, ext, 1024/ext
    float bbox_host[5] = {0, 0, 0, 1, 1024};
    int* status = nullptr;       // device status word

    // attributes (set by refit)
    int C = 0;
    int G = 0;                   // channels [0, G) with the foreshortening term, [G, C) without
    int Cp = 0;
    int dtype = 0;               // attribute storage: 0 float, 1 bf16
    void* mu = nullptr;          // [n, Cp] float or bf16, Morton order
    float* S = nullptr;          // [nn, 3 Cp]
    uint16_t* S16 = nullptr;     // [nn, srow16(Cp)] S rounded to bf16 (DIPOLE_BF16_MOMENTS), or NULL
    // refit scratch: fixed-point prefix of the leaf moments over preorder
    long long* fix_P = nullptr;     // [3 Cp, nn + 1 rounded up to 4], column-major
    long long* fix_tsum = nullptr;  // [tiles, 3 Cp] tile sums, then tile offsets
    unsigned* fix_cmax = nullptr;   // [3 Cp] largest |leaf moment| (float bits), 0 between refits
    int* fix_kexp = nullptr;        // [3 Cp] column scale exponents
    unsigned* fix_done = nullptr;   // tile arrival counter, 0 between refits
    float* dS = nullptr;         // [nn, 3 Cp] adjoint node accumulators
    float* dmu = nullptr;        // [n, Cp] adjoint opened-leaf accumulators
    float* dE = nullptr;         // [nn] adjoint d eps~_t sums (normal/radius gradients)
    float* dgeo = nullptr;       // [n, 4] adjoint opened-leaf normal and radius terms
    int attr_Cp_alloc = 0;
    int attr_dtype_alloc = -1;
    // treelet (dipole_set_treelet): the upper tree staged in shared memory by
    // the value forward; its block (records + node copy) is made on first use
    int treelet = 0;
    mutable void* tl_block = nullptr;  // TLRec [80], treelet node ids [80], node copy [nn]

    dip::TreeView view() const {
        dip::TreeView v;
        v.n = n;
        v.nn = nn;
        v.nodes = nodes;
        v.pts = pts;
        v.perm = perm;
        v.parent = parent;
        v.first = first;
        v.count = count;
        v.is_leaf = is_leaf;
        v.bbox = bbox;
        v.status = status;
        return v;
    }
};

namespace dip {

// Build everything but the attribute state.  Returns a dipole_status.
int build_tree(dipole_tree* t, const float* points, const float* normals, const float* areas,
               const float* radii, cudaStream_t s);

// Rebuild a tree from exported topology (host arrays) and point inputs (device),
// t->n, t->nn and the parameters already set; the host arrays are validated.
int import_tree(dipole_tree* t, const float* points, const float* normals, const float* areas,
                const float* radii, const uint32_t* codes_h, const uint32_t* perm_h,
                const int32_t* first_h, const int32_t* count_h, const int32_t* level_h,
                const int32_t* skip_h, const int32_t* is_leaf_h, cudaStream_t s);

// Tree update of node moments (eq. farfield_dipole_features).
// Channels [G, C) skip the foreshortening term: their moment row holds
// M^c = sum A mu^c in its first slot (0 in the other two).
int refit(dipole_tree* t, const void* attrs, int C, int dtype, int G, cudaStream_t s);

// Query modes: the dipole sum (eq. dipole_sum with Alg. 1), its adjoint, the
// traversal counters, the sum with its spatial gradient, the adjoint of both,
// and that adjoint extended to the normals and radii.
// kForwardGradDot: the spatial-gradient walk that returns only
// sum_c g^c grad D^c per query (the chain rule of a loss of D in the query
// positions).
enum { kForward = 0, kAdjoint = 1, kCount = 2, kForwardGrad = 3, kAdjointGrad = 4, kAdjointGeom = 5,
       kForwardGradDot = 6 };

// One query call.  Query plan (caller-owned, optional): plan_in = false writes
// the Morton permutation into plan_perm [q] and each packet's warp steps into
// plan_cost [ceil(q/32)]; plan_in = true reads them instead of sorting, and
// runs packets longest first.
struct QueryCall {
    int mode = kForward;
    const float* queries = nullptr;  // [q, 3]
    int64_t q = 0;
    float beta = 2.0f;
    float* out = nullptr;            // D [q, C] (kForward; optional in kForwardGrad)
    float* gout = nullptr;           // grad D [q, C, 3] (kForwardGrad)
    const float* g = nullptr;        // dL/dD [q, C] (kAdjoint; optional in kAdjointGrad)
    const float* gg = nullptr;       // dL/d(grad D) [q, C, 3] (optional in kAdjointGrad)
    float* grad = nullptr;           // dL/dmu [n, C] (adjoint modes; optional in kAdjointGeom)
    float* grad_n = nullptr;         // dL/dn [n, 3] (optional in kAdjointGeom)
    float* grad_eps = nullptr;       // dL/deps [n] (optional in kAdjointGeom)
    int accumulate = 0;
    float* gq = nullptr;             // dL/dx [q, 3] = sum_c g^c grad D^c (kForwardGradDot)
    // stage 1 only: the adjoint's node and opened-leaf sums go to acc
    // (adjoint_acc_floats entries: dS, then dmu_near) instead of the tree's
    // scratch, and stage 2 is not run
    float* acc = nullptr;
    int32_t* counts = nullptr;       // [q, 3] (kCount)
    int32_t* ucounts = nullptr;      // [ceil(q/32), 4] per-packet warp counts (kCount, optional)
    uint32_t* plan_perm = nullptr;
    uint32_t* plan_cost = nullptr;
    bool plan_in = false;
    // dense grid (kForward / kCount): queries = lo + h (i, j, k), out in
    // x-fastest grid order; grid_dim[0] = 0 means no grid
    float grid_lo[3] = {0.f, 0.f, 0.f};
    float grid_h = 0.f;
    int64_t grid_dim[3] = {0, 0, 0};
};

int query(const dipole_tree* t, const QueryCall& call, cudaStream_t s);

// Traversal timer (dipole_traversal_timer / dipole_traversal_elapsed): when
// enabled, every query call records a CUDA event pair on its stream around
// its traversal kernel launch, kept per query mode.
void timer_enable(bool on);
int timer_elapsed(int mode, float* total_ms, int64_t* launches);

// Forward queries with all scratch in a static device array (no allocation);
// q <= noalloc_max_queries().
int query_noalloc(const dipole_tree* t, const float* queries, int64_t q, float beta, float* out,
                  cudaStream_t s);
int64_t noalloc_max_queries();

// Stage 2 of the adjoint (eq. farfield_features_gradient) into grad [n, C],
// from the node sums dS [nn, srow(Cp)] and opened-leaf sums dmu [n, Cp].
int stage2(const dipole_tree* t, const float* dS, const float* dmu, float* grad, int accumulate,
           cudaStream_t s);

// Entries of a stage-1 accumulator: dS [nn, srow(Cp)], then dmu [n, Cp].
int64_t adjoint_acc_floats(const dipole_tree* t);

// Scratch of the normal/radius adjoint (dE, dgeo), allocated on first use.
int ensure_geom_scratch(dipole_tree* t, cudaStream_t s);

// Stage 2 for the normals and radii: grad_n [n, 3] and grad_eps [n] (either
// may be NULL), caller order.
int stage2_geom(const dipole_tree* t, float* grad_n, float* grad_eps, int accumulate,
                cudaStream_t s);

}  // namespace dip
