// C ABI entry points (include/dipole.h): argument checks, error reporting and
// the tree object's lifetime.  All compute runs in the kernels of
// tree_build.cu, refit.cu, traverse.cu and sort.cu.
#include <cmath>
#include <atomic>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/dipole.h"
#include "kernels.cuh"
#include "tree.cuh"

namespace {
thread_local std::string g_last_error;
std::atomic<unsigned long long> g_launches{0};
std::atomic<unsigned long long> g_allocs{0};

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Stream-ordered allocations return to the pool on free; keep the pool's
// memory instead of releasing it at every synchronization.
void configure_pool_once() {
    static bool done = false;
    if (done) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done = true;
}

void free_tree_memory(dipole_tree* t) {
    // the arrays live in these blocks, except the lazily made normal/radius scratch
    void* bufs[] = {t->point_block, t->topo_block, t->node_block, t->attr_block, t->dE, t->dgeo,
                    t->tl_block};
    for (void* b : bufs)
        if (b) cudaFree(b);
}

// Kernels of a query run on the current device and follow the tree's device
// pointers: the tree's device must be current.
int check_device(const dipole_tree* t, const char* fn) {
    int dev = -1;
    DIP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != t->device)
        return dip_fail(DIPOLE_EINVAL, std::string(fn) + ": the current CUDA device (" +
                                           std::to_string(dev) + ") is not the tree's device (" +
                                           std::to_string(t->device) + "); make it current first");
    return DIPOLE_OK;
}

int status_to_code(int st) {
    if (st & dip::kStatusBounds) return DIPOLE_EBOUNDS;
    if (st & dip::kStatusTraversal) return DIPOLE_ETRAVERSAL;
    if (st & dip::kStatusNonFinite) return DIPOLE_ENONFINITE;
    return DIPOLE_OK;
}
}  // namespace

void dip::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

cudaError_t dip::dev_alloc(void** p, size_t bytes, cudaStream_t s) {
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMallocAsync(p, bytes, s);
}

int dip_fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int dip_cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    char buf[512];
    snprintf(buf, sizeof(buf), "CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e),
             cudaGetErrorString(e), what, file, line);
    g_last_error = buf;
    return e == cudaErrorMemoryAllocation ? DIPOLE_ENOMEM : DIPOLE_ECUDA;
}

extern "C" {

const char* dipole_last_error(void) { return g_last_error.c_str(); }

uint64_t dipole_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

uint64_t dipole_device_allocations(void) { return g_allocs.load(std::memory_order_relaxed); }

int dipole_checked_build(void) { return dip::kChecked ? 1 : 0; }

int dipole_set_treelet(dipole_tree* tree, int32_t enable) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_set_treelet: tree is NULL");
    if (enable != 0 && enable != 1) return dip_fail(DIPOLE_EINVAL, "dipole_set_treelet: enable must be 0 or 1");
    tree->treelet = enable;
    return DIPOLE_OK;
}

int dipole_traversal_timer(int32_t enable) {
    if (enable != 0 && enable != 1)
        return dip_fail(DIPOLE_EINVAL, "dipole_traversal_timer: enable must be 0 or 1");
    dip::timer_enable(enable != 0);
    return DIPOLE_OK;
}

int dipole_traversal_elapsed(int32_t mode, float* total_ms, int64_t* launches) {
    if (!total_ms || !launches)
        return dip_fail(DIPOLE_EINVAL, "dipole_traversal_elapsed: total_ms and launches are required");
    return dip::timer_elapsed(mode, total_ms, launches);
}

int dipole_build_tree(const float* points, const float* normals, const float* areas,
                      const float* radii, int64_t n, const dipole_build_params* params,
                      void* stream, dipole_tree** out) {
    if (!out) return dip_fail(DIPOLE_EINVAL, "dipole_build_tree: out is NULL");
    *out = nullptr;
    if (!points || !normals || !areas)
        return dip_fail(DIPOLE_EINVAL, "dipole_build_tree: points, normals and areas are required");
    if (n < 1) return dip_fail(DIPOLE_EINVAL, "dipole_build_tree: n must be >= 1");
    if (n > (int64_t)INT32_MAX / 2)
        return dip_fail(DIPOLE_EINVAL, "dipole_build_tree: n must be < 2^30");
    int leaf_size = 8, max_depth = 10, kernel = DIPOLE_KERNEL_REGULARIZED;
    if (params) {
        leaf_size = params->leaf_size;
        max_depth = params->max_depth;
        kernel = params->kernel;
    }
    if (leaf_size < 1 || leaf_size > 64)
        return dip_fail(DIPOLE_EINVAL, "dipole_build_tree: leaf_size must be in [1, 64]");
    if (max_depth < 0 || max_depth > 10)
        return dip_fail(DIPOLE_EINVAL, "dipole_build_tree: max_depth must be in [0, 10]");
    if (kernel != DIPOLE_KERNEL_REGULARIZED && kernel != DIPOLE_KERNEL_DESINGULARIZED)
        return dip_fail(DIPOLE_EINVAL, "dipole_build_tree: kernel must be a dipole_kernel");
    configure_pool_once();
    dipole_tree* t = new (std::nothrow) dipole_tree();
    if (!t) return dip_fail(DIPOLE_ENOMEM, "dipole_build_tree: out of host memory");
    cudaGetDevice(&t->device);
    t->n = n;
    t->leaf_size = leaf_size;
    t->max_depth = max_depth;
    t->kernel = kernel;
    int rc = dip::build_tree(t, points, normals, areas, radii, as_stream(stream));
    if (rc != 0) {
        cudaStreamSynchronize(as_stream(stream));
        free_tree_memory(t);
        delete t;
        return rc;
    }
    *out = t;
    return DIPOLE_OK;
}

int dipole_tree_import(const float* points, const float* normals, const float* areas,
                       const float* radii, int64_t n, const uint32_t* codes, const uint32_t* perm,
                       const int32_t* first, const int32_t* count, const int32_t* level,
                       const int32_t* skip, const int32_t* is_leaf, int64_t n_nodes,
                       const dipole_build_params* params, void* stream, dipole_tree** out) {
    if (!out) return dip_fail(DIPOLE_EINVAL, "dipole_tree_import: out is NULL");
    *out = nullptr;
    if (!points || !normals || !areas || !perm || !first || !count || !level || !skip || !is_leaf)
        return dip_fail(DIPOLE_EINVAL, "dipole_tree_import: a required pointer is NULL");
    if (n < 1 || n > (int64_t)INT32_MAX / 2)
        return dip_fail(DIPOLE_EINVAL, "dipole_tree_import: n must be in [1, 2^30)");
    if (n_nodes < 1 || n_nodes > 2 * n + 1)
        return dip_fail(DIPOLE_EINVAL, "dipole_tree_import: n_nodes must be in [1, 2n+1]");
    int leaf_size = params ? params->leaf_size : 8, max_depth = params ? params->max_depth : 10;
    int kernel = params ? params->kernel : DIPOLE_KERNEL_REGULARIZED;
    if (leaf_size < 1 || leaf_size > 64 || max_depth < 0 || max_depth > 10)
        return dip_fail(DIPOLE_EINVAL, "dipole_tree_import: bad leaf_size or max_depth");
    if (kernel != DIPOLE_KERNEL_REGULARIZED && kernel != DIPOLE_KERNEL_DESINGULARIZED)
        return dip_fail(DIPOLE_EINVAL, "dipole_tree_import: kernel must be a dipole_kernel");
    // Every index a kernel will follow must stay in range; the structure itself
    // (nesting, order) is not checked: a traversal of a corrupt structure ends
    // at its step bound with DIPOLE_ETRAVERSAL.
    std::vector<char> seen((size_t)n, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (perm[i] >= (uint64_t)n || seen[perm[i]])
            return dip_fail(DIPOLE_EINVAL, "dipole_tree_import: perm is not a permutation");
        seen[perm[i]] = 1;
    }
    for (int64_t t = 0; t < n_nodes; ++t) {
        if (is_leaf[t] != 0 && is_leaf[t] != 1)
            return dip_fail(DIPOLE_EINVAL, "dipole_tree_import: is_leaf must be 0 or 1");
        if (level[t] < 0 || level[t] > max_depth)
            return dip_fail(DIPOLE_EINVAL, "dipole_tree_import: level out of range");
        if (first[t] < 0 || first[t] >= n || count[t] < 1 || (int64_t)count[t] > n - first[t])
            return dip_fail(DIPOLE_EINVAL, "dipole_tree_import: node point range out of range");
        if (skip[t] < 0 || (int64_t)skip[t] > n_nodes)
            return dip_fail(DIPOLE_EINVAL, "dipole_tree_import: skip out of range");
    }
    configure_pool_once();
    dipole_tree* t = new (std::nothrow) dipole_tree();
    if (!t) return dip_fail(DIPOLE_ENOMEM, "dipole_tree_import: out of host memory");
    cudaGetDevice(&t->device);
    t->n = n;
    t->nn = n_nodes;
    t->leaf_size = leaf_size;
    t->max_depth = max_depth;
    t->kernel = kernel;
    int rc = dip::import_tree(t, points, normals, areas, radii, codes, perm, first, count, level,
                              skip, is_leaf, as_stream(stream));
    if (rc != 0) {
        cudaStreamSynchronize(as_stream(stream));
        free_tree_memory(t);
        delete t;
        return rc;
    }
    *out = t;
    return DIPOLE_OK;
}

int dipole_refit(dipole_tree* tree, const void* attrs, int32_t channels, int32_t dtype,
                 void* stream) {
    if (!tree || !attrs) return dip_fail(DIPOLE_EINVAL, "dipole_refit: tree and attrs are required");
    if (int rc_dev = check_device(tree, "dipole_refit")) return rc_dev;
    if (channels < 1 || channels > dip::kMaxChannels)
        return dip_fail(DIPOLE_EINVAL, "dipole_refit: channels must be in [1, 64]");
    if (dtype != DIPOLE_F32 && dtype != DIPOLE_BF16 && dtype != DIPOLE_BF16_MOMENTS)
        return dip_fail(DIPOLE_EINVAL, "dipole_refit: dtype must be DIPOLE_F32, DIPOLE_BF16 or "
                                       "DIPOLE_BF16_MOMENTS");
    return dip::refit(tree, attrs, channels, dtype, channels, as_stream(stream));
}

int dipole_refit_appearance(dipole_tree* tree, const void* attrs, int32_t channels, int32_t dtype,
                            int32_t geometry_channels, void* stream) {
    if (!tree || !attrs)
        return dip_fail(DIPOLE_EINVAL, "dipole_refit_appearance: tree and attrs are required");
    if (int rc_dev = check_device(tree, "dipole_refit_appearance")) return rc_dev;
    if (channels < 1 || channels > dip::kMaxChannels)
        return dip_fail(DIPOLE_EINVAL, "dipole_refit_appearance: channels must be in [1, 64]");
    if (geometry_channels < 0 || geometry_channels > channels)
        return dip_fail(DIPOLE_EINVAL,
                        "dipole_refit_appearance: geometry_channels must be in [0, channels]");
    if (dtype != DIPOLE_F32 && dtype != DIPOLE_BF16 && dtype != DIPOLE_BF16_MOMENTS)
        return dip_fail(DIPOLE_EINVAL, "dipole_refit_appearance: dtype must be DIPOLE_F32, "
                                       "DIPOLE_BF16 or DIPOLE_BF16_MOMENTS");
    if (geometry_channels < channels && tree->kernel != DIPOLE_KERNEL_REGULARIZED)
        return dip_fail(DIPOLE_EINVAL, "dipole_refit_appearance: channels without the "
                                       "foreshortening term need the regularized kernel");
    return dip::refit(tree, attrs, channels, dtype, geometry_channels, as_stream(stream));
}

int dipole_forward(const dipole_tree* tree, const float* queries, int64_t q, float beta,
                   float* out, void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_forward: tree is NULL");
    if (int rc_dev = check_device(tree, "dipole_forward")) return rc_dev;
    if (tree->C == 0) return dip_fail(DIPOLE_ESTATE, "dipole_forward: call dipole_refit first");
    if (q < 0) return dip_fail(DIPOLE_EINVAL, "dipole_forward: q must be >= 0");
    if (q > 0 && (!queries || !out))
        return dip_fail(DIPOLE_EINVAL, "dipole_forward: queries and out are required");
    if (q > (int64_t)INT32_MAX) return dip_fail(DIPOLE_EINVAL, "dipole_forward: q must be < 2^31");
    if (!(beta > 0.0f)) return dip_fail(DIPOLE_EINVAL, "dipole_forward: beta must be > 0");
    if (q == 0) return DIPOLE_OK;
    dip::QueryCall c;
    c.mode = dip::kForward;
    c.queries = queries; c.q = q; c.beta = beta; c.out = out;
    return dip::query(tree, c, as_stream(stream));
}

int dipole_forward_noalloc(const dipole_tree* tree, const float* queries, int64_t q, float beta,
                           float* out, void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_forward_noalloc: tree is NULL");
    if (int rc_dev = check_device(tree, "dipole_forward_noalloc")) return rc_dev;
    if (tree->C == 0)
        return dip_fail(DIPOLE_ESTATE, "dipole_forward_noalloc: call dipole_refit first");
    if (q < 0) return dip_fail(DIPOLE_EINVAL, "dipole_forward_noalloc: q must be >= 0");
    if (q > 0 && (!queries || !out))
        return dip_fail(DIPOLE_EINVAL, "dipole_forward_noalloc: queries and out are required");
    if (q > dip::noalloc_max_queries())
        return dip_fail(DIPOLE_EINVAL,
                        "dipole_forward_noalloc: q exceeds the static scratch limit of 262144 "
                        "queries; split the queries or use dipole_forward");
    if (!(beta > 0.0f)) return dip_fail(DIPOLE_EINVAL, "dipole_forward_noalloc: beta must be > 0");
    if (q == 0) return DIPOLE_OK;
    return dip::query_noalloc(tree, queries, q, beta, out, as_stream(stream));
}

int dipole_adjoint(dipole_tree* tree, const float* queries, int64_t q, float beta,
                   const float* grad_out, float* grad_attrs, int32_t accumulate, void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint: tree is NULL");
    if (int rc_dev = check_device(tree, "dipole_adjoint")) return rc_dev;
    if (tree->C == 0) return dip_fail(DIPOLE_ESTATE, "dipole_adjoint: call dipole_refit first");
    if (q < 0) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint: q must be >= 0");
    if (!grad_attrs) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint: grad_attrs is required");
    if (q > 0 && (!queries || !grad_out))
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint: queries and grad_out are required");
    if (q > (int64_t)INT32_MAX) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint: q must be < 2^31");
    if (!(beta > 0.0f)) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint: beta must be > 0");
    if (accumulate != 0 && accumulate != 1)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint: accumulate must be 0 or 1");
    dip::QueryCall c;
    c.mode = dip::kAdjoint;
    c.queries = queries; c.q = q; c.beta = beta;
    c.g = grad_out; c.grad = grad_attrs; c.accumulate = accumulate;
    return dip::query(tree, c, as_stream(stream));
}

int dipole_adjoint_acc_size(const dipole_tree* tree, int64_t* floats) {
    if (!tree || !floats) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_acc_size: NULL argument");
    if (tree->C == 0) return dip_fail(DIPOLE_ESTATE, "dipole_adjoint_acc_size: call dipole_refit first");
    *floats = dip::adjoint_acc_floats(tree);
    return DIPOLE_OK;
}

int dipole_adjoint_stage1(const dipole_tree* tree, const float* queries, int64_t q, float beta,
                          const float* grad_out, float* acc, int32_t accumulate,
                          const uint32_t* plan_perm, const uint32_t* plan_cost, void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_stage1: tree is NULL");
    if (int rc_dev = check_device(tree, "dipole_adjoint_stage1")) return rc_dev;
    if (tree->C == 0) return dip_fail(DIPOLE_ESTATE, "dipole_adjoint_stage1: call dipole_refit first");
    if (q < 0 || q > (int64_t)INT32_MAX)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_stage1: q must be in [0, 2^31)");
    if (!acc) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_stage1: acc is required");
    if (q > 0 && (!queries || !grad_out))
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_stage1: queries and grad_out are required");
    if ((plan_perm == nullptr) != (plan_cost == nullptr))
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_stage1: plan_perm and plan_cost go together");
    if (!(beta > 0.0f)) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_stage1: beta must be > 0");
    if (accumulate != 0 && accumulate != 1)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_stage1: accumulate must be 0 or 1");
    dip::QueryCall c;
    c.mode = dip::kAdjoint;
    c.queries = queries; c.q = q; c.beta = beta;
    c.g = grad_out; c.acc = acc; c.accumulate = accumulate;
    c.plan_perm = const_cast<uint32_t*>(plan_perm);
    c.plan_cost = const_cast<uint32_t*>(plan_cost);
    c.plan_in = plan_perm != nullptr;
    return dip::query(tree, c, as_stream(stream));
}

int dipole_adjoint_stage2(const dipole_tree* tree, const float* acc, float* grad_attrs,
                          int32_t accumulate, void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_stage2: tree is NULL");
    if (int rc_dev = check_device(tree, "dipole_adjoint_stage2")) return rc_dev;
    if (tree->C == 0) return dip_fail(DIPOLE_ESTATE, "dipole_adjoint_stage2: call dipole_refit first");
    if (!acc || !grad_attrs)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_stage2: acc and grad_attrs are required");
    if (accumulate != 0 && accumulate != 1)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_stage2: accumulate must be 0 or 1");
    const int64_t nodes = tree->nn * (int64_t)dip::srow(tree->Cp);
    return dip::stage2(tree, acc, acc + nodes, grad_attrs, accumulate, as_stream(stream));
}

int dipole_adjoint_queries(const dipole_tree* tree, const float* queries, int64_t q, float beta,
                           const float* grad_out, float* grad_queries, int32_t accumulate,
                           void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_queries: tree is NULL");
    if (int rc_dev = check_device(tree, "dipole_adjoint_queries")) return rc_dev;
    if (tree->C == 0) return dip_fail(DIPOLE_ESTATE, "dipole_adjoint_queries: call dipole_refit first");
    if (tree->G < tree->C)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_queries: the spatial, normal and radius gradients are "
                                       "stated for channels with the foreshortening term only");
    if (q < 0 || q > (int64_t)INT32_MAX)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_queries: q must be in [0, 2^31)");
    if (q > 0 && (!queries || !grad_out || !grad_queries))
        return dip_fail(DIPOLE_EINVAL,
                        "dipole_adjoint_queries: queries, grad_out and grad_queries are required");
    if (!(beta > 0.0f)) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_queries: beta must be > 0");
    if (accumulate != 0 && accumulate != 1)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_queries: accumulate must be 0 or 1");
    if (q == 0) return DIPOLE_OK;
    dip::QueryCall c;
    c.mode = dip::kForwardGradDot;
    c.queries = queries; c.q = q; c.beta = beta;
    c.g = grad_out; c.gq = grad_queries; c.accumulate = accumulate;
    return dip::query(tree, c, as_stream(stream));
}

int dipole_forward_planned(const dipole_tree* tree, const float* queries, int64_t q, float beta,
                           float* out, uint32_t* plan_perm, uint32_t* plan_cost, void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_forward_planned: tree is NULL");
    if (int rc_dev = check_device(tree, "dipole_forward_planned")) return rc_dev;
    if (tree->C == 0) return dip_fail(DIPOLE_ESTATE, "dipole_forward_planned: call dipole_refit first");
    if (q < 0 || q > (int64_t)INT32_MAX)
        return dip_fail(DIPOLE_EINVAL, "dipole_forward_planned: q must be in [0, 2^31)");
    if (q > 0 && (!queries || !out || !plan_perm || !plan_cost))
        return dip_fail(DIPOLE_EINVAL, "dipole_forward_planned: queries, out and the plan are required");
    if (!(beta > 0.0f)) return dip_fail(DIPOLE_EINVAL, "dipole_forward_planned: beta must be > 0");
    if (q == 0) return DIPOLE_OK;
    dip::QueryCall c;
    c.mode = dip::kForward;
    c.queries = queries; c.q = q; c.beta = beta; c.out = out;
    c.plan_perm = plan_perm; c.plan_cost = plan_cost;
    return dip::query(tree, c, as_stream(stream));
}

int dipole_adjoint_planned(dipole_tree* tree, const float* queries, int64_t q, float beta,
                           const float* grad_out, float* grad_attrs, int32_t accumulate,
                           const uint32_t* plan_perm, const uint32_t* plan_cost, void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_planned: tree is NULL");
    if (int rc_dev = check_device(tree, "dipole_adjoint_planned")) return rc_dev;
    if (tree->C == 0) return dip_fail(DIPOLE_ESTATE, "dipole_adjoint_planned: call dipole_refit first");
    if (q < 0 || q > (int64_t)INT32_MAX)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_planned: q must be in [0, 2^31)");
    if (!grad_attrs) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_planned: grad_attrs is required");
    if (q > 0 && (!queries || !grad_out || !plan_perm || !plan_cost))
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_planned: queries, grad_out and the plan are required");
    if (!(beta > 0.0f)) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_planned: beta must be > 0");
    if (accumulate != 0 && accumulate != 1)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_planned: accumulate must be 0 or 1");
    dip::QueryCall c;
    c.mode = dip::kAdjoint;
    c.queries = queries; c.q = q; c.beta = beta;
    c.g = grad_out; c.grad = grad_attrs; c.accumulate = accumulate;
    c.plan_perm = const_cast<uint32_t*>(plan_perm);
    c.plan_cost = const_cast<uint32_t*>(plan_cost);
    c.plan_in = true;
    return dip::query(tree, c, as_stream(stream));
}

int dipole_forward_grad(const dipole_tree* tree, const float* queries, int64_t q, float beta,
                        float* out, float* grad_x, uint32_t* plan_perm, uint32_t* plan_cost,
                        void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_forward_grad: tree is NULL");
    if (int rc_dev = check_device(tree, "dipole_forward_grad")) return rc_dev;
    if (tree->C == 0) return dip_fail(DIPOLE_ESTATE, "dipole_forward_grad: call dipole_refit first");
    if (tree->G < tree->C)
        return dip_fail(DIPOLE_EINVAL, "dipole_forward_grad: the spatial, normal and radius gradients are "
                                       "stated for channels with the foreshortening term only");
    if (q < 0 || q > (int64_t)INT32_MAX)
        return dip_fail(DIPOLE_EINVAL, "dipole_forward_grad: q must be in [0, 2^31)");
    if (q > 0 && (!queries || !grad_x))
        return dip_fail(DIPOLE_EINVAL, "dipole_forward_grad: queries and grad_x are required");
    if ((plan_perm == nullptr) != (plan_cost == nullptr))
        return dip_fail(DIPOLE_EINVAL, "dipole_forward_grad: plan_perm and plan_cost go together");
    if (!(beta > 0.0f)) return dip_fail(DIPOLE_EINVAL, "dipole_forward_grad: beta must be > 0");
    if (q == 0) return DIPOLE_OK;
    dip::QueryCall c;
    c.mode = dip::kForwardGrad;
    c.queries = queries; c.q = q; c.beta = beta; c.out = out; c.gout = grad_x;
    c.plan_perm = plan_perm; c.plan_cost = plan_cost;
    return dip::query(tree, c, as_stream(stream));
}

int dipole_adjoint_grad(dipole_tree* tree, const float* queries, int64_t q, float beta,
                        const float* grad_out, const float* grad_grad, float* grad_attrs,
                        int32_t accumulate, const uint32_t* plan_perm, const uint32_t* plan_cost,
                        void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_grad: tree is NULL");
    if (int rc_dev = check_device(tree, "dipole_adjoint_grad")) return rc_dev;
    if (tree->C == 0) return dip_fail(DIPOLE_ESTATE, "dipole_adjoint_grad: call dipole_refit first");
    if (tree->G < tree->C)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_grad: the spatial, normal and radius gradients are "
                                       "stated for channels with the foreshortening term only");
    if (q < 0 || q > (int64_t)INT32_MAX)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_grad: q must be in [0, 2^31)");
    if (!grad_attrs) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_grad: grad_attrs is required");
    if (q > 0 && (!queries || (!grad_out && !grad_grad)))
        return dip_fail(DIPOLE_EINVAL,
                        "dipole_adjoint_grad: queries and one of grad_out, grad_grad are required");
    if ((plan_perm == nullptr) != (plan_cost == nullptr))
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_grad: plan_perm and plan_cost go together");
    if (!(beta > 0.0f)) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_grad: beta must be > 0");
    if (accumulate != 0 && accumulate != 1)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_grad: accumulate must be 0 or 1");
    dip::QueryCall c;
    c.mode = dip::kAdjointGrad;
    c.queries = queries; c.q = q; c.beta = beta;
    c.g = grad_out; c.gg = grad_grad; c.grad = grad_attrs; c.accumulate = accumulate;
    c.plan_perm = const_cast<uint32_t*>(plan_perm);
    c.plan_cost = const_cast<uint32_t*>(plan_cost);
    c.plan_in = plan_perm != nullptr;
    return dip::query(tree, c, as_stream(stream));
}

int dipole_adjoint_geom(dipole_tree* tree, const float* queries, int64_t q, float beta,
                        const float* grad_out, const float* grad_grad, float* grad_attrs,
                        float* grad_normals, float* grad_radii, int32_t accumulate,
                        const uint32_t* plan_perm, const uint32_t* plan_cost, void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_geom: tree is NULL");
    if (int rc_dev = check_device(tree, "dipole_adjoint_geom")) return rc_dev;
    if (tree->C == 0) return dip_fail(DIPOLE_ESTATE, "dipole_adjoint_geom: call dipole_refit first");
    if (tree->G < tree->C)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_geom: the spatial, normal and radius gradients are "
                                       "stated for channels with the foreshortening term only");
    if (q < 0 || q > (int64_t)INT32_MAX)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_geom: q must be in [0, 2^31)");
    if (!grad_attrs && !grad_normals && !grad_radii)
        return dip_fail(DIPOLE_EINVAL,
                        "dipole_adjoint_geom: one of grad_attrs, grad_normals, grad_radii is required");
    if (q > 0 && (!queries || (!grad_out && !grad_grad)))
        return dip_fail(DIPOLE_EINVAL,
                        "dipole_adjoint_geom: queries and one of grad_out, grad_grad are required");
    if ((plan_perm == nullptr) != (plan_cost == nullptr))
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_geom: plan_perm and plan_cost go together");
    if (!(beta > 0.0f)) return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_geom: beta must be > 0");
    if (accumulate != 0 && accumulate != 1)
        return dip_fail(DIPOLE_EINVAL, "dipole_adjoint_geom: accumulate must be 0 or 1");
    cudaStream_t s = as_stream(stream);
    int rc = dip::ensure_geom_scratch(tree, s);
    if (rc) return rc;
    dip::QueryCall c;
    c.mode = dip::kAdjointGeom;
    c.queries = queries; c.q = q; c.beta = beta;
    c.g = grad_out; c.gg = grad_grad;
    c.grad = grad_attrs; c.grad_n = grad_normals; c.grad_eps = grad_radii;
    c.accumulate = accumulate;
    c.plan_perm = const_cast<uint32_t*>(plan_perm);
    c.plan_cost = const_cast<uint32_t*>(plan_cost);
    c.plan_in = plan_perm != nullptr;
    return dip::query(tree, c, s);
}

int dipole_forward_grid(const dipole_tree* tree, const float* lo, float spacing,
                        const int64_t* dims, float beta, float* out, void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_forward_grid: tree is NULL");
    if (int rc_dev = check_device(tree, "dipole_forward_grid")) return rc_dev;
    if (tree->C == 0) return dip_fail(DIPOLE_ESTATE, "dipole_forward_grid: call dipole_refit first");
    if (!lo || !dims || !out)
        return dip_fail(DIPOLE_EINVAL, "dipole_forward_grid: lo, dims and out are required");
    if (!(spacing > 0.0f) || !std::isfinite(spacing))
        return dip_fail(DIPOLE_EINVAL, "dipole_forward_grid: spacing must be finite and > 0");
    int64_t total = 1;
    for (int d = 0; d < 3; ++d) {
        if (!std::isfinite(lo[d])) return dip_fail(DIPOLE_EINVAL, "dipole_forward_grid: lo must be finite");
        if (dims[d] < 1 || dims[d] > (int64_t(1) << 24))
            return dip_fail(DIPOLE_EINVAL, "dipole_forward_grid: dims must be in [1, 2^24]");
        total *= dims[d];
        if (total > (int64_t(1) << 40))
            return dip_fail(DIPOLE_EINVAL, "dipole_forward_grid: more than 2^40 grid points");
    }
    if (!(beta > 0.0f)) return dip_fail(DIPOLE_EINVAL, "dipole_forward_grid: beta must be > 0");
    dip::QueryCall c;
    c.mode = dip::kForward;
    c.q = total; c.beta = beta; c.out = out;
    for (int d = 0; d < 3; ++d) {
        c.grid_lo[d] = lo[d];
        c.grid_dim[d] = dims[d];
    }
    c.grid_h = spacing;
    return dip::query(tree, c, as_stream(stream));
}

int dipole_query_counts(const dipole_tree* tree, const float* queries, int64_t q, float beta,
                        int32_t* counts, void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_query_counts: tree is NULL");
    if (int rc_dev = check_device(tree, "dipole_query_counts")) return rc_dev;
    if (q < 0) return dip_fail(DIPOLE_EINVAL, "dipole_query_counts: q must be >= 0");
    if (q > 0 && (!queries || !counts))
        return dip_fail(DIPOLE_EINVAL, "dipole_query_counts: queries and counts are required");
    if (q > (int64_t)INT32_MAX) return dip_fail(DIPOLE_EINVAL, "dipole_query_counts: q must be < 2^31");
    if (!(beta > 0.0f)) return dip_fail(DIPOLE_EINVAL, "dipole_query_counts: beta must be > 0");
    if (q == 0) return DIPOLE_OK;
    dip::QueryCall c;
    c.mode = dip::kCount;
    c.queries = queries; c.q = q; c.beta = beta; c.counts = counts;
    return dip::query(tree, c, as_stream(stream));
}

int dipole_query_packet_counts(const dipole_tree* tree, const float* queries, int64_t q,
                               float beta, int32_t* counts, int32_t* packet_counts,
                               void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_query_packet_counts: tree is NULL");
    if (int rc_dev = check_device(tree, "dipole_query_packet_counts")) return rc_dev;
    if (q < 0 || q > (int64_t)INT32_MAX)
        return dip_fail(DIPOLE_EINVAL, "dipole_query_packet_counts: q must be in [0, 2^31)");
    if (q > 0 && (!queries || !packet_counts))
        return dip_fail(DIPOLE_EINVAL,
                        "dipole_query_packet_counts: queries and packet_counts are required");
    if (!(beta > 0.0f)) return dip_fail(DIPOLE_EINVAL, "dipole_query_packet_counts: beta must be > 0");
    if (q == 0) return DIPOLE_OK;
    dip::QueryCall c;
    c.mode = dip::kCount;
    c.queries = queries; c.q = q; c.beta = beta; c.counts = counts; c.ucounts = packet_counts;
    return dip::query(tree, c, as_stream(stream));
}

int dipole_sync_status(dipole_tree* tree, void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_sync_status: tree is NULL");
    int st = 0;
    DIP_CUDA_TRY(cudaMemcpyAsync(&st, tree->status, sizeof(int), cudaMemcpyDeviceToHost,
                                 as_stream(stream)));
    DIP_CUDA_TRY(cudaMemsetAsync(tree->status, 0, sizeof(int), as_stream(stream)));
    DIP_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    DIP_CUDA_TRY(cudaGetLastError());
    int code = status_to_code(st);
    if (code == DIPOLE_EBOUNDS)
        return dip_fail(code, "an index outside its array was caught and skipped (checked build)");
    if (code == DIPOLE_ETRAVERSAL)
        return dip_fail(code, "a traversal exceeded its step bound (corrupt tree)");
    if (code == DIPOLE_ENONFINITE) return dip_fail(code, "a non-finite query point was seen");
    return DIPOLE_OK;
}

int dipole_tree_info_get(const dipole_tree* tree, dipole_tree_info* info) {
    if (!tree || !info) return dip_fail(DIPOLE_EINVAL, "dipole_tree_info_get: NULL argument");
    info->n_points = tree->n;
    info->n_nodes = tree->nn;
    info->channels = tree->C;
    info->dtype = tree->S16 ? DIPOLE_BF16_MOMENTS : tree->dtype;
    info->leaf_size = tree->leaf_size;
    info->max_depth = tree->max_depth;
    for (int a = 0; a < 3; ++a) info->bbox_lo[a] = tree->bbox_host[a];
    info->bbox_ext = tree->bbox_host[3];
    info->kernel = tree->kernel;
    return DIPOLE_OK;
}

int dipole_tree_export(const dipole_tree* tree, uint32_t* codes, uint32_t* perm, int32_t* first,
                       int32_t* count, int32_t* level, int32_t* parent, int32_t* skip,
                       int32_t* is_leaf, float* centroid, float* radius, double* area,
                       float* eps, float* moments, void* stream) {
    if (!tree) return dip_fail(DIPOLE_EINVAL, "dipole_tree_export: tree is NULL");
    if (moments && tree->C == 0)
        return dip_fail(DIPOLE_ESTATE, "dipole_tree_export: moments need a refit first");
    cudaStream_t s = as_stream(stream);
    const size_t n = (size_t)tree->n, nn = (size_t)tree->nn;
    auto cp = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
        return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) : cudaSuccess;
    };
    DIP_CUDA_TRY(cp(codes, tree->code, n * 4));
    DIP_CUDA_TRY(cp(perm, tree->perm, n * 4));
    DIP_CUDA_TRY(cp(first, tree->first, nn * 4));
    DIP_CUDA_TRY(cp(count, tree->count, nn * 4));
    DIP_CUDA_TRY(cp(level, tree->level, nn * 4));
    DIP_CUDA_TRY(cp(parent, tree->parent, nn * 4));
    DIP_CUDA_TRY(cp(skip, tree->skip, nn * 4));
    DIP_CUDA_TRY(cp(is_leaf, tree->is_leaf, nn * 4));
    DIP_CUDA_TRY(cp(eps, tree->eps_node, nn * 4));
    if (centroid || radius || area) {
        dip::NodeRec* hn = new dip::NodeRec[nn];
        double* agg = new double[nn * 5];
        cudaError_t e1 = cudaMemcpyAsync(hn, tree->nodes, nn * sizeof(dip::NodeRec),
                                         cudaMemcpyDeviceToHost, s);
        cudaError_t e2 = cudaMemcpyAsync(agg, tree->agg64, nn * 5 * sizeof(double),
                                         cudaMemcpyDeviceToHost, s);
        cudaError_t e3 = cudaStreamSynchronize(s);
        if (e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess) {
            for (size_t t = 0; t < nn; ++t) {
                if (centroid) {
                    centroid[3 * t] = hn[t].geo.x;
                    centroid[3 * t + 1] = hn[t].geo.y;
                    centroid[3 * t + 2] = hn[t].geo.z;
                }
                if (radius) radius[t] = hn[t].geo.w;
                if (area) area[t] = agg[5 * t];
            }
        }
        delete[] hn;
        delete[] agg;
        DIP_CUDA_TRY(e1);
        DIP_CUDA_TRY(e2);
        DIP_CUDA_TRY(e3);
    }
    if (moments) {
        const int C = tree->C, SR = dip::srow(tree->Cp);
        float* hs = new float[nn * SR];
        cudaError_t e1 = cudaMemcpyAsync(hs, tree->S, nn * SR * sizeof(float),
                                         cudaMemcpyDeviceToHost, s);
        cudaError_t e2 = cudaStreamSynchronize(s);
        if (e1 == cudaSuccess && e2 == cudaSuccess)
            for (size_t t = 0; t < nn; ++t)
                for (int j = 0; j < 3 * C; ++j) moments[t * 3 * C + j] = hs[t * SR + j];
        delete[] hs;
        DIP_CUDA_TRY(e1);
        DIP_CUDA_TRY(e2);
    }
    DIP_CUDA_TRY(cudaStreamSynchronize(s));
    return DIPOLE_OK;
}

int dipole_probe_l2(const void* buf, int64_t bytes, int32_t passes, float* sink, void* stream) {
    if (!buf || !sink) return dip_fail(DIPOLE_EINVAL, "dipole_probe_l2: buf and sink are required");
    if (bytes < 16 || (bytes % 16) != 0 || (reinterpret_cast<uintptr_t>(buf) % 16) != 0)
        return dip_fail(DIPOLE_EINVAL, "dipole_probe_l2: bytes must be a positive multiple of 16 "
                                       "and buf 16-byte aligned");
    if (passes < 1) return dip_fail(DIPOLE_EINVAL, "dipole_probe_l2: passes must be >= 1");
    dip::probe_l2(buf, bytes, passes, sink, as_stream(stream));
    DIP_CUDA_TRY(cudaGetLastError());
    return DIPOLE_OK;
}

void dipole_tree_destroy(dipole_tree* tree) {
    if (!tree) return;
    cudaDeviceSynchronize();
    free_tree_memory(tree);
    delete tree;
}

}  // extern "C"
