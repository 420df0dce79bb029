/*
 * dipole.h -- C ABI of the GB300 (sm_103a) library for Barnes-Hut fast
 * summation of regularized dipole sums, forward and adjoint.
 *
 * Method: Chen, Miller, Gkioulekas, "3D Reconstruction with Fast Dipole Sums"
 * (arXiv 2405.16788).  For points p_m with outward unit normals n_m, area
 * weights A_m > 0, regularization radii eps_m >= 0 and C attribute channels
 * mu_m^c, the library evaluates at query points x
 *
 *   D^c(x) = sum_m A_m rho(|p_m - x| / eps_m) n_m.(p_m - x) / (4 pi |p_m - x|^3) mu_m^c,
 *   rho(t) = erf(t) - (2t/sqrt(pi)) exp(-t^2)
 *
 * (Sec. 4.2, eq. dipole_sum; Sec. 4.1, eq. regularized_poisson; Sec. 5.1,
 * eq. appearance_features for several channels), approximated by Barnes-Hut
 * (Sec. 6.1, eq. farfield; Alg. 1, PrimalQuery), and its adjoint with respect
 * to mu by the two-stage scheme of Sec. 6.2 (Alg. 1, AdjointQuery; App. C,
 * eqs. farfield_gradient and farfield_features_gradient).
 *
 * Conventions shared by every entry point:
 *  - Array arguments are DEVICE pointers on the current CUDA device, owned by
 *    the caller, unless a comment says "host".  Float arrays are row-major
 *    and contiguous.  Points, attributes and gradients are in the caller's
 *    order; the library keeps its own Morton-ordered copies.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *    asynchronous on it unless a comment says otherwise.
 *  - Every call returns a dipole_status; nothing crosses the ABI as a C++
 *    exception.  On failure dipole_last_error() gives a message for the
 *    calling thread.  Errors found by kernels (a traversal that exceeded its
 *    step bound, a non-finite query) set a device status word that
 *    dipole_sync_status() returns and clears.
 *  - The tree owns its device memory; dipole_tree_destroy releases it.
 */
#ifndef DIPOLE_H
#define DIPOLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dipole_tree dipole_tree;

typedef enum {
    DIPOLE_OK = 0,
    DIPOLE_EINVAL = -1,      /* bad argument (null pointer, size, non-positive area, ...) */
    DIPOLE_ENOMEM = -2,      /* device allocation failed */
    DIPOLE_ECUDA = -3,       /* a CUDA call failed; see dipole_last_error() */
    DIPOLE_ENONFINITE = -4,  /* a non-finite input was found */
    DIPOLE_ETRAVERSAL = -5,  /* a traversal exceeded its step bound (corrupt tree) */
    DIPOLE_ESTATE = -6,      /* call out of order (e.g. forward before any refit) */
    DIPOLE_EBOUNDS = -7      /* checked build only (compiled with -DDIPOLE_CHECKED): a
                                traversal met an index outside its array and skipped the
                                access; the outputs of that call are incomplete */
} dipole_status;

/* Attribute storage.  DIPOLE_BF16_MOMENTS stores the attributes as bf16 like
 * DIPOLE_BF16 and adds a bf16 copy of the node moments S_t^c, which the
 * value forward (dipole_forward and its planned, grid and no-alloc forms)
 * reads for far nodes; the gradient and adjoint queries keep the float
 * moments.  Arithmetic is float in every case. */
typedef enum { DIPOLE_F32 = 0, DIPOLE_BF16 = 1, DIPOLE_BF16_MOMENTS = 2 } dipole_dtype;

/* Radial factor of the kernel.  REGULARIZED is the paper's method:
 * rho(r/eps)/r^3 with rho of eq. regularized_poisson (Sec. 4.1).
 * DESINGULARIZED is the ablation baseline the paper compares against
 * (Sec. 4.1 footnote; Sec. 7 ablation), which bounds the kernel's
 * denominator away from zero; read as 1/max(r, eps)^3 with the point's radius
 * eps as the cutoff (eps~ at a far node); eps = 0 gives the singular kernel in
 * both. */
typedef enum { DIPOLE_KERNEL_REGULARIZED = 0, DIPOLE_KERNEL_DESINGULARIZED = 1 } dipole_kernel;

/* Octree parameters.  leaf_size in [1, 64] (the paper's leaves are single
 * points, Sec. 6.1; 8 is the default here); max_depth in [0, 10] octal digits
 * of the 30-bit Morton code; kernel a dipole_kernel (default REGULARIZED). */
typedef struct {
    int32_t leaf_size;
    int32_t max_depth;
    int32_t kernel;
} dipole_build_params;

typedef struct {
    int64_t n_points;
    int64_t n_nodes;
    int32_t channels;    /* C of the last refit, 0 before the first */
    int32_t dtype;       /* dipole_dtype of the last refit */
    int32_t leaf_size;
    int32_t max_depth;
    float bbox_lo[3];    /* bounding cube of the Morton quantisation */
    float bbox_ext;
    int32_t kernel;      /* dipole_kernel of the build */
} dipole_tree_info;

/*
 * Build the octree over n points (Sec. 6.3, "tree construction and update":
 * built once, positions are not optimized) and the node geometry of
 * Sec. 6.1, eq. farfield_dipole: area A~_t = sum A_m, centroid
 * p~_t = sum A_m p_m / A~_t, radius r~_t = max |p_m - p~_t|, and the node
 * regularization radius eps~_t = sum A_m eps_m / A~_t.
 *
 *   points  [n,3] float   positions p_m
 *   normals [n,3] float   outward unit normals n_m
 *   areas   [n]   float   area weights A_m, each > 0
 *   radii   [n]   float   regularization radii eps_m >= 0, or NULL for all 0
 *                         (eps = 0 is the singular kernel of eq. pcwn)
 *   n       >= 1
 *   params  NULL for {leaf_size 8, max_depth 10}
 *   out     receives the new tree (host pointer to a host pointer)
 *
 * The tree is the compressed 30-bit Morton octree: bounding cube, per-axis
 * quantisation to 1024 cells, codes sorted stably, nodes = maximal runs of
 * equal code prefixes that branch, leaves = runs of at most leaf_size points
 * (or at max_depth), in depth-first preorder.  Its integer arrays are
 * bit-identical to the CPU oracle's.
 *
 * Synchronizes `stream` once (the node count sizes the node arrays).
 * Errors: DIPOLE_EINVAL for a null pointer, n < 1, bad params, an area <= 0
 * or a negative radius; DIPOLE_ENONFINITE for a non-finite input.
 */
int dipole_build_tree(const float* points, const float* normals, const float* areas,
                      const float* radii, int64_t n, const dipole_build_params* params,
                      void* stream, dipole_tree** out);

/*
 * Tree update of the node moments (Sec. 6.3: done at the start of every
 * iteration; Sec. 6.1, eq. farfield_dipole_features):
 *   S_t^c = A~_t n~_t^c = sum_{m in t} A_m n_m mu_m^c   (3 values per channel)
 *
 *   attrs     [n, channels] float (dtype DIPOLE_F32) or bfloat16 (DIPOLE_BF16,
 *             DIPOLE_BF16_MOMENTS)
 *   channels  in [1, 64]
 *
 * The attributes are copied into Morton order in the given dtype (bf16
 * storage halves their bytes; arithmetic is float).  A leaf's moments are
 * float sums over its points; a larger node's are exact sums of its leaves'
 * (64-bit fixed point) rounded once to float.  DIPOLE_BF16_MOMENTS rounds
 * those floats once more, to bf16 (nearest even), for the value forward.
 * Errors: DIPOLE_EINVAL for a null pointer or a bad channel count/dtype.
 */
int dipole_refit(dipole_tree* tree, const void* attrs, int32_t channels, int32_t dtype,
                 void* stream);

/*
 * dipole_refit with appearance channels that skip the foreshortening term
 * (Sec. 5.3, radiance field details: the paper interpolates its appearance
 * attributes by eq. appearance_features without that term and says no more).
 * Read here as: the term is the cosine n.(p - x)/|p - x| of the kernel, so a
 * point contributes A_m rho(r/eps_m)/(4 pi r^2) mu_m^c and a far node
 * rho(d/eps~_t)/(4 pi d^2) M_t^c with M_t^c = sum_{m in t} A_m mu_m^c (the
 * zeroth-order far field of eq. farfield for this kernel); the adjoint's
 * stage 2 gives dL/dmu_m^c = A_m sum_{t holding m} dM_t^c.
 *
 *   geometry_channels  G in [0, channels]: channels [0, G) use eq. dipole_sum
 *                      (with the term), channels [G, channels) skip it;
 *                      G = channels is dipole_refit
 *
 * Every query entry point evaluates each channel with its kernel, in one
 * traversal.  The spatial, normal and radius gradients (dipole_forward_grad,
 * dipole_adjoint_grad, dipole_adjoint_geom, dipole_adjoint_queries) are
 * stated for channels with the term only and return DIPOLE_EINVAL on a tree
 * refit with G < channels.  dipole_tree_export's moments hold M_t^c in the
 * first slot of such a channel (0 in the other two).
 * Errors: as dipole_refit; DIPOLE_EINVAL for G outside [0, channels] or, when
 * G < channels, a tree built with the desingularized kernel.
 */
int dipole_refit_appearance(dipole_tree* tree, const void* attrs, int32_t channels, int32_t dtype,
                            int32_t geometry_channels, void* stream);

/*
 * Primal queries (Alg. 1, PrimalQuery; all channels in one traversal, Sec.
 * 5.3): out[j, c] = Barnes-Hut estimate of D^c(queries[j]).  A node t is far
 * when |x - p~_t| > beta r~_t (strict), evaluated in float as
 *   dx = x - p~ (per axis), d2 = fma(dz,dz, fma(dy,dy, dx*dx)), R = beta*r~,
 *   far = d2 > R*R;
 * a far node contributes rho(d/eps~_t) S_t.(p~_t - x) / (4 pi d^3) (eq.
 * farfield with the 1/(4 pi) of eq. pcwn); an opened leaf adds its points
 * exactly.  Sums are float with Kahan compensation.
 *
 *   queries [q,3] float; q >= 0 (q = 0 is a no-op)
 *   beta    > 0 (larger is more accurate; the paper gives no value)
 *   out     [q, channels] float (channels of the last refit)
 *
 * Queries are sorted internally along a Hilbert curve through the tree's
 * cube (cells of 2^-5 of its side), so that the 32 queries of a warp are
 * neighbours.  Reentrant: concurrent
 * forward calls on one tree are allowed.  Errors: DIPOLE_ESTATE before the
 * first refit; DIPOLE_EINVAL for null pointers or beta <= 0.
 */
int dipole_forward(const dipole_tree* tree, const float* queries, int64_t q, float beta,
                   float* out, void* stream);

/*
 * dipole_forward without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc — code that
 * runs under a fixed device-memory budget or inside a host application whose
 * own allocator owns all device memory, and loops that must not allocate
 * because cudaMalloc/cudaFree can synchronize the device or fail part way
 * through under memory pressure.  dipole_forward allocates its query-sort
 * buffers and work counter per call; this variant takes them from a
 * file-scope device array instead.
 *
 *   Same arguments, results (up to float rounding: each packet's walk runs in
 *   one piece here) and errors as dipole_forward, and additionally
 *   q <= 262144 (2^18): larger q returns DIPOLE_EINVAL with a message saying
 *   so (split the queries, or use dipole_forward).
 *
 * The array (about 4.5 MB) exists on every GPU that loads this library and
 * stays there until the process exits.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) for that device; make
 * that first call before any stream capture.  The address is kept for the
 * life of the process: after a cudaDeviceReset it is stale, and this entry
 * point must not be called again in that process.  The tree's device must be
 * the current device (else DIPOLE_EINVAL).  Every call uses the same array
 * and leaves its contents behind; the work counter is cleared at the start of
 * each call.  Calls that overlap on the GPU (different streams or threads,
 * any tree) race on the array and give wrong results: serialize them.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 */
int dipole_forward_noalloc(const dipole_tree* tree, const float* queries, int64_t q, float beta,
                           float* out, void* stream);

/*
 * Adjoint queries, two-stage (Sec. 6.2, App. C).  Given grad_out[j, c] =
 * dL/dD^c(queries[j]):
 *   stage 1 (Alg. 1, AdjointQuery; eq. farfield_gradient): the same traversal
 *     as dipole_forward adds rho(d/eps~) (p~ - x)/(4 pi d^3) g^c into dS_t^c at
 *     every far node and the exact per-point term into the points of opened
 *     leaves;
 *   stage 2 (eq. farfield_features_gradient): dL/dmu_m^c = A_m n_m . sum over
 *     the nodes holding m of dS_t^c, plus the opened-leaf terms.
 *
 *   grad_out   [q, channels] float
 *   grad_attrs [n, channels] float, caller's point order
 *   accumulate 0: overwrite grad_attrs; 1: add to it
 *
 * The result does not depend on the attributes (D is linear in mu), only on
 * the geometry and channels of the last refit.  Uses scratch owned by the
 * tree: adjoint calls on one tree must not overlap.
 */
int dipole_adjoint(dipole_tree* tree, const float* queries, int64_t q, float beta,
                   const float* grad_out, float* grad_attrs, int32_t accumulate, void* stream);

/*
 * The adjoint in its two stages as separate calls, for a data-parallel step
 * (Sec. 6.2, App. C): stage 1 is a sum over queries, so ranks holding
 * disjoint query batches can each run stage 1 into their own accumulator,
 * sum the accumulators (an all-reduce), and run stage 2 once on the sum; the
 * result equals dipole_adjoint over all the queries (up to float rounding
 * of the sums' order).
 *
 * dipole_adjoint_acc_size: *floats = entries of an accumulator for the tree's
 *   current channel count (node sums dS_t^c, then opened-leaf sums
 *   dmu_near_m^c; the layout is internal to the library and fixed between
 *   refits with the same channel count; entries are summed elementwise).
 * dipole_adjoint_stage1: Alg. 1 AdjointQuery (eq. farfield_gradient) for the
 *   given queries into acc [floats] float, device; accumulate 0 overwrites
 *   acc, 1 adds to it.  plan_perm, plan_cost: NULL, or the plan of a
 *   dipole_forward_planned on the same queries.  Does not touch the tree's
 *   own adjoint scratch: stage-1 calls with different accumulators may
 *   overlap.
 * dipole_adjoint_stage2: eq. farfield_features_gradient from acc into
 *   grad_attrs [n, channels] float (caller's point order); accumulate 0 or 1.
 * Errors: as dipole_adjoint; DIPOLE_ESTATE before the first refit.
 */
int dipole_adjoint_acc_size(const dipole_tree* tree, int64_t* floats);
int dipole_adjoint_stage1(const dipole_tree* tree, const float* queries, int64_t q, float beta,
                          const float* grad_out, float* acc, int32_t accumulate,
                          const uint32_t* plan_perm, const uint32_t* plan_cost, void* stream);
int dipole_adjoint_stage2(const dipole_tree* tree, const float* acc, float* grad_attrs,
                          int32_t accumulate, void* stream);

/*
 * Forward and adjoint sharing a query plan (caller-owned device buffers):
 *   plan_perm [q]                  uint32, written by dipole_forward_planned: the sorted
 *                                  order of the queries (a permutation of [0, q))
 *   plan_cost [8 * ceil(q / 32)]   uint32, written by dipole_forward_planned: 8 words per
 *                                  32-query packet: its traversal steps, the nodes its walk
 *                                  visited at steps 128, 256, 384 of its lower part, the node
 *                                  where the walk was split in two, and the same three for its
 *                                  upper part (0 = none)
 * dipole_forward_planned = dipole_forward that also writes the plan.  (Every forward
 *   of 65,536 queries or more walks each packet as two preorder ranges run by two
 *   warps, cut at the leaf holding the middle point of the packet's code range: a
 *   lane enters a range in the state its depth-first walk has there, which the range
 *   start's ancestors decide.)
 * dipole_adjoint_planned = dipole_adjoint that reads the plan of a forward on the
 *   same queries (the order of every training step: primal queries, then their
 *   adjoint, Sec. 6.2) instead of sorting them again; it cuts every packet's walk at
 *   the recorded nodes into preorder ranges of about 128 steps and runs the ranges
 *   longest first.  Results do not depend on the plan: any increasing sequence of
 *   cuts partitions the walk; a plan from other queries only changes the balance.  It
 *   must come from a forward with the same q (plan_perm a permutation of [0, q)),
 *   complete on `stream` or ordered before the adjoint.
 * Same arguments, results and errors as dipole_forward / dipole_adjoint otherwise.
 */
int dipole_forward_planned(const dipole_tree* tree, const float* queries, int64_t q, float beta,
                           float* out, uint32_t* plan_perm, uint32_t* plan_cost, void* stream);
int dipole_adjoint_planned(dipole_tree* tree, const float* queries, int64_t q, float beta,
                           const float* grad_out, float* grad_attrs, int32_t accumulate,
                           const uint32_t* plan_perm, const uint32_t* plan_cost, void* stream);

/*
 * Spatial gradient of the dipole sum with respect to the query position.  The
 * paper differentiates D only with respect to the point attributes (Sec. 6.2);
 * the position gradient follows from the same kernel (Sec. 4.1, eq.
 * regularized_poisson) and serves losses on the field's normal or slope.
 * With u = p - x, r = |u|, a = rho(r/eps)/r^3 and b = a'(r)/r, a point adds
 * -A mu (a n + b (n.u) u)/(4 pi); a far node (eq. farfield, v = p~ - x) adds
 * -(a S + b (S.v) v)/(4 pi).  Same walk and far decisions as dipole_forward.
 *
 *   queries [q,3] float
 *   out     [q, channels] float: D, as dipole_forward; may be NULL
 *   grad_x  [q, channels, 3] float: grad_x[j, c, k] = dD^c/dx_k at queries[j]
 *   plan_perm, plan_cost: a query plan as for dipole_forward_planned, written
 *           here; both NULL (no plan) or both set
 *
 * Channels are walked in groups of up to 4 (one traversal per group).
 * Errors: as dipole_forward; grad_x is required.
 */
int dipole_forward_grad(const dipole_tree* tree, const float* queries, int64_t q, float beta,
                        float* out, float* grad_x, uint32_t* plan_perm, uint32_t* plan_cost,
                        void* stream);

/*
 * Adjoint of dipole_forward_grad: dL/dmu for a loss of D and grad D, given
 * grad_out[j, c] = dL/dD^c and grad_grad[j, c, k] = dL/d(dD^c/dx_k) (either
 * may be NULL, not both).  Stage 1 adds, at a far node,
 *   [a g^c v - a G^c - b (v.G^c) v]/(4 pi)  to dS_t^c,
 * and at a point of an opened leaf (w = A n)
 *   [a (w.u) g^c - a (w.G^c) - b (w.u)(u.G^c)]/(4 pi)  to dmu_m^c;
 * stage 2 is that of dipole_adjoint (eq. farfield_features_gradient).
 *
 *   grad_attrs [n, channels] float, caller's point order; accumulate 0 or 1
 *   plan_perm, plan_cost: NULL, or the plan of a dipole_forward_grad on the
 *           same queries (read, as in dipole_adjoint_planned)
 *
 * With grad_grad NULL the result equals dipole_adjoint's.  Uses the tree's
 * adjoint scratch: adjoint calls on one tree must not overlap.
 */
int dipole_adjoint_grad(dipole_tree* tree, const float* queries, int64_t q, float beta,
                        const float* grad_out, const float* grad_grad, float* grad_attrs,
                        int32_t accumulate, const uint32_t* plan_perm, const uint32_t* plan_cost,
                        void* stream);

/*
 * Gradient of a loss of D with respect to the query positions (the chain
 * rule through the spatial gradient of dipole_forward_grad; the paper does not
 * differentiate in x, Sec. 6.2, but its renderer samples along rays whose
 * positions may be trained):
 *   grad_queries[j, k] (+)= sum_c grad_out[j, c] dD^c/dx_k (queries[j]).
 * Same walk and far decisions as dipole_forward_grad; the per-channel
 * gradients are summed in the kernel and never stored.
 *
 *   grad_out     [q, channels] float
 *   grad_queries [q, 3] float; accumulate 0 overwrites, 1 adds
 * Errors: as dipole_forward_grad.
 */
int dipole_adjoint_queries(const dipole_tree* tree, const float* queries, int64_t q, float beta,
                           const float* grad_out, float* grad_queries, int32_t accumulate,
                           void* stream);

/*
 * Adjoint with respect to the attributes, the normals and the radii.  The
 * paper trains the normals and the regularization eps besides the attributes
 * (Sec. 7, inverse rendering) but states the adjoint only for the attributes
 * (App. C).  Every term is linear in n_m, and a node's moment S_t^c =
 * sum A_m mu_m^c n_m, so
 *   dL/dn_m   = A_m sum_c mu_m^c sum_{t holding m} dS_t^c + opened-leaf terms
 *               A_m sum_c mu_m^c [g^c a u - a G^c - b (u.G^c) u]/(4 pi);
 * eps enters through rho(r/eps) and, at a far node, through eps~_t =
 * sum A_m eps_m / A~_t, with da/deps = -(4/sqrt(pi)) t^3 e^{-t^2}/(eps r^3)
 * and db/deps = (8/sqrt(pi)) t^5 e^{-t^2}/(eps r^5):
 *   dL/deps_m = A_m sum_{t holding m} dE_t / A~_t + opened-leaf terms,
 *   dE_t = sum_c [g^c a_e (S^c.v) - a_e (S^c.G^c) - b_e (S^c.v)(v.G^c)]/(4 pi).
 * Both are evaluated in float for t < 10 (0 beyond, where exp(-t^2)
 * underflows) and are 0 for eps = 0.  A single global eps receives
 * sum_m dL/deps_m.
 *
 *   grad_out [q, channels], grad_grad [q, channels, 3]: upstream gradients of
 *                D and grad D (either may be NULL, not both)
 *   grad_attrs [n, channels], grad_normals [n, 3], grad_radii [n] float,
 *                caller's point order; any may be NULL, not all
 *   accumulate 0 or 1, for every output given
 *   plan_perm, plan_cost: NULL, or the plan of a forward on the same queries
 *
 * Uses the tree's adjoint scratch plus n*16 + n_nodes*4 bytes allocated on
 * the first call: adjoint calls on one tree must not overlap.
 */
int dipole_adjoint_geom(dipole_tree* tree, const float* queries, int64_t q, float beta,
                        const float* grad_out, const float* grad_grad, float* grad_attrs,
                        float* grad_normals, float* grad_radii, int32_t accumulate,
                        const uint32_t* plan_perm, const uint32_t* plan_cost, void* stream);

/*
 * Primal queries on a dense grid, e.g. the 512^3 or 1024^3 evaluation grid of
 * the geometry field that the paper meshes with marching cubes (Sec. 7):
 * point (i, j, k) is lo + spacing * (i, j, k), computed in float as
 * lo[0] + ((float)i * spacing) with one rounding per operation (likewise j,
 * k), 0 <= i < dims[0], 0 <= j < dims[1], 0 <= k < dims[2].  The points are
 * generated inside the traversal kernel, 32 at a time as 4x4x2 bricks (no
 * query array and no sort), with the same far test and sums as dipole_forward.
 *
 *   lo [3], dims [3]  host arrays; 1 <= dims[d] <= 2^24, product <= 2^40
 *   spacing           > 0
 *   out               [dims[2], dims[1], dims[0], channels] float (x fastest)
 * Errors: as dipole_forward.
 */
int dipole_forward_grid(const dipole_tree* tree, const float* lo, float spacing,
                        const int64_t* dims, float beta, float* out, void* stream);

/*
 * Per-query traversal counts of Alg. 1's PrimalQuery: counts[j] = {nodes
 * tested, nodes taken as far, leaf points summed} (int32 [q,3], device).  Same
 * traversal and decisions as dipole_forward; used for the roofline's
 * algorithmic bytes and to check the traversal decisions against the oracle.
 */
int dipole_query_counts(const dipole_tree* tree, const float* queries, int64_t q, float beta,
                        int32_t* counts, void* stream);

/*
 * The traversal counts of each 32-query packet as the warp walks it (the
 * packets of the internal Hilbert-curve sort, in that order), for the
 * roofline's per-warp bytes: packet_counts[p] = {warp steps (the union of the
 * lanes' tested nodes), steps at which some lane took the node as far (the
 * warp fetches its moment row), points of leaves some lane opened (the warp
 * fetches their records), valid lanes}, int32 [ceil(q/32), 4], device.
 * counts [q, 3] as dipole_query_counts, or NULL.  Diagnostics; the paper has
 * no counterpart (packet queries are its future work, Sec. 6.3).
 */
int dipole_query_packet_counts(const dipole_tree* tree, const float* queries, int64_t q,
                               float beta, int32_t* counts, int32_t* packet_counts,
                               void* stream);

/* Synchronize `stream`, then return and clear the device status word:
 * DIPOLE_OK, DIPOLE_ETRAVERSAL or DIPOLE_ENONFINITE.  Error reporting of
 * this library; the paper has no counterpart. */
int dipole_sync_status(dipole_tree* tree, void* stream);

/* Sizes and parameters of the tree (host struct; no device work).  The
 * paper has no counterpart. */
int dipole_tree_info_get(const dipole_tree* tree, dipole_tree_info* info);

/*
 * Copy the tree to HOST arrays (synchronizes `stream`): the octree of Sec. 6.1
 * with its node aggregates (eq. farfield_dipole) and moments (eq.
 * farfield_dipole_features), for checkpoints and checks.  Any pointer may be
 * NULL.  Node arrays have n_nodes entries in preorder; point arrays n_points
 * entries in Morton order.
 *   codes, perm              uint32 [n]   sorted codes; perm[i] = caller index of point i
 *   first, count, level,     int32 [nn]   point range, octree level, parent (-1 at root),
 *   parent, skip, is_leaf                 index past the subtree, leaf flag
 *   centroid [nn,3] float, radius [nn] float, area [nn] double, eps [nn] float
 *   moments  [nn, 3*channels] float  S_t^c as (c, axis), or NULL; needs a refit
 */
int dipole_tree_export(const dipole_tree* tree, uint32_t* codes, uint32_t* perm, int32_t* first,
                       int32_t* count, int32_t* level, int32_t* parent, int32_t* skip,
                       int32_t* is_leaf, float* centroid, float* radius, double* area,
                       float* eps, float* moments, void* stream);

/*
 * Diagnostics, not part of the method (the paper has no counterpart): reads
 * `bytes` of `buf` `passes` times with L2-only loads in one kernel, so that
 * the caller can time it (a buffer smaller than L2 measures L2 read
 * bandwidth).  buf 16-byte aligned, bytes a positive multiple of 16; sink is
 * a device float array of 1024 * (multiprocessor count) entries that receives
 * one value per thread.  Asynchronous on `stream`.
 */
int dipole_probe_l2(const void* buf, int64_t bytes, int32_t passes, float* sink, void* stream);

/*
 * Rebuild a tree from an export (checkpoint / resume): the point inputs as for
 * dipole_build_tree (DEVICE, caller order) and the topology arrays written by
 * dipole_tree_export (HOST): perm [n], first/count/level/skip/is_leaf
 * [n_nodes], codes [n] (informational, may be NULL).  No sorting and no
 * topology construction: the node geometry (eq. farfield_dipole) and node
 * records are recomputed from the given ranges, so an export of the result
 * equals the original export.  Synchronizes `stream` once.
 *
 * Validation (host, before any device work): perm is a permutation of
 * [0, n); for every node 0 <= first < n, 1 <= count <= n - first,
 * 0 <= level <= max_depth, 0 <= skip <= n_nodes, is_leaf in {0, 1}; else
 * DIPOLE_EINVAL.  Every index a kernel follows is therefore in range.  The
 * structure (nesting, preorder) is not checked: queries on a corrupt
 * structure stop at their step bound and dipole_sync_status() reports
 * DIPOLE_ETRAVERSAL.
 */
int dipole_tree_import(const float* points, const float* normals, const float* areas,
                       const float* radii, int64_t n, const uint32_t* codes, const uint32_t* perm,
                       const int32_t* first, const int32_t* count, const int32_t* level,
                       const int32_t* skip, const int32_t* is_leaf, int64_t n_nodes,
                       const dipole_build_params* params, void* stream, dipole_tree** out);

/* Release the tree and its device memory (synchronizes the device).  NULL is
 * a no-op.  Resource management; the paper has no counterpart. */
void dipole_tree_destroy(dipole_tree* tree);

/* Message of the last failed call on this thread ("" if none); owned by the
 * library, valid until the next failed call on this thread.  The paper has no
 * counterpart. */
const char* dipole_last_error(void);

/* Number of CUDA kernels this library has launched in this process (all
 * threads, all trees).  Host counter, no device work; for accounting.  The
 * paper has no counterpart. */
uint64_t dipole_kernel_launches(void);

/* Number of device allocations this library has made in this process (all
 * threads, all trees): every one is a stream-ordered cudaMallocAsync from the
 * device's default memory pool.  Host counter, no device work; lets a caller
 * (or a test) check that a call allocates nothing.  The paper has no
 * counterpart. */
uint64_t dipole_device_allocations(void);

/*
 * 1 in the checked build of the library (compiled with -DDIPOLE_CHECKED: the
 * traversals test every index they read from an array before using it and
 * report DIPOLE_EBOUNDS), 0 in the normal build.  A testing aid with no
 * counterpart in the paper.
 */
int dipole_checked_build(void);

/*
 * Treelet: with enable = 1, the value forward (dipole_forward, the planned and
 * grid forms; not the no-allocation form) of trees with up to 4 channels and
 * float moments stages the upper tree — the nodes of depth < 3 (at most 73),
 * their records and their first moment chunk — in each block's shared memory
 * by one bulk copy (cp.async.bulk, no multicast) and reads those nodes from
 * there (Alg. 1 PrimalQuery, the nodes every walk visits first).  Results are
 * bit-identical with and without it.  The first forward after enabling
 * allocates a block of 32 bytes per node plus 8 KB for the tree (freed with
 * it); every forward rewrites the staged records, so forwards of one tree that
 * overlap on the GPU race on them.  Measured 2% slower than without it on the
 * 1M-point workload (the walk is issue bound; the nodes staged are L1 hits
 * anyway), so it is off by default.  enable = 0 turns it off.
 * Errors: DIPOLE_EINVAL for a NULL tree or enable not 0 or 1.
 */
int dipole_set_treelet(dipole_tree* tree, int32_t enable);

/* Query modes of the traversal timer below. */
typedef enum {
    DIPOLE_TIMER_FORWARD = 0,       /* dipole_forward*, dipole_forward_grid */
    DIPOLE_TIMER_ADJOINT = 1,       /* dipole_adjoint*, dipole_adjoint_stage1 (stage 1) */
    DIPOLE_TIMER_COUNTS = 2,        /* dipole_query_counts, dipole_query_packet_counts */
    DIPOLE_TIMER_FORWARD_GRAD = 3,  /* dipole_forward_grad */
    DIPOLE_TIMER_ADJOINT_GRAD = 4,  /* dipole_adjoint_grad (stage 1) */
    DIPOLE_TIMER_ADJOINT_GEOM = 5,  /* dipole_adjoint_geom (stage 1) */
    DIPOLE_TIMER_QUERY_GRAD = 6     /* dipole_adjoint_queries */
} dipole_timer_mode;
/*
 * Timing of the traversal kernels, for the roofline of the dominant kernel
 * (diagnostics; the paper has no counterpart).  dipole_traversal_timer(1)
 * makes every later query call record a CUDA event pair on its stream
 * directly before and after its traversal kernel (query sort, work-item
 * setup and stage 2 are outside the pair); dipole_traversal_timer(0) stops
 * it.  dipole_traversal_elapsed(mode, &ms, &launches) waits for the recorded
 * events of that mode, returns their summed elapsed time and count, and
 * forgets them.  mode: a dipole_timer_mode.  Costs two event records per call
 * while enabled; off by default.
 */
int dipole_traversal_timer(int32_t enable);
int dipole_traversal_elapsed(int32_t mode, float* total_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* DIPOLE_H */
