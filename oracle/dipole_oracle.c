/*
 * Oracle for the regularized dipole sum and its Barnes-Hut evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, double-precision CPU
 * statement of what the GPU library computes.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it; the product path never
 * does.  It shares no code, header or constant table with the CUDA library.
 *
 * Paper: Chen, Miller, Gkioulekas, "3D Reconstruction with Fast Dipole Sums"
 * (arXiv 2405.16788).  Citations name the paper's sections and equations.
 *
 *   rho, P_eps          Sec. 4.1, eq. (regularized_poisson) and eq. (pcwn)
 *   dipole sum          Sec. 4.2, eq. (dipole_sum); multi-channel: eq. (appearance_features)
 *   node aggregates     Sec. 6.1, eqs. (farfield_dipole), (farfield_dipole_features)
 *   far field           Sec. 6.1, eq. (farfield)
 *   primal query        Alg. 1, PrimalQuery
 *   adjoint, stage 1    Alg. 1, AdjointQuery; App. C, eq. (farfield_gradient)
 *   adjoint, stage 2    Sec. 6.2 (two-stage scheme); App. C, eq. (farfield_features_gradient)
 *
 * Readings of the paper that this file takes where the paper is silent or
 * ambiguous (the tests and the CUDA library follow the same readings):
 *   R1  The 1/(4 pi) of eq. (pcwn) is kept in the far field, in GetContribution
 *       and in IncrementGradient (the printed forms drop it).
 *   R2  rho(t) = erf(t) - 2t/sqrt(pi) exp(-t^2) with t = r/eps, as printed.
 *       eps = 0 means rho = 1 (the singular kernel).  A term with r = 0 is 0.
 *   R3  Leaves hold up to leaf_size points (single points in the paper); an
 *       opened leaf sums its points exactly.  The far test comes first, then
 *       the leaf test, as in Alg. 1.
 *   R4  The octree is the compressed 30-bit Morton octree specified below.
 *   R5  Per-point eps_m: a node uses the area-weighted mean eps of its points.
 *   R6  The far test is evaluated in single precision on single-precision node
 *       geometry with the fixed operation order below, so that a CPU and a GPU
 *       implementation take identical decisions.  All values are double.
 *   R7  Node sums (area, area-weighted position, area-weighted eps) are formed
 *       in float inside a leaf, point by point in Morton order with every
 *       product and sum rounded to float, and in double inside an internal
 *       node, child by child in Morton order from its children's sums.  The ratios are taken as the sums
 *       times the correctly rounded reciprocal of the area; the node centroid
 *       is that product rounded to float; the node radius is the largest float
 *       distance from that float centroid to a point of the node.
 *   R8  AS(m) in eq. (farfield_features_gradient) includes the leaf holding m.
 *   R9  Spatial gradient (the paper needs grad D for eq. surface_density and
 *       the implicit normal of Sec. 5.1 but does not say how it is computed):
 *       the gradient in x of each term, with u = p - x, r = |u|, t = r/eps,
 *       is -A/(4 pi) [a n + b (n.u) u], a = rho/r^3,
 *       b = rho'(t)/(eps r^4) - 3 rho/r^5, rho'(t) = (4/sqrt(pi)) t^2 exp(-t^2);
 *       a far node uses the same with n -> n~^c, p -> p~, eps -> eps~, A -> A~.
 *       A zero-distance term contributes nothing to D or to grad D.
 *   R10 Gradients with respect to the normals and the regularization radii
 *       (the paper trains normals and eps but states the adjoint only for
 *       the attributes, App. C).  A point term is linear in n_m: d/dn_m of
 *       A mu a (n.u)/(4 pi) is A mu a u/(4 pi), and of its x-gradient
 *       -A mu (a I + b u u^T)/(4 pi).  A far node's n~_t^c depends on n_m
 *       through A_m mu_m^c/A~_t (eq. farfield_dipole_features), so n_m
 *       receives (A_m mu_m^c/A~_t) dn~_t^c from every node t holding it (the
 *       stage-1 sums of eq. farfield_features_gradient).  With t = r/eps,
 *       da/deps = -(4/sqrt(pi)) t^3 exp(-t^2)/(eps r^3) and
 *       db/deps = (8/sqrt(pi)) t^5 exp(-t^2)/(eps r^5); a far node depends on
 *       eps_m through eps~_t (R5), d eps~_t/d eps_m = A_m/A~_t, with one
 *       scalar stage-1 sum d eps~_t per node.  eps = 0 has zero eps-gradient.
 *       The paper's single global eps receives the sum over m.
 *   R11 Desingularized kernel (the ablation baseline of Sec. 4.1, footnote,
 *       and Sec. 7, which bounds the Poisson kernel's denominator from below):
 *       1/r^3 -> 1/max(r, eps)^3 with the point's radius as the cutoff, eps~
 *       at a far node; written as rho_d(r, eps) = min(1, (r/eps)^3) in place
 *       of rho so that every formula above applies: a = 1/max(r, eps)^3,
 *       b = -3/r^5 outside the cutoff and 0 inside, da/deps = -3/eps^4 inside
 *       and 0 outside, db/deps = 0.  Selected by orc_set_kernel(1).
 *   R12 Appearance channels without the foreshortening term (Sec. 5.3,
 *       radiance field details: the paper skips it for its appearance
 *       attributes in eq. appearance_features and says no more).  The
 *       foreshortening term is the cosine n.(p - x)/|p - x| of the kernel
 *       A rho(r/eps) n.(p - x)/(4 pi r^3); without it a point contributes
 *       A rho(r/eps)/(4 pi r^2) mu.  Channels [0, G) keep the term, channels
 *       [G, C) skip it (G = C unless set).  A far node contributes, in the
 *       order of eq. farfield, A~_t rho(d/eps~_t)/(4 pi d^2) m~_t^c with
 *       m~_t^c = sum_{m in t} A_m mu_m^c / A~_t (the area-weighted mean
 *       attribute, the counterpart of n~_t^c), and stage 2 of the adjoint
 *       gives d mu_m^c = sum_{t in AS(m)} (A_m / A~_t) d m~_t^c.
 *   R13 bf16 node moments (an option of the storage, not in the paper): the
 *       far field of PrimalQuery uses the node sums A~_t n~_t^c (and A~_t m~_t^c
 *       for R12 channels) rounded to float and then to bfloat16, each rounding
 *       to nearest with ties to even; every other query keeps the double
 *       moments.  Set by orc_tree_round_moments_bf16 after an update.  Where
 *       a node sum lies so close to a rounding boundary of bf16 that an
 *       implementation summing the same values in float (every product and
 *       partial sum rounded) could round it the other way, both results are
 *       correct: such a sum S is one whose interval S -+ delta, delta =
 *       2^-19 sum |A n mu| + 2^-22 |S| over the node's points, holds a
 *       boundary, and the forward reports per query and channel the largest
 *       change such choices can make, sum |v_k| (round(S+delta) - round(S-delta))
 *       over the far nodes' moments (orc_bh_forward_bf16).
 * Compile with -ffp-contract=off: the Morton quantisation, the far test and
 * the radius are specified operation by operation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_MAX_LEVEL 10 /* 30-bit codes: 10 octal digits */

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Kernel (Sec. 4.1)                                                          */
/* ------------------------------------------------------------------------ */

/* rho(t) = erf(t) - (2 t / sqrt(pi)) exp(-t^2): the regularizing factor of
 * eq. (regularized_poisson).  t = +inf gives 1. */
double orc_rho(double t) {
    if (isinf(t)) return 1.0;
    return erf(t) - 2.0 * t / sqrt(ORC_PI) * exp(-t * t);
}

/* Kernel of the queries: 0 the regularized kernel of the paper, 1 the
 * desingularized kernel of R11. */
static int g_kernel = 0;

void orc_set_kernel(int kernel) { g_kernel = kernel; }

/* rho(r / eps), with eps = 0 meaning the singular kernel (R2); for the
 * desingularized kernel min(1, (r/eps)^3) (R11). */
static double rho_r(double r, double eps) {
    if (eps == 0.0) return 1.0;
    if (g_kernel == 1) {
        double q = r / eps;
        return q >= 1.0 ? 1.0 : q * q * q;
    }
    return orc_rho(r / eps);
}

/* A * P_eps(x, p) : area times the regularized Poisson kernel, eq. (pcwn) with
 * the factor of eq. (regularized_poisson).  Returns 0 when x == p (R2). */
static double point_weight(const double x[3], double px, double py, double pz,
                           double nx, double ny, double nz, double A, double eps) {
    double dx = px - x[0], dy = py - x[1], dz = pz - x[2];
    double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return 0.0;
    double r = sqrt(r2);
    return A * rho_r(r, eps) * (nx * dx + ny * dy + nz * dz) / (4.0 * ORC_PI * r2 * r);
}

/* a = rho/r^3 and b = rho'(t)/(eps r^4) - 3 rho/r^5 of reading R9 (r > 0). */
static void grad_factors(double r, double eps, double* a, double* b) {
    double r3 = r * r * r;
    if (eps == 0.0) {
        *a = 1.0 / r3;
        *b = -3.0 / (r3 * r * r);
        return;
    }
    double t = r / eps;
    if (g_kernel == 1) { /* R11: 1/max(r, eps)^3 */
        if (t >= 1.0) {
            *a = 1.0 / r3;
            *b = -3.0 / (r3 * r * r);
        } else {
            *a = 1.0 / (eps * eps * eps);
            *b = 0.0;
        }
        return;
    }
    double rho = orc_rho(t);
    double drho = 4.0 / sqrt(ORC_PI) * t * t * exp(-t * t);
    *a = rho / r3;
    *b = drho / (eps * r3 * r) - 3.0 * rho / (r3 * r * r);
}

/* da/deps and db/deps of reading R10 (r > 0); both 0 for eps = 0. */
static void eps_factors(double r, double eps, double* da, double* db) {
    if (eps == 0.0) {
        *da = 0.0;
        *db = 0.0;
        return;
    }
    if (g_kernel == 1) { /* R11 */
        *da = r < eps ? -3.0 / (eps * eps * eps * eps) : 0.0;
        *db = 0.0;
        return;
    }
    double t = r / eps, e = exp(-t * t), r3 = r * r * r, c = 4.0 / sqrt(ORC_PI);
    *da = -c * t * t * t * e / (eps * r3);
    *db = 2.0 * c * t * t * t * t * t * e / (eps * r3 * r * r);
}

/* Gradient in x of A P_eps(x, p): -A/(4 pi) [a n + b (n.u) u], u = p - x (R9).
 * g receives 3 values; zero when x == p. */
static void point_grad(const double x[3], double px, double py, double pz, double nx,
                       double ny, double nz, double A, double eps, double g[3]) {
    double ux = px - x[0], uy = py - x[1], uz = pz - x[2];
    double r2 = ux * ux + uy * uy + uz * uz;
    g[0] = g[1] = g[2] = 0.0;
    if (r2 == 0.0) return;
    double a, b;
    grad_factors(sqrt(r2), eps, &a, &b);
    double nu = nx * ux + ny * uy + nz * uz;
    double f = -A / (4.0 * ORC_PI);
    g[0] = f * (a * nx + b * nu * ux);
    g[1] = f * (a * ny + b * nu * uy);
    g[2] = f * (a * nz + b * nu * uz);
}

/* ------------------------------------------------------------------------ */
/* Brute force: the plain definition, eq. (dipole_sum) / (appearance_features) */
/* ------------------------------------------------------------------------ */

/* out[j*C + c] = sum_m A_m P_eps_m(x_j, p_m) mu[m*C + c].
 * pts, nrm: [n,3]; area, eps: [n] (eps may be NULL: all zero); mu: [n,C]. */
/* A rho(r/eps) / (4 pi r^2): the kernel without its foreshortening cosine
 * (R12).  Returns 0 when x == p (R2). */
static double point_weight_nf(const double x[3], double px, double py, double pz, double A,
                              double eps) {
    double dx = px - x[0], dy = py - x[1], dz = pz - x[2];
    double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return 0.0;
    return A * rho_r(sqrt(r2), eps) / (4.0 * ORC_PI * r2);
}

/* The plain definition with channels [G, C) without the foreshortening term
 * (R12): out[j*C + c] = sum_m w_c(x_j, m) mu_m^c. */
void orc_brute_forward_app(int64_t n, const float* pts, const float* nrm, const float* area,
                           const float* eps, int C, int G, const float* mu, int64_t q,
                           const float* qry, double* out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < q; ++j) {
        double x[3] = {qry[3 * j], qry[3 * j + 1], qry[3 * j + 2]};
        double* o = out + j * C;
        for (int c = 0; c < C; ++c) o[c] = 0.0;
        for (int64_t m = 0; m < n; ++m) {
            double e = eps ? (double)eps[m] : 0.0;
            double w = point_weight(x, pts[3 * m], pts[3 * m + 1], pts[3 * m + 2], nrm[3 * m],
                                    nrm[3 * m + 1], nrm[3 * m + 2], area[m], e);
            double wf = point_weight_nf(x, pts[3 * m], pts[3 * m + 1], pts[3 * m + 2], area[m], e);
            for (int c = 0; c < C; ++c) o[c] += (c < G ? w : wf) * (double)mu[m * C + c];
        }
    }
}

/* Its transpose: grad[m*C + c] = sum_j g[j*C + c] w_c(x_j, m). */
void orc_brute_adjoint_app(int64_t n, const float* pts, const float* nrm, const float* area,
                           const float* eps, int C, int G, int64_t q, const float* qry,
                           const double* g, double* grad) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t m = 0; m < n; ++m) {
        double* gm = grad + m * C;
        for (int c = 0; c < C; ++c) gm[c] = 0.0;
        double e = eps ? (double)eps[m] : 0.0;
        for (int64_t j = 0; j < q; ++j) {
            double x[3] = {qry[3 * j], qry[3 * j + 1], qry[3 * j + 2]};
            double w = point_weight(x, pts[3 * m], pts[3 * m + 1], pts[3 * m + 2], nrm[3 * m],
                                    nrm[3 * m + 1], nrm[3 * m + 2], area[m], e);
            double wf = point_weight_nf(x, pts[3 * m], pts[3 * m + 1], pts[3 * m + 2], area[m], e);
            for (int c = 0; c < C; ++c) gm[c] += (c < G ? w : wf) * g[j * C + c];
        }
    }
}

void orc_brute_forward(int64_t n, const float* pts, const float* nrm, const float* area,
                       const float* eps, int C, const float* mu, int64_t q,
                       const float* qry, double* out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < q; ++j) {
        double x[3] = {qry[3 * j], qry[3 * j + 1], qry[3 * j + 2]};
        double* o = out + j * C;
        for (int c = 0; c < C; ++c) o[c] = 0.0;
        for (int64_t m = 0; m < n; ++m) {
            double w = point_weight(x, pts[3 * m], pts[3 * m + 1], pts[3 * m + 2], nrm[3 * m],
                                    nrm[3 * m + 1], nrm[3 * m + 2], area[m],
                                    eps ? (double)eps[m] : 0.0);
            for (int c = 0; c < C; ++c) o[c] += w * (double)mu[m * C + c];
        }
    }
}

/* Spatial gradient of the dipole sum: grad[(j*C + c)*3 + k] = d D^c / d x_k at
 * x_j (R9), the plain definition. */
void orc_brute_forward_grad(int64_t n, const float* pts, const float* nrm, const float* area,
                            const float* eps, int C, const float* mu, int64_t q,
                            const float* qry, double* grad) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < q; ++j) {
        double x[3] = {qry[3 * j], qry[3 * j + 1], qry[3 * j + 2]};
        double* o = grad + j * C * 3;
        for (int k = 0; k < 3 * C; ++k) o[k] = 0.0;
        for (int64_t m = 0; m < n; ++m) {
            double g[3];
            point_grad(x, pts[3 * m], pts[3 * m + 1], pts[3 * m + 2], nrm[3 * m], nrm[3 * m + 1],
                       nrm[3 * m + 2], area[m], eps ? (double)eps[m] : 0.0, g);
            for (int c = 0; c < C; ++c)
                for (int k = 0; k < 3; ++k) o[3 * c + k] += g[k] * (double)mu[m * C + c];
        }
    }
}

/* Gradient of L with respect to mu when dL/dD(x_j) = g[j*C + c]:
 * grad[m*C + c] = sum_j g[j*C + c] A_m P_eps_m(x_j, p_m).  D is linear in mu. */
void orc_brute_adjoint(int64_t n, const float* pts, const float* nrm, const float* area,
                       const float* eps, int C, int64_t q, const float* qry, const double* g,
                       double* grad) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t m = 0; m < n; ++m) {
        double* gm = grad + m * C;
        for (int c = 0; c < C; ++c) gm[c] = 0.0;
        for (int64_t j = 0; j < q; ++j) {
            double x[3] = {qry[3 * j], qry[3 * j + 1], qry[3 * j + 2]};
            double w = point_weight(x, pts[3 * m], pts[3 * m + 1], pts[3 * m + 2], nrm[3 * m],
                                    nrm[3 * m + 1], nrm[3 * m + 2], area[m],
                                    eps ? (double)eps[m] : 0.0);
            for (int c = 0; c < C; ++c) gm[c] += w * g[j * C + c];
        }
    }
}

/* One point's contributions to the gradients of L with respect to mu_m, n_m
 * and eps_m (R9, R10), for the upstream gradients gv[c] = dL/dD^c and
 * gg[3c + k] = dL/d(dD^c/dx_k) at x (either may be NULL), u = p - x:
 *   dmu^c += A/(4 pi) [g^c a (n.u) - a (n.G^c) - b (n.u)(u.G^c)]
 *   dn    += A/(4 pi) sum_c mu^c [g^c a u - a G^c - b (u.G^c) u]
 *   deps  += A/(4 pi) sum_c mu^c [g^c a_e (n.u) - a_e (n.G^c) - b_e (n.u)(u.G^c)]
 * with a_e = da/deps, b_e = db/deps.  Nothing for x == p. */
static void point_geom_terms(const double x[3], const float* p, const float* nrm, double A,
                             double eps, int C, const double* mu, const double* gv,
                             const double* gg, double* dmu, double* dn, double* deps) {
    double ux = p[0] - x[0], uy = p[1] - x[1], uz = p[2] - x[2];
    double r2 = ux * ux + uy * uy + uz * uz;
    if (r2 == 0.0) return;
    double r = sqrt(r2), a, b, ae, be;
    grad_factors(r, eps, &a, &b);
    eps_factors(r, eps, &ae, &be);
    double nx = nrm[0], ny = nrm[1], nz = nrm[2];
    double nu = nx * ux + ny * uy + nz * uz;
    double f = A / (4.0 * ORC_PI);
    for (int c = 0; c < C; ++c) {
        double g = gv ? gv[c] : 0.0;
        double G0 = gg ? gg[3 * c] : 0.0, G1 = gg ? gg[3 * c + 1] : 0.0, G2 = gg ? gg[3 * c + 2] : 0.0;
        double nG = nx * G0 + ny * G1 + nz * G2, uG = ux * G0 + uy * G1 + uz * G2;
        dmu[c] += f * (g * a * nu - a * nG - b * nu * uG);
        double mc = mu[c];
        dn[0] += f * mc * (g * a * ux - a * G0 - b * uG * ux);
        dn[1] += f * mc * (g * a * uy - a * G1 - b * uG * uy);
        dn[2] += f * mc * (g * a * uz - a * G2 - b * uG * uz);
        *deps += f * mc * (g * ae * nu - ae * nG - be * nu * uG);
    }
}

/* Plain definition of dL/dmu [n,C], dL/dn [n,3] and dL/deps [n] (R9, R10) for
 * dL/dD = g [q,C] and dL/d(grad D) = gg [q,C,3] (either may be NULL); sums of
 * point_geom_terms over all queries.  Outputs may be NULL. */
void orc_brute_adjoint_geom(int64_t n, const float* pts, const float* nrm, const float* area,
                            const float* eps, int C, const float* mu, int64_t q,
                            const float* qry, const double* g, const double* gg, double* dmu,
                            double* dn, double* deps) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t m = 0; m < n; ++m) {
        double* mu_m = (double*)malloc(sizeof(double) * C);
        double* dm = (double*)calloc((size_t)C, sizeof(double));
        double dv[3] = {0.0, 0.0, 0.0}, de = 0.0;
        for (int c = 0; c < C; ++c) mu_m[c] = mu[m * C + c];
        for (int64_t j = 0; j < q; ++j) {
            double x[3] = {qry[3 * j], qry[3 * j + 1], qry[3 * j + 2]};
            point_geom_terms(x, pts + 3 * m, nrm + 3 * m, area[m], eps ? (double)eps[m] : 0.0, C,
                             mu_m, g ? g + j * C : NULL, gg ? gg + j * 3 * C : NULL, dm, dv, &de);
        }
        if (dmu)
            for (int c = 0; c < C; ++c) dmu[m * C + c] = dm[c];
        if (dn)
            for (int k = 0; k < 3; ++k) dn[3 * m + k] = dv[k];
        if (deps) deps[m] = de;
        free(mu_m);
        free(dm);
    }
}

/* ------------------------------------------------------------------------ */
/* Octree (R4), Sec. 6.1 and Sec. 6.3 "tree construction"                     */
/* ------------------------------------------------------------------------ */
/*
 * Bounding cube: lo = per-axis float minimum; ext = largest per-axis
 * (max - min), computed in float; ext = 1 when it is 0.
 * Quantisation: s = 1024 / ext (float division); per axis
 *   q = min(1023, floor((p - lo) * s)) with the subtraction and the product
 *   rounded to float one at a time.
 * Code: bit k of qx goes to bit 3k+2, of qy to 3k+1, of qz to 3k.
 * Order: by (code, original index).
 * A node at level l is a maximal run of sorted codes sharing their top 3l
 * bits.  A run with at most leaf_size points, or at level max_depth, is a
 * leaf.  Otherwise its children are the runs at level l+1 inside it, in code
 * order; when there is only one, the node is that child (chains collapse).
 * Nodes are stored in depth-first preorder; skip[t] is the index just past
 * t's subtree.
 */

static uint32_t spread10(uint32_t v) {
    uint32_t r = 0;
    for (int k = 0; k < 10; ++k) r |= ((v >> k) & 1u) << (3 * k);
    return r;
}

uint32_t orc_interleave(uint32_t qx, uint32_t qy, uint32_t qz) {
    return (spread10(qx) << 2) | (spread10(qy) << 1) | spread10(qz);
}

/* Bounding cube and 30-bit codes in input order. lo_ext: out[4] = lo.xyz, ext. */
void orc_morton(int64_t n, const float* pts, float* lo_ext, uint32_t* codes) {
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = pts[a]; hi[a] = pts[a]; }
    for (int64_t m = 1; m < n; ++m)
        for (int a = 0; a < 3; ++a) {
            float v = pts[3 * m + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    float ext = 0.0f;
    for (int a = 0; a < 3; ++a) {
        float e = hi[a] - lo[a];
        if (e > ext) ext = e;
    }
    if (!(ext > 0.0f)) ext = 1.0f;
    float s = 1024.0f / ext;
    for (int64_t m = 0; m < n; ++m) {
        uint32_t qv[3];
        for (int a = 0; a < 3; ++a) {
            float d = pts[3 * m + a] - lo[a];
            float t = d * s;
            float f = floorf(t);
            uint32_t qa = (uint32_t)f;
            qv[a] = qa > 1023u ? 1023u : qa;
        }
        codes[m] = orc_interleave(qv[0], qv[1], qv[2]);
    }
    lo_ext[0] = lo[0]; lo_ext[1] = lo[1]; lo_ext[2] = lo[2]; lo_ext[3] = ext;
}

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

typedef struct orc_tree {
    int64_t n, nn, cap;
    int leaf_size, max_depth;
    float lo_ext[4];
    uint32_t* code;  /* [n] sorted */
    uint32_t* perm;  /* [n] sorted position -> input index */
    float* p;        /* [n,3] sorted positions */
    float* nrm;      /* [n,3] sorted normals */
    float* A;        /* [n] sorted areas */
    float* eps;      /* [n] sorted regularization radii */
    int32_t *first, *count, *level, *parent, *skip, *is_leaf; /* [nn] */
    int32_t* leaf_of; /* [n] sorted position -> leaf node */
    double* area;     /* [nn]  A~_t */
    double* cen;      /* [nn,3] p~_t (double) */
    double* epsn;     /* [nn]  eps~_t */
    float* cen32;     /* [nn,3] p~_t rounded to float (far test, R6/R7) */
    float* r32;       /* [nn]  r~_t (R7) */
    int C;
    double* mu;       /* [n,C] sorted attributes */
    double* nt;       /* [nn,3C] n~_t^c, eq. (farfield_dipole_features) */
    int G;            /* channels [0, G) with the foreshortening term, [G, C) without (R12) */
    double* mt;       /* [nn,C] m~_t^c = sum A mu / A~ (R12) */
    double* s16;      /* [nn,3C] A~ n~ rounded to bf16 (R13), or NULL */
    double* m16;      /* [nn,C] A~ m~ rounded to bf16 (R13), or NULL */
    double* a16;      /* [nn,3C] width of s16's rounding ambiguity (R13), often 0 */
    double* am16;     /* [nn,C] the same for m16 */
    double *s_area, *s_ap, *s_ae; /* [nn], [nn,3], [nn] double node sums (R7) */
} orc_tree;

static int32_t emit(orc_tree* T, int64_t a, int64_t cnt, int level, int32_t parent, int leaf) {
    int64_t i = T->nn++;
    T->first[i] = (int32_t)a;
    T->count[i] = (int32_t)cnt;
    T->level[i] = level;
    T->parent[i] = parent;
    T->is_leaf[i] = leaf;
    T->skip[i] = (int32_t)(i + 1);
    return (int32_t)i;
}

static void build_node(orc_tree* T, int64_t a, int64_t b, int level, int32_t parent) {
    int64_t cnt = b - a;
    if (cnt <= T->leaf_size || level >= T->max_depth) {
        int32_t t = emit(T, a, cnt, level, parent, 1);
        for (int64_t m = a; m < b; ++m) T->leaf_of[m] = t;
        return;
    }
    int shift = 3 * (ORC_MAX_LEVEL - 1 - level);
    uint32_t d0 = (T->code[a] >> shift) & 7u, d1 = (T->code[b - 1] >> shift) & 7u;
    if (d0 == d1) { /* one child: the node is that child */
        build_node(T, a, b, level + 1, parent);
        return;
    }
    int32_t t = emit(T, a, cnt, level, parent, 0);
    int64_t s = a;
    while (s < b) {
        uint32_t d = (T->code[s] >> shift) & 7u;
        int64_t e = s + 1;
        while (e < b && ((T->code[e] >> shift) & 7u) == d) ++e;
        build_node(T, s, e, level + 1, t);
        s = e;
    }
    T->skip[t] = (int32_t)T->nn;
}

/* Children of internal node t in order: t+1, skip[t+1], ... while < skip[t]. */

/* Node sums in the order of R7, then centroid, mean eps, float centroid. */
static void node_sums(orc_tree* T, int32_t t) {
    double sa = 0.0, sx = 0.0, sy = 0.0, sz = 0.0, se = 0.0;
    if (T->is_leaf[t]) {
        /* R7: float sums inside a leaf (no fused multiply-add: -ffp-contract=off) */
        float fa = 0.0f, fx = 0.0f, fy = 0.0f, fz = 0.0f, fe = 0.0f;
        for (int64_t m = T->first[t]; m < (int64_t)T->first[t] + T->count[t]; ++m) {
            float A = T->A[m];
            fa = fa + A;
            fx = fx + A * T->p[3 * m];
            fy = fy + A * T->p[3 * m + 1];
            fz = fz + A * T->p[3 * m + 2];
            fe = fe + A * T->eps[m];
        }
        sa = fa; sx = fx; sy = fy; sz = fz; se = fe;
    } else {
        for (int32_t c = t + 1; c < T->skip[t]; c = T->skip[c]) {
            node_sums(T, c);
            sa += T->s_area[c];
            sx += T->s_ap[3 * c];
            sy += T->s_ap[3 * c + 1];
            sz += T->s_ap[3 * c + 2];
            se += T->s_ae[c];
        }
    }
    T->s_area[t] = sa;
    T->s_ap[3 * t] = sx; T->s_ap[3 * t + 1] = sy; T->s_ap[3 * t + 2] = sz;
    T->s_ae[t] = se;
    /* eq. (farfield_dipole): A~ = sum A; p~ = sum A p / A~, as (sum A p) * (1/A~) (R7) */
    T->area[t] = sa;
    double rs = 1.0 / sa;
    T->cen[3 * t] = sx * rs; T->cen[3 * t + 1] = sy * rs; T->cen[3 * t + 2] = sz * rs;
    T->epsn[t] = se * rs; /* R5 */
    for (int a = 0; a < 3; ++a) T->cen32[3 * t + a] = (float)T->cen[3 * t + a];
    /* r~ = max_m |p_m - p~| over the node's points, in float (R7) */
    float r = 0.0f;
    for (int64_t m = T->first[t]; m < (int64_t)T->first[t] + T->count[t]; ++m) {
        float ex = T->p[3 * m] - T->cen32[3 * t];
        float ey = T->p[3 * m + 1] - T->cen32[3 * t + 1];
        float ez = T->p[3 * m + 2] - T->cen32[3 * t + 2];
        float d2 = fmaf(ez, ez, fmaf(ey, ey, ex * ex));
        float d = sqrtf(d2);
        if (d > r) r = d;
    }
    T->r32[t] = r;
}

void orc_tree_free(orc_tree* T) {
    if (!T) return;
    free(T->code); free(T->perm); free(T->p); free(T->nrm); free(T->A); free(T->eps);
    free(T->first); free(T->count); free(T->level); free(T->parent); free(T->skip);
    free(T->is_leaf); free(T->leaf_of); free(T->area); free(T->cen); free(T->epsn);
    free(T->cen32); free(T->r32); free(T->mu); free(T->nt); free(T->mt);
    free(T->s16); free(T->m16); free(T->a16); free(T->am16);
    free(T->s_area); free(T->s_ap); free(T->s_ae);
    free(T);
}

/* Build the octree over n points (input order).  eps may be NULL (all zero).
 * Returns NULL on bad arguments: n < 1, leaf_size < 1, max_depth outside
 * [0, 10], or a non-positive area (R: areas must be > 0 for p~ to exist). */
orc_tree* orc_tree_build(int64_t n, const float* pts, const float* nrm, const float* area,
                         const float* eps, int leaf_size, int max_depth) {
    if (n < 1 || leaf_size < 1 || max_depth < 0 || max_depth > ORC_MAX_LEVEL) return NULL;
    for (int64_t m = 0; m < n; ++m)
        if (!(area[m] > 0.0f)) return NULL;
    orc_tree* T = (orc_tree*)calloc(1, sizeof(orc_tree));
    T->n = n;
    T->cap = 2 * n + 1;
    T->leaf_size = leaf_size;
    T->max_depth = max_depth;
    uint32_t* codes_in = (uint32_t*)malloc(sizeof(uint32_t) * n);
    orc_morton(n, pts, T->lo_ext, codes_in);
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * n);
    for (int64_t m = 0; m < n; ++m) key[m] = ((uint64_t)codes_in[m] << 32) | (uint64_t)m;
    qsort(key, (size_t)n, sizeof(uint64_t), cmp_u64);
    T->code = (uint32_t*)malloc(sizeof(uint32_t) * n);
    T->perm = (uint32_t*)malloc(sizeof(uint32_t) * n);
    T->p = (float*)malloc(sizeof(float) * 3 * n);
    T->nrm = (float*)malloc(sizeof(float) * 3 * n);
    T->A = (float*)malloc(sizeof(float) * n);
    T->eps = (float*)malloc(sizeof(float) * n);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t m = (uint32_t)(key[i] & 0xffffffffu);
        T->code[i] = (uint32_t)(key[i] >> 32);
        T->perm[i] = m;
        for (int a = 0; a < 3; ++a) {
            T->p[3 * i + a] = pts[3 * (int64_t)m + a];
            T->nrm[3 * i + a] = nrm[3 * (int64_t)m + a];
        }
        T->A[i] = area[m];
        T->eps[i] = eps ? eps[m] : 0.0f;
    }
    free(key);
    free(codes_in);
    int64_t cap = T->cap;
    T->first = (int32_t*)malloc(sizeof(int32_t) * cap);
    T->count = (int32_t*)malloc(sizeof(int32_t) * cap);
    T->level = (int32_t*)malloc(sizeof(int32_t) * cap);
    T->parent = (int32_t*)malloc(sizeof(int32_t) * cap);
    T->skip = (int32_t*)malloc(sizeof(int32_t) * cap);
    T->is_leaf = (int32_t*)malloc(sizeof(int32_t) * cap);
    T->leaf_of = (int32_t*)malloc(sizeof(int32_t) * n);
    T->nn = 0;
    build_node(T, 0, n, 0, -1);
    int64_t nn = T->nn;
    T->area = (double*)malloc(sizeof(double) * nn);
    T->cen = (double*)malloc(sizeof(double) * 3 * nn);
    T->epsn = (double*)malloc(sizeof(double) * nn);
    T->cen32 = (float*)malloc(sizeof(float) * 3 * nn);
    T->r32 = (float*)malloc(sizeof(float) * nn);
    T->s_area = (double*)malloc(sizeof(double) * nn);
    T->s_ap = (double*)malloc(sizeof(double) * 3 * nn);
    T->s_ae = (double*)malloc(sizeof(double) * nn);
    node_sums(T, 0);
    return T;
}

int64_t orc_tree_num_nodes(const orc_tree* T) { return T->nn; }

/* Copy out the tree.  Any pointer may be NULL. */
void orc_tree_export(const orc_tree* T, float* lo_ext, uint32_t* code, uint32_t* perm,
                     int32_t* first, int32_t* count, int32_t* level, int32_t* parent,
                     int32_t* skip, int32_t* is_leaf, double* area, double* cen, double* epsn,
                     float* cen32, float* r32) {
    int64_t n = T->n, nn = T->nn;
    if (lo_ext) memcpy(lo_ext, T->lo_ext, sizeof(float) * 4);
    if (code) memcpy(code, T->code, sizeof(uint32_t) * n);
    if (perm) memcpy(perm, T->perm, sizeof(uint32_t) * n);
    if (first) memcpy(first, T->first, sizeof(int32_t) * nn);
    if (count) memcpy(count, T->count, sizeof(int32_t) * nn);
    if (level) memcpy(level, T->level, sizeof(int32_t) * nn);
    if (parent) memcpy(parent, T->parent, sizeof(int32_t) * nn);
    if (skip) memcpy(skip, T->skip, sizeof(int32_t) * nn);
    if (is_leaf) memcpy(is_leaf, T->is_leaf, sizeof(int32_t) * nn);
    if (area) memcpy(area, T->area, sizeof(double) * nn);
    if (cen) memcpy(cen, T->cen, sizeof(double) * 3 * nn);
    if (epsn) memcpy(epsn, T->epsn, sizeof(double) * nn);
    if (cen32) memcpy(cen32, T->cen32, sizeof(float) * 3 * nn);
    if (r32) memcpy(r32, T->r32, sizeof(float) * nn);
}

/* ------------------------------------------------------------------------ */
/* Tree update: eq. (farfield_dipole_features)                                */
/* ------------------------------------------------------------------------ */

/* n~_t^c = (1/A~_t) sum_{m in t} A_m n_m mu_m^c for every node; mu: [n,C] in
 * input order. */
void orc_tree_update(orc_tree* T, const float* mu, int C) {
    int64_t n = T->n, nn = T->nn;
    free(T->mu);
    free(T->nt);
    free(T->mt);
    free(T->s16);
    free(T->m16);
    free(T->a16);
    free(T->am16);
    T->s16 = T->m16 = T->a16 = T->am16 = NULL;
    T->C = C;
    T->G = C;
    T->mu = (double*)malloc(sizeof(double) * n * C);
    T->nt = (double*)calloc((size_t)(nn * 3 * C), sizeof(double));
    T->mt = (double*)calloc((size_t)(nn * C), sizeof(double));
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < C; ++c) T->mu[i * C + c] = mu[(int64_t)T->perm[i] * C + c];
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < nn; ++t) {
        double* o = T->nt + t * 3 * C;
        for (int64_t m = T->first[t]; m < (int64_t)T->first[t] + T->count[t]; ++m) {
            double A = T->A[m];
            for (int c = 0; c < C; ++c) {
                double v = A * T->mu[m * C + c];
                o[3 * c] += v * T->nrm[3 * m];
                o[3 * c + 1] += v * T->nrm[3 * m + 1];
                o[3 * c + 2] += v * T->nrm[3 * m + 2];
            }
        }
        for (int k = 0; k < 3 * C; ++k) o[k] /= T->area[t];
        /* R12: the area-weighted mean attribute */
        double* mo = T->mt + t * C;
        for (int64_t m = T->first[t]; m < (int64_t)T->first[t] + T->count[t]; ++m)
            for (int c = 0; c < C; ++c) mo[c] += (double)T->A[m] * T->mu[m * C + c];
        for (int c = 0; c < C; ++c) mo[c] /= T->area[t];
    }
}

/* x rounded to float, then to bfloat16 (the upper 16 bits of the float's
 * encoding), each to nearest with ties to even (R13).  Infinities and NaNs
 * pass through. */
double orc_round_bf16(double x) {
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    if ((u & 0x7f800000u) != 0x7f800000u) {
        /* add just under half of the dropped part's unit, plus its last kept
         * bit: a tie rounds up only when the kept part is odd */
        u += 0x7fffu + ((u >> 16) & 1u);
        u &= 0xffff0000u;
    }
    memcpy(&f, &u, sizeof f);
    return f;
}

void orc_round_bf16_n(int64_t n, const double* x, double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = orc_round_bf16(x[i]);
}

/* R13: the bf16 node moments used by PrimalQuery's far field; call after an
 * update (the next update drops them). */
static double ambiguity_bf16(double S, double abs_sum) {
    const double delta = ldexp(abs_sum, -19) + ldexp(fabs(S), -22);
    return orc_round_bf16(S + delta) - orc_round_bf16(S - delta);
}

void orc_tree_round_moments_bf16(orc_tree* T) {
    int64_t nn = T->nn;
    int C = T->C;
    free(T->s16);
    free(T->m16);
    free(T->a16);
    free(T->am16);
    T->s16 = (double*)malloc(sizeof(double) * nn * 3 * C);
    T->m16 = (double*)malloc(sizeof(double) * nn * C);
    T->a16 = (double*)malloc(sizeof(double) * nn * 3 * C);
    T->am16 = (double*)malloc(sizeof(double) * nn * C);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < nn; ++t) {
        double* ab = (double*)calloc((size_t)(4 * C), sizeof(double)); /* sums of |terms| */
        for (int64_t m = T->first[t]; m < (int64_t)T->first[t] + T->count[t]; ++m)
            for (int c = 0; c < C; ++c) {
                double v = fabs((double)T->A[m] * T->mu[m * C + c]);
                ab[3 * c] += v * fabs((double)T->nrm[3 * m]);
                ab[3 * c + 1] += v * fabs((double)T->nrm[3 * m + 1]);
                ab[3 * c + 2] += v * fabs((double)T->nrm[3 * m + 2]);
                ab[3 * C + c] += v;
            }
        for (int k = 0; k < 3 * C; ++k) {
            double S = T->area[t] * T->nt[t * 3 * C + k];
            T->s16[t * 3 * C + k] = orc_round_bf16(S);
            T->a16[t * 3 * C + k] = ambiguity_bf16(S, ab[k]);
        }
        for (int c = 0; c < C; ++c) {
            double S = T->area[t] * T->mt[t * C + c];
            T->m16[t * C + c] = orc_round_bf16(S);
            T->am16[t * C + c] = ambiguity_bf16(S, ab[3 * C + c]);
        }
        free(ab);
    }
}

/* Channels [G, C) skip the foreshortening term (R12); call after an update. */
void orc_tree_set_geometry_channels(orc_tree* T, int G) { T->G = G < 0 ? 0 : G > T->C ? T->C : G; }

/* ------------------------------------------------------------------------ */
/* Barnes-Hut queries: Alg. 1                                                 */
/* ------------------------------------------------------------------------ */

/* Far test of Alg. 1, |x - p~_t| > beta r~_t, in float with a fixed order (R6). */
static int far_test(const float x[3], const float* c, float r, float beta) {
    float dx = x[0] - c[0];
    float dy = x[1] - c[1];
    float dz = x[2] - c[2];
    float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    float R = beta * r;
    return d2 > R * R;
}

int orc_far_test(const float* x, const float* c, float r, float beta) {
    return far_test(x, c, r, beta);
}

/* rho(|p~ - x| / eps~) (p~ - x) / (4 pi |p~ - x|^3): the common factor of
 * GetContribution (eq. farfield) and IncrementGradient (eq. farfield_gradient),
 * without A~ and n~ (R1). */
static void far_vector(const orc_tree* T, int32_t t, const double x[3], double v[3]) {
    double dx = T->cen[3 * t] - x[0], dy = T->cen[3 * t + 1] - x[1], dz = T->cen[3 * t + 2] - x[2];
    double d2 = dx * dx + dy * dy + dz * dz;
    double d = sqrt(d2);
    double k = rho_r(d, T->epsn[t]) / (4.0 * ORC_PI * d2 * d);
    v[0] = k * dx; v[1] = k * dy; v[2] = k * dz;
}

/* rho(|p~ - x| / eps~) / (4 pi |p~ - x|^2): the far-field factor of the
 * channels without the foreshortening term (R12), without A~ and m~. */
static double far_scalar(const orc_tree* T, int32_t t, const double x[3]) {
    double dx = T->cen[3 * t] - x[0], dy = T->cen[3 * t + 1] - x[1], dz = T->cen[3 * t + 2] - x[2];
    double d2 = dx * dx + dy * dy + dz * dz;
    return rho_r(sqrt(d2), T->epsn[t]) / (4.0 * ORC_PI * d2);
}

typedef struct { int64_t tested, accepted, leafpts; } counters;

/* PrimalQuery(x, node): returns all C channels at once (Sec. 6.3). */
static void primal_query(const orc_tree* T, const float xf[3], const double x[3], int32_t t,
                         float beta, double* out, counters* k, double* allow) {
    int C = T->C;
    k->tested++;
    if (far_test(xf, T->cen32 + 3 * t, T->r32[t], beta)) {
        /* GetContribution: A~ rho (p~ - x)/|p~ - x|^3 . n~ / (4 pi) */
        double v[3];
        far_vector(T, t, x, v);
        if (T->s16) { /* R13: the bf16 sums A~ n~ and A~ m~ */
            const double* s = T->s16 + (int64_t)t * 3 * C;
            const double* a = T->a16 + (int64_t)t * 3 * C;
            for (int c = 0; c < T->G; ++c) {
                out[c] += v[0] * s[3 * c] + v[1] * s[3 * c + 1] + v[2] * s[3 * c + 2];
                if (allow)
                    allow[c] += fabs(v[0]) * a[3 * c] + fabs(v[1]) * a[3 * c + 1] +
                                fabs(v[2]) * a[3 * c + 2];
            }
            if (T->G < C) {
                double f = far_scalar(T, t, x);
                for (int c = T->G; c < C; ++c) {
                    out[c] += f * T->m16[(int64_t)t * C + c];
                    if (allow) allow[c] += fabs(f) * T->am16[(int64_t)t * C + c];
                }
            }
            k->accepted++;
            return;
        }
        const double* nt = T->nt + (int64_t)t * 3 * C;
        for (int c = 0; c < T->G; ++c)
            out[c] += T->area[t] * (v[0] * nt[3 * c] + v[1] * nt[3 * c + 1] + v[2] * nt[3 * c + 2]);
        if (T->G < C) { /* R12 */
            double f = far_scalar(T, t, x);
            for (int c = T->G; c < C; ++c) out[c] += T->area[t] * f * T->mt[(int64_t)t * C + c];
        }
        k->accepted++;
        return;
    }
    if (T->is_leaf[t]) { /* exact sum over the leaf's points (R3) */
        for (int64_t m = T->first[t]; m < (int64_t)T->first[t] + T->count[t]; ++m) {
            double w = point_weight(x, T->p[3 * m], T->p[3 * m + 1], T->p[3 * m + 2],
                                    T->nrm[3 * m], T->nrm[3 * m + 1], T->nrm[3 * m + 2],
                                    T->A[m], T->eps[m]);
            double wf = point_weight_nf(x, T->p[3 * m], T->p[3 * m + 1], T->p[3 * m + 2], T->A[m],
                                        T->eps[m]);
            for (int c = 0; c < C; ++c) out[c] += (c < T->G ? w : wf) * T->mu[m * C + c];
        }
        k->leafpts += T->count[t];
        return;
    }
    for (int32_t c = t + 1; c < T->skip[t]; c = T->skip[c])
        primal_query(T, xf, x, c, beta, out, k, allow);
}

/* out[j*C + c] = Barnes-Hut dipole sum at qry[j]; cnt (may be NULL) receives
 * per query {nodes tested, nodes accepted, leaf points summed}. */
/* As orc_bh_forward; with bf16 moments (R13), allow [q, C] (may be NULL)
 * receives the bound on the change that the ambiguous roundings can make. */
void orc_bh_forward_bf16(const orc_tree* T, int64_t q, const float* qry, float beta, double* out,
                         int64_t* cnt, double* allow) {
    int C = T->C;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < q; ++j) {
        float xf[3] = {qry[3 * j], qry[3 * j + 1], qry[3 * j + 2]};
        double x[3] = {xf[0], xf[1], xf[2]};
        double* o = out + j * C;
        double* al = allow ? allow + j * C : NULL;
        for (int c = 0; c < C; ++c) o[c] = 0.0;
        if (al)
            for (int c = 0; c < C; ++c) al[c] = 0.0;
        counters k = {0, 0, 0};
        primal_query(T, xf, x, 0, beta, o, &k, al);
        if (cnt) { cnt[3 * j] = k.tested; cnt[3 * j + 1] = k.accepted; cnt[3 * j + 2] = k.leafpts; }
    }
}

void orc_bh_forward(const orc_tree* T, int64_t q, const float* qry, float beta, double* out,
                    int64_t* cnt) {
    orc_bh_forward_bf16(T, q, qry, beta, out, cnt, NULL);
}

/* Near ties of the far test (R6): the walk of PrimalQuery, counting the
 * tested nodes whose distance from the query is within 1e-6 d of beta r~
 * in double, |d - beta r~| < 1e-6 d.  There the float decision could differ
 * from a double one; the float decision itself is the one taken (R6), so a
 * GPU taking the same float steps agrees with the oracle even there.  A
 * diagnostic of how close a workload's decisions come to the boundary. */
static int64_t near_ties_query(const orc_tree* T, const float xf[3], const double x[3], int32_t t,
                               float beta) {
    double dx = (double)T->cen32[3 * t] - x[0], dy = (double)T->cen32[3 * t + 1] - x[1],
           dz = (double)T->cen32[3 * t + 2] - x[2];
    double d = sqrt(dx * dx + dy * dy + dz * dz);
    int64_t k = fabs(d - (double)beta * (double)T->r32[t]) < 1e-6 * d ? 1 : 0;
    if (far_test(xf, T->cen32 + 3 * t, T->r32[t], beta) || T->is_leaf[t]) return k;
    for (int32_t c = t + 1; c < T->skip[t]; c = T->skip[c]) k += near_ties_query(T, xf, x, c, beta);
    return k;
}

void orc_bh_near_ties(const orc_tree* T, int64_t q, const float* qry, float beta, int64_t* out) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < q; ++j) {
        float xf[3] = {qry[3 * j], qry[3 * j + 1], qry[3 * j + 2]};
        double x[3] = {xf[0], xf[1], xf[2]};
        out[j] = near_ties_query(T, xf, x, 0, beta);
    }
}

/* AdjointQuery(dD, x, node): stage 1 of the two-stage scheme (Sec. 6.2).
 * dnt: [nn,3C] node gradients d n~_t; dmu: [n,C] sorted, for opened leaves. */
static void adjoint_query(const orc_tree* T, const float xf[3], const double x[3],
                          const double* g, int32_t t, float beta, double* dnt, double* dmu) {
    int C = T->C;
    if (far_test(xf, T->cen32 + 3 * t, T->r32[t], beta)) {
        /* IncrementGradient, eq. (farfield_gradient) */
        double v[3];
        far_vector(T, t, x, v);
        double* o = dnt + (int64_t)t * 3 * C;
        for (int c = 0; c < T->G; ++c)
            for (int a = 0; a < 3; ++a) {
                double inc = T->area[t] * v[a] * g[c];
#pragma omp atomic
                o[3 * c + a] += inc;
            }
        if (T->G < C) { /* R12: d m~_t^c in the channel's first slot */
            double f = far_scalar(T, t, x);
            for (int c = T->G; c < C; ++c) {
                double inc = T->area[t] * f * g[c];
#pragma omp atomic
                o[3 * c] += inc;
            }
        }
        return;
    }
    if (T->is_leaf[t]) { /* opened leaf: exact per-point derivative (R3) */
        for (int64_t m = T->first[t]; m < (int64_t)T->first[t] + T->count[t]; ++m) {
            double w = point_weight(x, T->p[3 * m], T->p[3 * m + 1], T->p[3 * m + 2],
                                    T->nrm[3 * m], T->nrm[3 * m + 1], T->nrm[3 * m + 2],
                                    T->A[m], T->eps[m]);
            double wf = point_weight_nf(x, T->p[3 * m], T->p[3 * m + 1], T->p[3 * m + 2], T->A[m],
                                        T->eps[m]);
            for (int c = 0; c < C; ++c) {
                double inc = (c < T->G ? w : wf) * g[c];
#pragma omp atomic
                dmu[m * C + c] += inc;
            }
        }
        return;
    }
    for (int32_t c = t + 1; c < T->skip[t]; c = T->skip[c])
        adjoint_query(T, xf, x, g, c, beta, dnt, dmu);
}

/* grad[m*C + c] (input order) = d L / d mu_m^c, given g[j*C + c] = dL/dD^c(x_j):
 * stage 1 over all queries, then stage 2, eq. (farfield_features_gradient):
 *   d mu_m = sum_{t in AS(m)} (A_m / A~_t) n_m . d n~_t   (R8). */
void orc_bh_adjoint(const orc_tree* T, int64_t q, const float* qry, float beta, const double* g,
                    double* grad) {
    int C = T->C;
    int64_t n = T->n, nn = T->nn;
    double* dnt = (double*)calloc((size_t)(nn * 3 * C), sizeof(double));
    double* dmu = (double*)calloc((size_t)(n * C), sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < q; ++j) {
        float xf[3] = {qry[3 * j], qry[3 * j + 1], qry[3 * j + 2]};
        double x[3] = {xf[0], xf[1], xf[2]};
        adjoint_query(T, xf, x, g + j * C, 0, beta, dnt, dmu);
    }
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < n; ++m) {
        double* gm = grad + (int64_t)T->perm[m] * C;
        for (int c = 0; c < C; ++c) gm[c] = dmu[m * C + c];
        for (int32_t t = T->leaf_of[m]; t >= 0; t = T->parent[t]) {
            double f = (double)T->A[m] / T->area[t];
            const double* d = dnt + (int64_t)t * 3 * C;
            for (int c = 0; c < T->G; ++c)
                gm[c] += f * (T->nrm[3 * m] * d[3 * c] + T->nrm[3 * m + 1] * d[3 * c + 1] +
                              T->nrm[3 * m + 2] * d[3 * c + 2]);
            for (int c = T->G; c < C; ++c) gm[c] += f * d[3 * c]; /* R12 */
        }
    }
    free(dnt);
    free(dmu);
}

/* ------------------------------------------------------------------------ */
/* Spatial gradient with Barnes-Hut (R9) and its adjoint                      */
/* ------------------------------------------------------------------------ */

/* PrimalQuery for grad D: the same walk and far test; a far node adds
 * -A~/(4 pi) [a n~^c + b (n~^c.v) v], v = p~ - x; an opened leaf adds its
 * points' exact gradients. */
static void primal_query_grad(const orc_tree* T, const float xf[3], const double x[3], int32_t t,
                              float beta, double* g) {
    int C = T->C;
    if (far_test(xf, T->cen32 + 3 * t, T->r32[t], beta)) {
        double vx = T->cen[3 * t] - x[0], vy = T->cen[3 * t + 1] - x[1], vz = T->cen[3 * t + 2] - x[2];
        double d = sqrt(vx * vx + vy * vy + vz * vz);
        double a, b;
        grad_factors(d, T->epsn[t], &a, &b);
        double f = -T->area[t] / (4.0 * ORC_PI);
        const double* nt = T->nt + (int64_t)t * 3 * C;
        for (int c = 0; c < C; ++c) {
            double nv = nt[3 * c] * vx + nt[3 * c + 1] * vy + nt[3 * c + 2] * vz;
            g[3 * c] += f * (a * nt[3 * c] + b * nv * vx);
            g[3 * c + 1] += f * (a * nt[3 * c + 1] + b * nv * vy);
            g[3 * c + 2] += f * (a * nt[3 * c + 2] + b * nv * vz);
        }
        return;
    }
    if (T->is_leaf[t]) {
        for (int64_t m = T->first[t]; m < (int64_t)T->first[t] + T->count[t]; ++m) {
            double pg[3];
            point_grad(x, T->p[3 * m], T->p[3 * m + 1], T->p[3 * m + 2], T->nrm[3 * m],
                       T->nrm[3 * m + 1], T->nrm[3 * m + 2], T->A[m], T->eps[m], pg);
            for (int c = 0; c < C; ++c)
                for (int k = 0; k < 3; ++k) g[3 * c + k] += pg[k] * T->mu[m * C + c];
        }
        return;
    }
    for (int32_t c = t + 1; c < T->skip[t]; c = T->skip[c]) primal_query_grad(T, xf, x, c, beta, g);
}

/* grad[(j*C + c)*3 + k] = Barnes-Hut estimate of d D^c / d x_k at qry[j]. */
void orc_bh_forward_grad(const orc_tree* T, int64_t q, const float* qry, float beta, double* grad) {
    int C = T->C;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < q; ++j) {
        float xf[3] = {qry[3 * j], qry[3 * j + 1], qry[3 * j + 2]};
        double x[3] = {xf[0], xf[1], xf[2]};
        double* o = grad + j * 3 * C;
        for (int k = 0; k < 3 * C; ++k) o[k] = 0.0;
        primal_query_grad(T, xf, x, 0, beta, o);
    }
}

/* AdjointQuery for L(D, grad D): gv[c] = dL/dD^c, gg[3c + k] = dL/d(dD^c/dx_k)
 * at this query (either may be NULL).  A far node gets
 *   d n~^c += A~ rho v/(4 pi d^3) gv[c] + M gg^c,  M = -A~/(4 pi) (a I + b v v^T),
 * an opened leaf's point m gets the exact derivative of its terms. */
static void adjoint_query_grad(const orc_tree* T, const float xf[3], const double x[3],
                               const double* gv, const double* gg, int32_t t, float beta,
                               double* dnt, double* dmu) {
    int C = T->C;
    if (far_test(xf, T->cen32 + 3 * t, T->r32[t], beta)) {
        double vx = T->cen[3 * t] - x[0], vy = T->cen[3 * t + 1] - x[1], vz = T->cen[3 * t + 2] - x[2];
        double d = sqrt(vx * vx + vy * vy + vz * vz);
        double a, b;
        grad_factors(d, T->epsn[t], &a, &b);
        double fa = T->area[t] / (4.0 * ORC_PI);
        double* o = dnt + (int64_t)t * 3 * C;
        for (int c = 0; c < C; ++c) {
            double inc[3] = {0.0, 0.0, 0.0};
            if (gv) { /* d/d n~ of A~ a n~.v / (4 pi) = A~ a v / (4 pi) */
                inc[0] += fa * a * vx * gv[c]; inc[1] += fa * a * vy * gv[c]; inc[2] += fa * a * vz * gv[c];
            }
            if (gg) {
                const double* G = gg + 3 * c;
                double vg = vx * G[0] + vy * G[1] + vz * G[2];
                inc[0] -= fa * (a * G[0] + b * vg * vx);
                inc[1] -= fa * (a * G[1] + b * vg * vy);
                inc[2] -= fa * (a * G[2] + b * vg * vz);
            }
            for (int k = 0; k < 3; ++k) {
#pragma omp atomic
                o[3 * c + k] += inc[k];
            }
        }
        return;
    }
    if (T->is_leaf[t]) {
        for (int64_t m = T->first[t]; m < (int64_t)T->first[t] + T->count[t]; ++m) {
            double w = point_weight(x, T->p[3 * m], T->p[3 * m + 1], T->p[3 * m + 2], T->nrm[3 * m],
                                    T->nrm[3 * m + 1], T->nrm[3 * m + 2], T->A[m], T->eps[m]);
            double pg[3];
            point_grad(x, T->p[3 * m], T->p[3 * m + 1], T->p[3 * m + 2], T->nrm[3 * m],
                       T->nrm[3 * m + 1], T->nrm[3 * m + 2], T->A[m], T->eps[m], pg);
            for (int c = 0; c < C; ++c) {
                double inc = 0.0;
                if (gv) inc += w * gv[c];
                if (gg) inc += pg[0] * gg[3 * c] + pg[1] * gg[3 * c + 1] + pg[2] * gg[3 * c + 2];
#pragma omp atomic
                dmu[m * C + c] += inc;
            }
        }
        return;
    }
    for (int32_t c = t + 1; c < T->skip[t]; c = T->skip[c])
        adjoint_query_grad(T, xf, x, gv, gg, c, beta, dnt, dmu);
}

/* dL/dmu [n, C] (input order) for dL/dD = g [q, C] (may be NULL) and
 * dL/d(grad D) = gg [q, C, 3] (may be NULL): stage 1 as above, stage 2 by
 * eq. (farfield_features_gradient). */
void orc_bh_adjoint_grad(const orc_tree* T, int64_t q, const float* qry, float beta,
                         const double* g, const double* gg, double* grad) {
    int C = T->C;
    int64_t n = T->n, nn = T->nn;
    double* dnt = (double*)calloc((size_t)(nn * 3 * C), sizeof(double));
    double* dmu = (double*)calloc((size_t)(n * C), sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < q; ++j) {
        float xf[3] = {qry[3 * j], qry[3 * j + 1], qry[3 * j + 2]};
        double x[3] = {xf[0], xf[1], xf[2]};
        adjoint_query_grad(T, xf, x, g ? g + j * C : NULL, gg ? gg + j * 3 * C : NULL, 0, beta,
                           dnt, dmu);
    }
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < n; ++m) {
        double* gm = grad + (int64_t)T->perm[m] * C;
        for (int c = 0; c < C; ++c) gm[c] = dmu[m * C + c];
        for (int32_t t = T->leaf_of[m]; t >= 0; t = T->parent[t]) {
            double f = (double)T->A[m] / T->area[t];
            const double* d = dnt + (int64_t)t * 3 * C;
            for (int c = 0; c < T->G; ++c)
                gm[c] += f * (T->nrm[3 * m] * d[3 * c] + T->nrm[3 * m + 1] * d[3 * c + 1] +
                              T->nrm[3 * m + 2] * d[3 * c + 2]);
            for (int c = T->G; c < C; ++c) gm[c] += f * d[3 * c]; /* R12 */
        }
    }
    free(dnt);
    free(dmu);
}

/* ------------------------------------------------------------------------ */
/* Gradients with respect to mu, the normals and eps (R10)                    */
/* ------------------------------------------------------------------------ */

/* AdjointQuery for all point parameters.  A far node (v = p~ - x) adds
 *   dn~_t^c += A~/(4 pi) [g^c a v - a G^c - b (v.G^c) v]
 *   deps~_t += A~/(4 pi) sum_c [g^c a_e (n~^c.v) - a_e (n~^c.G^c) - b_e (n~^c.v)(v.G^c)]
 * (a, b, a_e, b_e at d = |v| and eps~_t); an opened leaf adds its points'
 * point_geom_terms. */
static void adjoint_query_geom(const orc_tree* T, const float xf[3], const double x[3],
                               const double* gv, const double* gg, int32_t t, float beta,
                               double* dnt, double* det, double* dmu, double* dnp, double* dep) {
    int C = T->C;
    if (far_test(xf, T->cen32 + 3 * t, T->r32[t], beta)) {
        double vx = T->cen[3 * t] - x[0], vy = T->cen[3 * t + 1] - x[1], vz = T->cen[3 * t + 2] - x[2];
        double d = sqrt(vx * vx + vy * vy + vz * vz);
        double a, b, ae, be;
        grad_factors(d, T->epsn[t], &a, &b);
        eps_factors(d, T->epsn[t], &ae, &be);
        double f = T->area[t] / (4.0 * ORC_PI);
        const double* nt = T->nt + (int64_t)t * 3 * C;
        double* o = dnt + (int64_t)t * 3 * C;
        double e_acc = 0.0;
        for (int c = 0; c < C; ++c) {
            double g = gv ? gv[c] : 0.0;
            double G0 = gg ? gg[3 * c] : 0.0, G1 = gg ? gg[3 * c + 1] : 0.0, G2 = gg ? gg[3 * c + 2] : 0.0;
            double vG = vx * G0 + vy * G1 + vz * G2;
            double nv = nt[3 * c] * vx + nt[3 * c + 1] * vy + nt[3 * c + 2] * vz;
            double nG = nt[3 * c] * G0 + nt[3 * c + 1] * G1 + nt[3 * c + 2] * G2;
            double inc[3] = {f * (g * a * vx - a * G0 - b * vG * vx),
                             f * (g * a * vy - a * G1 - b * vG * vy),
                             f * (g * a * vz - a * G2 - b * vG * vz)};
            for (int k = 0; k < 3; ++k) {
#pragma omp atomic
                o[3 * c + k] += inc[k];
            }
            e_acc += f * (g * ae * nv - ae * nG - be * nv * vG);
        }
#pragma omp atomic
        det[t] += e_acc;
        return;
    }
    if (T->is_leaf[t]) {
        double* dm = (double*)calloc((size_t)C, sizeof(double));
        for (int64_t m = T->first[t]; m < (int64_t)T->first[t] + T->count[t]; ++m) {
            double dv[3] = {0.0, 0.0, 0.0}, de = 0.0;
            for (int c = 0; c < C; ++c) dm[c] = 0.0;
            point_geom_terms(x, T->p + 3 * m, T->nrm + 3 * m, T->A[m], T->eps[m], C,
                             T->mu + m * C, gv, gg, dm, dv, &de);
            for (int c = 0; c < C; ++c) {
#pragma omp atomic
                dmu[m * C + c] += dm[c];
            }
            for (int k = 0; k < 3; ++k) {
#pragma omp atomic
                dnp[3 * m + k] += dv[k];
            }
#pragma omp atomic
            dep[m] += de;
        }
        free(dm);
        return;
    }
    for (int32_t c = t + 1; c < T->skip[t]; c = T->skip[c])
        adjoint_query_geom(T, xf, x, gv, gg, c, beta, dnt, det, dmu, dnp, dep);
}

/* dL/dmu [n,C], dL/dn [n,3] and dL/deps [n] (input order; any output may be
 * NULL) for dL/dD = g [q,C] and dL/d(grad D) = gg [q,C,3] (either may be
 * NULL).  Stage 2 per point m, over the nodes t holding it (R8):
 *   dmu_m^c = near + sum_t (A_m/A~_t) n_m . dn~_t^c   (eq. farfield_features_gradient)
 *   dn_m    = near + sum_t sum_c (A_m mu_m^c/A~_t) dn~_t^c
 *   deps_m  = near + sum_t (A_m/A~_t) deps~_t */
void orc_bh_adjoint_geom(const orc_tree* T, int64_t q, const float* qry, float beta,
                         const double* g, const double* gg, double* gmu, double* gn,
                         double* geps) {
    int C = T->C;
    int64_t n = T->n, nn = T->nn;
    double* dnt = (double*)calloc((size_t)(nn * 3 * C), sizeof(double));
    double* det = (double*)calloc((size_t)nn, sizeof(double));
    double* dmu = (double*)calloc((size_t)(n * C), sizeof(double));
    double* dnp = (double*)calloc((size_t)(n * 3), sizeof(double));
    double* dep = (double*)calloc((size_t)n, sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < q; ++j) {
        float xf[3] = {qry[3 * j], qry[3 * j + 1], qry[3 * j + 2]};
        double x[3] = {xf[0], xf[1], xf[2]};
        adjoint_query_geom(T, xf, x, g ? g + j * C : NULL, gg ? gg + j * 3 * C : NULL, 0, beta,
                           dnt, det, dmu, dnp, dep);
    }
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < n; ++m) {
        int64_t o = T->perm[m];
        const float* nm = T->nrm + 3 * m;
        for (int c = 0; c < C; ++c) {
            double s = dmu[m * C + c];
            for (int32_t t = T->leaf_of[m]; t >= 0; t = T->parent[t]) {
                const double* d = dnt + (int64_t)t * 3 * C + 3 * c;
                s += (double)T->A[m] / T->area[t] * (nm[0] * d[0] + nm[1] * d[1] + nm[2] * d[2]);
            }
            if (gmu) gmu[o * C + c] = s;
        }
        double v[3] = {dnp[3 * m], dnp[3 * m + 1], dnp[3 * m + 2]}, e = dep[m];
        for (int32_t t = T->leaf_of[m]; t >= 0; t = T->parent[t]) {
            double f = (double)T->A[m] / T->area[t];
            for (int c = 0; c < C; ++c) {
                const double* d = dnt + (int64_t)t * 3 * C + 3 * c;
                for (int k = 0; k < 3; ++k) v[k] += f * T->mu[m * C + c] * d[k];
            }
            e += f * det[t];
        }
        if (gn)
            for (int k = 0; k < 3; ++k) gn[3 * o + k] = v[k];
        if (geps) geps[o] = e;
    }
    free(dnt);
    free(det);
    free(dmu);
    free(dnp);
    free(dep);
}
