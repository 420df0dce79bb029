// Tree update of the node moments (Sec. 6.1, eq. farfield_dipole_features;
// Sec. 6.3: refreshed at the start of every iteration) and the second stage
// of the adjoint (Sec. 6.2; App. C, eq. farfield_features_gradient).
//
// Moments are stored as S_t^c = A~_t n~_t^c = sum_{m in t} A_m n_m mu_m^c, so the
// far field needs no division by A~_t and stage 2 needs no multiplication by
// A_m / A~_t: d mu_m^c = (A_m n_m) . sum_{t holding m} dS_t^c.
#include "kernels.cuh"
#include "tree.cuh"

namespace dip {
namespace {

template <typename AT>
__device__ __forceinline__ float to_f(AT v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename AT>
__device__ __forceinline__ AT from_f(float v);
template <>
__device__ __forceinline__ float from_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// Bottom-up in two kinds of launches: every leaf gathers its points'
// attributes into Morton order and sums its moments in float; then, level by
// level from the deepest, every internal node sums its children in order, in
// double when it holds at least kBigNode points.
template <int CP, typename AT>
__global__ void __launch_bounds__(128) k_refit_leaves(
    int64_t nn, const PointRec* __restrict__ pts, const uint32_t* __restrict__ perm,
    const int32_t* __restrict__ first, const int32_t* __restrict__ count,
    const int32_t* __restrict__ is_leaf, const int32_t* __restrict__ big_idx,
    const AT* __restrict__ attrs, int C, AT* __restrict__ mu, float* __restrict__ S,
    double* __restrict__ S64) {
    constexpr int SR = srow(CP);
    for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t0 < nn;
         t0 += (int64_t)gridDim.x * blockDim.x) {
        if (!is_leaf[t0]) continue;
        const int64_t f = first[t0], k = count[t0];
        for (int64_t m = f; m < f + k; ++m) {
            const int64_t o = perm[m];
#pragma unroll
            for (int c = 0; c < CP; ++c) mu[m * CP + c] = c < C ? attrs[o * C + c] : from_f<AT>(0.0f);
        }
        const int32_t bl = big_idx[t0];
#pragma unroll
        for (int c0 = 0; c0 < CP; c0 += 4) {
            float sacc[12];
#pragma unroll
            for (int j = 0; j < 12; ++j) sacc[j] = 0.0f;
            for (int64_t m = f; m < f + k; ++m) {
                const float4 w = pts[m].w;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (c0 + c >= CP) break;
                    const float v = to_f<AT>(mu[m * CP + c0 + c]);
                    sacc[3 * c] = fmaf(w.x, v, sacc[3 * c]);
                    sacc[3 * c + 1] = fmaf(w.y, v, sacc[3 * c + 1]);
                    sacc[3 * c + 2] = fmaf(w.z, v, sacc[3 * c + 2]);
                }
            }
#pragma unroll
            for (int j = 0; j < 12; ++j) {
                if (3 * c0 + j >= 3 * CP) break;
                S[t0 * SR + 3 * c0 + j] = sacc[j];
                if (bl >= 0) S64[(int64_t)bl * SR + 3 * c0 + j] = (double)sacc[j];
            }
        }
    }
}

template <int CP>
__global__ void __launch_bounds__(128) k_refit_level(int l, const int32_t* __restrict__ lvl_off,
                                                     const int32_t* __restrict__ lvl_list,
                                                     const int32_t* __restrict__ skip,
                                                     const int32_t* __restrict__ big_idx,
                                                     float* __restrict__ S, double* __restrict__ S64) {
    constexpr int SR = srow(CP);
    const int32_t b = lvl_off[l], e = lvl_off[l + 1];
    for (int64_t i = b + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < e;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = lvl_list[i];
        const int32_t bp = big_idx[p];
        const int32_t end = skip[p];
#pragma unroll 1
        for (int j0 = 0; j0 < 3 * CP; j0 += 12) {
            if (bp >= 0) {
                double q[12];
#pragma unroll
                for (int j = 0; j < 12; ++j) q[j] = 0.0;
                int kc = 0;
                for (int32_t ch = p + 1; ch < end && kc < 8; ++kc) {
                    const int32_t bc = big_idx[ch];
#pragma unroll
                    for (int j = 0; j < 12; ++j) {
                        if (j0 + j >= 3 * CP) break;
                        q[j] += bc >= 0 ? S64[(int64_t)bc * SR + j0 + j]
                                        : (double)S[(int64_t)ch * SR + j0 + j];
                    }
                    const int32_t nx = skip[ch];
                    if (nx <= ch) break;  // only an imported, corrupt tree gets here
                    ch = nx;
                }
#pragma unroll
                for (int j = 0; j < 12; ++j) {
                    if (j0 + j >= 3 * CP) break;
                    S64[(int64_t)bp * SR + j0 + j] = q[j];
                    S[(int64_t)p * SR + j0 + j] = (float)q[j];
                }
            } else {
                float q[12];
#pragma unroll
                for (int j = 0; j < 12; ++j) q[j] = 0.0f;
                int kc = 0;
                for (int32_t ch = p + 1; ch < end && kc < 8; ++kc) {
#pragma unroll
                    for (int j = 0; j < 12; ++j) {
                        if (j0 + j >= 3 * CP) break;
                        q[j] += S[(int64_t)ch * SR + j0 + j];
                    }
                    const int32_t nx = skip[ch];
                    if (nx <= ch) break;  // only an imported, corrupt tree gets here
                    ch = nx;
                }
#pragma unroll
                for (int j = 0; j < 12; ++j) {
                    if (j0 + j >= 3 * CP) break;
                    S[(int64_t)p * SR + j0 + j] = q[j];
                }
            }
        }
    }
}

// Stage 2 (eq. farfield_features_gradient): for each leaf, D^c = sum of dS^c
// over the leaf and its ancestors; each point of the leaf gets
// (A_m n_m) . D^c plus its opened-leaf term, written in the caller's order.
template <int CP>
__global__ void __launch_bounds__(128) k_stage2(
    int64_t nn, const PointRec* __restrict__ pts, const uint32_t* __restrict__ perm,
    const int32_t* __restrict__ first, const int32_t* __restrict__ count,
    const int32_t* __restrict__ is_leaf, const int32_t* __restrict__ parent,
    const float* __restrict__ dS, const float* __restrict__ dmu, int C, int accumulate,
    float* __restrict__ grad) {
    constexpr int SR = srow(CP);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (!is_leaf[t]) continue;
        const int64_t f = first[t], k = count[t];
#pragma unroll 1
        for (int c0 = 0; c0 < CP; c0 += 4) {
            float D[12];
#pragma unroll
            for (int j = 0; j < 12; ++j) D[j] = 0.0f;
            for (int64_t u = t; u >= 0; u = parent[u]) {
#pragma unroll
                for (int j = 0; j < 12; ++j) {
                    if (3 * c0 + j >= 3 * CP) break;
                    D[j] += dS[u * SR + 3 * c0 + j];
                }
            }
            for (int64_t m = f; m < f + k; ++m) {
                const float4 w = pts[m].w;
                const int64_t o = perm[m];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int ch = c0 + c;
                    if (ch >= CP) break;
                    if (ch >= C) continue;
                    float v = fmaf(w.x, D[3 * c], fmaf(w.y, D[3 * c + 1], w.z * D[3 * c + 2]));
                    v += dmu[m * CP + ch];
                    float* dst = grad + o * C + ch;
                    *dst = accumulate ? *dst + v : v;
                }
            }
        }
    }
}

// Stage 2 for the normals and radii (reading of the paper's training of n and
// eps, Sec. 7 with App. C).  Per leaf, over the nodes u holding it:
//   dL/dn_m   = A_m sum_c mu_m^c sum_u dS_u^c + opened-leaf terms,
//   dL/deps_m = A_m sum_u dE_u / A~_u       + opened-leaf terms,
// since S_u^c = sum A_m mu_m^c n_m and eps~_u = sum A_m eps_m / A~_u.
template <int CP, typename AT>
__global__ void __launch_bounds__(128) k_stage2_geom(
    int64_t nn, const PointRec* __restrict__ pts, const uint32_t* __restrict__ perm,
    const int32_t* __restrict__ first, const int32_t* __restrict__ count,
    const int32_t* __restrict__ is_leaf, const int32_t* __restrict__ parent,
    const double* __restrict__ agg64, const float* __restrict__ dS, const float* __restrict__ dE,
    const AT* __restrict__ mu, const float* __restrict__ dgeo, int accumulate,
    float* __restrict__ grad_n, float* __restrict__ grad_eps) {
    constexpr int SR = srow(CP);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nn;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (!is_leaf[t]) continue;
        const int64_t f = first[t], k = count[t];
        if (grad_eps) {
            float E = 0.0f;
            for (int64_t u = t; u >= 0; u = parent[u])
                E = fmaf(dE[u], __frcp_rn((float)agg64[5 * u]), E);
            for (int64_t m = f; m < f + k; ++m) {
                const float v = fmaf(pts[m].w.w, E, dgeo[4 * m + 3]);
                float* dst = grad_eps + perm[m];
                *dst = accumulate ? *dst + v : v;
            }
        }
        if (!grad_n) continue;
#pragma unroll 1
        for (int c0 = 0; c0 < CP; c0 += 4) {
            float D[12];
#pragma unroll
            for (int j = 0; j < 12; ++j) D[j] = 0.0f;
            for (int64_t u = t; u >= 0; u = parent[u]) {
#pragma unroll
                for (int j = 0; j < 12; ++j) {
                    if (3 * c0 + j >= 3 * CP) break;
                    D[j] += dS[u * SR + 3 * c0 + j];
                }
            }
            for (int64_t m = f; m < f + k; ++m) {
                float v[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (c0 + c >= CP) break;
                    const float mc = to_f<AT>(mu[m * CP + c0 + c]);
#pragma unroll
                    for (int j = 0; j < 3; ++j) v[j] = fmaf(mc, D[3 * c + j], v[j]);
                }
                const float A = pts[m].w.w;
                float* dst = grad_n + 3 * (int64_t)perm[m];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float x = A * v[j];
                    if (c0 == 0) {
                        x += dgeo[4 * m + j];
                        dst[j] = accumulate ? dst[j] + x : x;
                    } else {
                        dst[j] += x;
                    }
                }
            }
        }
    }
}

template <int CP, typename AT>
void launch_stage2_geom(const dipole_tree* t, float* grad_n, float* grad_eps, int accumulate,
                        cudaStream_t s) {
    int64_t blocks = (t->nn + 127) / 128;
    int64_t cap = (int64_t)num_sms() * 16;
    note_launch();
    k_stage2_geom<CP, AT><<<(unsigned)(blocks < cap ? blocks : cap), 128, 0, s>>>(
        t->nn, t->pts, t->perm, t->first, t->count, t->is_leaf, t->parent, t->agg64, t->dS, t->dE,
        (const AT*)t->mu, t->dgeo, accumulate, grad_n, grad_eps);
}

template <int CP, typename AT>
void launch_refit(dipole_tree* t, const void* attrs, cudaStream_t s) {
    int64_t blocks = (t->nn + 127) / 128;
    int64_t cap = (int64_t)num_sms() * 16;
    const unsigned grid = (unsigned)(blocks < cap ? blocks : cap);
    note_launch();
    k_refit_leaves<CP, AT><<<grid, 128, 0, s>>>(t->nn, t->pts, t->perm, t->first, t->count,
                                                t->is_leaf, t->big_idx, (const AT*)attrs, t->C,
                                                (AT*)t->mu, t->S, t->S64);
    for (int l = t->max_depth - 1; l >= 0; --l) {
        note_launch();
        k_refit_level<CP><<<4u * (unsigned)num_sms(), 128, 0, s>>>(l, t->lvl_off, t->lvl_list, t->skip, t->big_idx,
                                                t->S, t->S64);
    }
}

template <int CP>
void launch_stage2(const dipole_tree* t, float* grad, int accumulate, cudaStream_t s) {
    int64_t blocks = (t->nn + 127) / 128;
    int64_t cap = (int64_t)num_sms() * 16;
    note_launch(); k_stage2<CP><<<(unsigned)(blocks < cap ? blocks : cap), 128, 0, s>>>(
        t->nn, t->pts, t->perm, t->first, t->count, t->is_leaf, t->parent, t->dS, t->dmu, t->C,
        accumulate, grad);
}

}  // namespace

int padded_channels(int C) {
    if (C <= 1) return 1;
    if (C <= 2) return 2;
    if (C <= 4) return 4;
    if (C <= 8) return 8;
    if (C <= 16) return 16;
    if (C <= 32) return 32;
    return 64;
}

int refit(dipole_tree* t, const void* attrs, int C, int dtype, cudaStream_t s) {
    const int Cp = padded_channels(C);
    const int SR = srow(Cp);
    if (t->attr_Cp_alloc != Cp || t->attr_dtype_alloc != dtype) {
        // (re)allocate the attribute state; previous buffers are freed in stream order
        void* bufs[] = {t->mu, t->S, t->S64, t->dS, t->dmu};
        for (void* b : bufs)
            if (b) cudaFreeAsync(b, s);
        t->mu = nullptr; t->S = nullptr; t->S64 = nullptr; t->dS = nullptr; t->dmu = nullptr;
        const size_t esz = dtype == 1 ? 2 : 4;
        DIP_CUDA_TRY(cudaMallocAsync(&t->mu, esz * (size_t)t->n * Cp, s));
        DIP_CUDA_TRY(cudaMallocAsync((void**)&t->S, sizeof(float) * (size_t)t->nn * SR, s));
        DIP_CUDA_TRY(cudaMallocAsync((void**)&t->S64, sizeof(double) * (size_t)(t->nbig + 1) * SR, s));
        DIP_CUDA_TRY(cudaMallocAsync((void**)&t->dS, sizeof(float) * (size_t)t->nn * SR, s));
        DIP_CUDA_TRY(cudaMallocAsync((void**)&t->dmu, sizeof(float) * (size_t)t->n * Cp, s));
        DIP_CUDA_TRY(cudaMemsetAsync(t->S, 0, sizeof(float) * (size_t)t->nn * SR, s));
        t->attr_Cp_alloc = Cp;
        t->attr_dtype_alloc = dtype;
    }
    t->C = C;
    t->Cp = Cp;
    t->dtype = dtype;
#define DIP_REFIT_CASE(K)                                                          \
    case K:                                                                        \
        if (dtype == 1) launch_refit<K, __nv_bfloat16>(t, attrs, s);               \
        else launch_refit<K, float>(t, attrs, s);                                  \
        break;
    switch (Cp) {
        DIP_REFIT_CASE(1)
        DIP_REFIT_CASE(2)
        DIP_REFIT_CASE(4)
        DIP_REFIT_CASE(8)
        DIP_REFIT_CASE(16)
        DIP_REFIT_CASE(32)
        DIP_REFIT_CASE(64)
        default:
            return dip_fail(-1, "dipole_refit: unsupported channel count");
    }
#undef DIP_REFIT_CASE
    DIP_CUDA_TRY(cudaGetLastError());
    return 0;
}

int stage2(const dipole_tree* t, float* grad, int accumulate, cudaStream_t s) {
    switch (t->Cp) {
        case 1: launch_stage2<1>(t, grad, accumulate, s); break;
        case 2: launch_stage2<2>(t, grad, accumulate, s); break;
        case 4: launch_stage2<4>(t, grad, accumulate, s); break;
        case 8: launch_stage2<8>(t, grad, accumulate, s); break;
        case 16: launch_stage2<16>(t, grad, accumulate, s); break;
        case 32: launch_stage2<32>(t, grad, accumulate, s); break;
        case 64: launch_stage2<64>(t, grad, accumulate, s); break;
        default: return dip_fail(-1, "dipole_adjoint: unsupported channel count");
    }
    DIP_CUDA_TRY(cudaGetLastError());
    return 0;
}

int ensure_geom_scratch(dipole_tree* t, cudaStream_t s) {
    if (!t->dE) DIP_CUDA_TRY(cudaMallocAsync((void**)&t->dE, sizeof(float) * (size_t)t->nn, s));
    if (!t->dgeo) DIP_CUDA_TRY(cudaMallocAsync((void**)&t->dgeo, sizeof(float) * 4 * (size_t)t->n, s));
    return 0;
}

int stage2_geom(const dipole_tree* t, float* grad_n, float* grad_eps, int accumulate,
                cudaStream_t s) {
    if (!grad_n && !grad_eps) return 0;
#define DIP_S2G_CASE(K)                                                                   \
    case K:                                                                               \
        if (t->dtype == 1) launch_stage2_geom<K, __nv_bfloat16>(t, grad_n, grad_eps, accumulate, s); \
        else launch_stage2_geom<K, float>(t, grad_n, grad_eps, accumulate, s);            \
        break;
    switch (t->Cp) {
        DIP_S2G_CASE(1)
        DIP_S2G_CASE(2)
        DIP_S2G_CASE(4)
        DIP_S2G_CASE(8)
        DIP_S2G_CASE(16)
        DIP_S2G_CASE(32)
        DIP_S2G_CASE(64)
        default:
            return dip_fail(-1, "stage2_geom: unsupported channel count");
    }
#undef DIP_S2G_CASE
    DIP_CUDA_TRY(cudaGetLastError());
    return 0;
}

}  // namespace dip
