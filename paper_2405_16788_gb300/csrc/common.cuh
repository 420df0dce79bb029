// Internal declarations shared by the CUDA translation units of libdipole.
// Paper: "3D Reconstruction with Fast Dipole Sums" (arXiv 2405.16788).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace dip {

constexpr float kInv4Pi = 0.0795774715459476679f;  // 1 / (4 pi), eq. pcwn
constexpr int kMaxLevel = 10;                       // 30-bit codes: 10 octal digits
constexpr int kMaxChannels = 64;

// Bottom-up node geometry: levels above kTopLevel one launch each; levels
// kTopLevel to 0 (few nodes) in one block of kTopThreads threads.
constexpr int kTopLevel = 4;
constexpr int kTopThreads = 1024;

// Device status bits (OR-ed by kernels, read by dipole_sync_status).
constexpr int kStatusTraversal = 1;
constexpr int kStatusNonFinite = 2;
constexpr int kStatusBadArea = 4;
constexpr int kStatusBadRadius = 8;

// One octree node, 32 bytes = one L2 sector, read by every visiting warp.
//   geo  = {p~.x, p~.y, p~.z, r~}            (Sec. 6.1, eq. farfield_dipole)
//   meta = {skip, first, leaf point count (0 for internal nodes), bits of 1/eps~}
struct __align__(32) NodeRec {
    float4 geo;
    int4 meta;
};

// One point in Morton order, 32 bytes.
//   geo = {p.x, p.y, p.z, 1/eps}  (1/eps = +inf for eps = 0)
//   w   = {A n.x, A n.y, A n.z, A}
struct __align__(32) PointRec {
    float4 geo;
    float4 w;
};

// Everything a kernel needs to see of a tree.
struct TreeView {
    int64_t n;
    int64_t nn;
    const NodeRec* nodes;
    const PointRec* pts;
    const uint32_t* perm;
    const int32_t* parent;
    const int32_t* first;
    const int32_t* count;
    const int32_t* is_leaf;
    const float* bbox;  // lo.x, lo.y, lo.z, ext, scale
    int* status;
};

// ---------------------------------------------------------------- sorting
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of key.
// keys/vals are sorted in place; tmp buffers hold n entries each.  hist must
// hold radix_hist_entries(n) uint32 entries.
int64_t radix_hist_entries(int64_t n);
void radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                      uint32_t* hist, int64_t n, int bits, cudaStream_t s);

// Exclusive scan of n uint32 values in place; tmp holds scan_tmp_entries(n).
int64_t scan_tmp_entries(int64_t n);
void exclusive_scan_u32(uint32_t* data, int64_t n, uint32_t* tmp, cudaStream_t s);

// 30-bit Morton code (shifted right by `shift`) of each point in the tree's
// bounding cube (clamped to it) and the identity permutation; codes/idx hold
// q entries.
void query_codes(const float* queries, int64_t q, const float* bbox, int shift, uint32_t* codes,
                 uint32_t* idx, int* status, cudaStream_t s);

// Query sort key: the top 16 bits of the Morton code keep warps as coherent
// as all 30 bits do and take two radix passes instead of four.
constexpr int kQueryKeyBits = 16;

int num_sms();

// Read `bytes` of buf `passes` times with L2-only loads (sink: 1024 * SMs floats).
void probe_l2(const void* buf, int64_t bytes, int passes, float* sink, cudaStream_t s);

// Counts the library's kernel launches (dipole_kernel_launches).
void note_launch();


// Padded channel counts with a compiled kernel instantiation.
int padded_channels(int C);

}  // namespace dip

// Error helper used by host code: records the message and returns DIPOLE_ECUDA.
#define DIP_CUDA_TRY(expr)                                                  \
    do {                                                                    \
        cudaError_t _e = (expr);                                            \
        if (_e != cudaSuccess) return dip_cuda_fail(_e, #expr, __FILE__, __LINE__); \
    } while (0)

int dip_cuda_fail(cudaError_t e, const char* what, const char* file, int line);
int dip_fail(int code, const std::string& msg);
