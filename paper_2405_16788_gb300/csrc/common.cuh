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
constexpr int kStatusBounds = 16;

// The checked build (nvcc -DDIPOLE_CHECKED, a separate library) tests the
// indexes that the traversals read from arrays (work items and their order,
// the query permutation, parents, a leaf's point range) before using them: one
// outside its array sets kStatusBounds and the access is skipped, so the call
// returns DIPOLE_EBOUNDS instead of reading or writing out of bounds.  In the
// normal build the tests compile to nothing.
#ifdef DIPOLE_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
__device__ __forceinline__ bool in_bounds(bool ok, int* status) {
    if (kChecked && !ok) {
        atomicOr(status, kStatusBounds);
        return false;
    }
    return true;
}

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

// ---------------------------------------------------------- cube cells
// Cell (10 bits per axis) of a point in the tree's bounding cube, clamped to
// it: floor((x - lo) s) with one rounding per operation; cvt.rzi.u32
// saturates negatives and NaN to 0.
__device__ __forceinline__ void cube_cell(float x, float y, float z, const float* bbox,
                                          uint32_t& qx, uint32_t& qy, uint32_t& qz) {
    const float s = bbox[4];
    qx = min(__float2uint_rz(__fmul_rn(__fsub_rn(x, bbox[0]), s)), 1023u);
    qy = min(__float2uint_rz(__fmul_rn(__fsub_rn(y, bbox[1]), s)), 1023u);
    qz = min(__float2uint_rz(__fmul_rn(__fsub_rn(z, bbox[2]), s)), 1023u);
}

__device__ __forceinline__ uint32_t spread_bits10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// 30-bit Morton code: bit k of qx, qy, qz goes to bit 3k+2, 3k+1, 3k.
__device__ __forceinline__ uint32_t morton30(uint32_t qx, uint32_t qy, uint32_t qz) {
    return (spread_bits10(qx) << 2) | (spread_bits10(qy) << 1) | spread_bits10(qz);
}

// 30-bit index of the cell on the 3-D Hilbert curve of order 10, by
// Skilling's transform ("Programming the Hilbert curve", AIP Conf. Proc. 707,
// 2004): the axes are turned into the curve's transposed index in place, whose
// bits, interleaved like a Morton code, are the index.  Consecutive indices
// are face-adjacent cells, so a run of them stays more compact than a run of
// Morton codes (which jump at every octant boundary).
__device__ __forceinline__ uint32_t hilbert30(uint32_t qx, uint32_t qy, uint32_t qz) {
    uint32_t x[3] = {qx, qy, qz};
#pragma unroll
    for (uint32_t Q = 1u << 9; Q > 1u; Q >>= 1) {
        const uint32_t P = Q - 1u;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (x[i] & Q) {
                x[0] ^= P;
            } else {
                const uint32_t t = (x[0] ^ x[i]) & P;
                x[0] ^= t;
                x[i] ^= t;
            }
        }
    }
    x[1] ^= x[0];
    x[2] ^= x[1];
    uint32_t t = 0;
#pragma unroll
    for (uint32_t Q = 1u << 9; Q > 1u; Q >>= 1)
        if (x[2] & Q) t ^= Q - 1u;
    return morton30(x[0] ^ t, x[1] ^ t, x[2] ^ t);
}

// ------------------------------------------------------- memory blocks
// Several arrays in one device allocation (each API call costs the host
// microseconds): call the same sequence of take() twice, first with base ==
// nullptr to size the block, then with the block; each array starts on a
// 256-byte boundary.
struct Carve {
    char* base = nullptr;
    size_t off = 0;
    template <typename T>
    void take(T** p, int64_t count) {
        off = (off + 255) & ~size_t(255);
        *p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += sizeof(T) * (size_t)(count > 0 ? count : 1);
    }
};

// ---------------------------------------------------------------- sorting
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of key.
// keys/vals are sorted in place; tmp buffers hold n entries each.  hist must
// hold radix_hist_entries(n) uint32 entries.
int64_t radix_hist_entries(int64_t n);
// done_zero: an arrival counter that is zero (kept zero), else one in hist is
// cleared first.
void radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                      uint32_t* hist, int64_t n, int bits, cudaStream_t s,
                      unsigned* done_zero = nullptr);

// Exclusive scan in one launch, tile-local: the scan's value at i is
// data[i] + ws[i / kScanTileSize]; ws holds scan_local_entries(n) entries and
// *grand (if given) receives the sum of all values.
constexpr int kScanTileSize = 4096;
int64_t scan_local_entries(int64_t n);
void exclusive_scan_local(uint32_t* data, int64_t n, uint32_t* ws, uint32_t* grand,
                          cudaStream_t s, unsigned* done_zero = nullptr);


// 30-bit Morton code (Hilbert index with `hilbert`), shifted right by
// `shift`, of each point in the tree's bounding cube (clamped to it) and the
// identity permutation; codes/idx hold q entries.
void query_codes(const float* queries, int64_t q, const float* bbox, int shift, uint32_t* codes,
                 uint32_t* idx, int* status, cudaStream_t s, bool hilbert = false);

// Query sort key: the top 16 bits of the Hilbert index keep warps about as
// coherent as all 30 bits do and take two radix passes instead of four.
constexpr int kQueryKeyBits = 16;

int num_sms();

// Read `bytes` of buf `passes` times with L2-only loads (sink: 1024 * SMs floats).
void probe_l2(const void* buf, int64_t bytes, int passes, float* sink, cudaStream_t s);

// Counts the library's kernel launches (dipole_kernel_launches).
void note_launch();

// Every device allocation of the library goes through here: stream-ordered
// cudaMallocAsync, counted for dipole_device_allocations.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);


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
