// Internal declarations of libhtex (not part of the public ABI).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "htex.h"

// Host-side halfedge mesh: the six operators of the paper's halfedge
// representation (Section 2, Fig. 2), one int32 array each.
struct htex_mesh {
    int32_t H = 0, E = 0, B = 0, V = 0, F = 0;
    std::vector<int32_t> twin, next, prev, vert, edge, face;
};

// Device-resident asset: packed per-halfedge lookup records, per-edge
// texture headers, per-edge scales and the texel pool.
//
// Lookup record of halfedge h (16 bytes): the three halfedges Alg. 3
// visits are h, Next(h) and Prev(h); for each, the edge (texture) it maps
// to through Edge(.) and whether Alg. 2 reflects its coordinates
// (bit 31 set when g < Twin(g)).  w holds Face(h).
//
// Texture header of edge e (16 bytes): x = byte offset / 16, y = log2 N_e,
// z = scale bits (float), w = 0.
struct HostPath;   // staging for htex_lookup_host (host_path.cu)

struct htex_textures {
    int32_t H = 0, E = 0, C = 0;
    htex_dtype dtype = HTEX_F32;
    int32_t uniform_log2n = -1;      // >= 0 when every texture has that resolution
    int64_t uniform_stride = 0;      // bytes per texture when uniform
    int64_t pool_bytes = 0;
    int64_t device_bytes = 0;
    int32_t max_log2n = 0;
    bool has_scales = false;
    void* d_rec = nullptr;           // int4 [H]
    void* d_hdr = nullptr;           // int4 [E]
    void* d_scale = nullptr;         // float [E]
    void* d_pool = nullptr;          // bytes [pool_bytes]
    int device = 0;
    int num_sms = 0;
    HostPath* host_path = nullptr;   // created by the first htex_lookup_host
    cudaStream_t free_stream = nullptr;  // set: buffers came from a pool, freed stream-ordered here
};

void htex_host_path_destroy(HostPath* hp);

// Host-side arrays of a resident asset: packed records, headers, scales
// (padded to whole 16-byte words) and layout facts.
struct HtexAssetArrays {
    std::vector<int32_t> rec;    // 4 per halfedge
    std::vector<int32_t> hdr;    // 4 per edge
    std::vector<float> scale;    // per edge, padded
    int32_t H = 0, E = 0, C = 0;
    htex_dtype dtype = HTEX_F32;
    int32_t uniform_log2n = -1, max_log2n = 0;
    int64_t uniform_stride = 0, pool_bytes = 0;
};

// Build the arrays (no GPU work).
htex_status htex_asset_arrays(const htex_mesh* m, int32_t C, htex_dtype dtype, const int32_t* log2n,
                              const float* scales, HtexAssetArrays* out);
// Allocate the device memory of an asset described by 'a' on the current
// device (no copies); device_bytes counts it.
htex_status htex_asset_allocate(const HtexAssetArrays& a, htex_textures** out);
// Same, from a memory pool, stream-ordered on 'stream' (the buffers are
// released stream-ordered on that stream by htex_textures_destroy).
htex_status htex_asset_allocate_async(const HtexAssetArrays& a, cudaMemPool_t pool, cudaStream_t stream,
                                      htex_textures** out);
// Device bytes an asset described by 'a' occupies.
int64_t htex_asset_device_bytes(const HtexAssetArrays& a);
// Enqueue the copies of records, headers, scales and the pool (host
// buffers must stay valid until 'stream' has run them).
htex_status htex_asset_copy_async(const HtexAssetArrays& a, const void* pool, htex_textures* t, cudaStream_t stream);

constexpr uint32_t kFlipBit = 0x80000000u;
constexpr int kMaxLog2Res = 13;   // texture-relative byte offsets fit 32 bits

int htex_elem_size(htex_dtype d);
bool htex_dtype_valid(int32_t d);

// Texels of a full chain 2^n, 2^(n-1), ..., 1.
inline int64_t htex_chain_texels(int n) {
    return ((int64_t(1) << (2 * n + 2)) - 1) / 3;
}

// Texel offset of level l inside a chain of base 2^n.
inline int64_t htex_level_texels(int n, int l) {
    return ((int64_t(1) << (2 * n + 2)) - (int64_t(1) << (2 * (n - l) + 2))) / 3;
}

// Byte offsets of every texture in the pool; returns total bytes.
int64_t htex_pool_offsets(int32_t E, const int32_t* log2n, int32_t C, htex_dtype dt,
                          int64_t* offsets /* [E+1], nullable */);

// Stream-ordered scratch memory of the library: one pool per device that
// keeps its memory between calls (lookup.cu).
cudaMemPool_t htex_scratch_pool(int device);

// log2 of the halfedges per sort range so that a range's textures take
// about 32 MB; -1 when the pool is too small for sorting to pay (lookup.cu).
int htex_bin_shift(const htex_textures* t);

// Kernel launchers (lookup.cu, backward.cu).  They validate nothing: the
// C-ABI entry points have checked every argument.
htex_status htex_launch_lookup(const htex_textures* t, const htex_query* q, int64_t n,
                               float* out, uint32_t flags, htex_stream stream,
                               int32_t* d_status);
// flags: kBackwardAggregate merges the scatter-adds of lanes of a warp that
// hit the same texels (for sorted queries); other bits are ignored.
constexpr uint32_t kBackwardAggregate = 1u << 16;
htex_status htex_launch_backward(const htex_textures* t, const htex_query* q, int64_t n,
                                 const float* grad_out, float* grad_texels, uint32_t flags,
                                 htex_stream stream, int32_t* d_status);
// The adjoint on queries sorted by halfedge range (HTEX_LOOKUP_BIN), chunk
// by chunk, with warp-aggregated atomics (lookup.cu).  Falls back to the
// unsorted adjoint for pools that fit L2.
htex_status htex_launch_backward_sorted(const htex_textures* t, const htex_query* q, int64_t n,
                                        const float* grad_out, float* grad_texels, htex_stream stream,
                                        int32_t* d_status);
