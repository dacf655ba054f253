// Forward filtered lookup (paper Section 4.4, Alg. 3 with Alg. 2): query
// binning, the launch paths and the htex_lookup entry points.  The filter
// kernels themselves are in lookup_kernels.cuh, instantiated per texel
// format in lookup_<format>.cu.
//
// One thread per query in a grid-stride loop over a persistent grid.  Per
// query: one streaming 16-byte query load, one 16-byte packed record
// (edges and Alg. 2 reflections of h, Next(h), Prev(h)), then up to three
// fetches, each one or two levels of 2x2 border-aware taps; a fetch whose
// taps all fall outside its texture loads nothing.  Two memory paths: the
// pool gathered through the read-only cache from global memory (queries
// two iterations and records one iteration ahead in flight), or staged in
// shared memory for small assets and many queries (two queries per thread
// and iteration).  Both come in a variant for assets whose textures share
// one resolution, which keeps everything derived from it warp-uniform, and
// use 32-bit indices when the query count allows.
//
// Binning (HTEX_LOOKUP_BIN), for pools well beyond L2: the queries are
// counting-sorted into 128 ranges of consecutive halfedges, in chunks of
// 2^24 queries, before filtering.  The filter kernel then works through
// one range of the asset at a time, so that a texel sector fetched for one
// query is still in L2 when the queries next to it in the range need it;
// the ranges' order matters, the order inside a range does not.  The
// results are filtered into a sorted copy and gathered back into query
// order.  The allocation-free variant sorts the whole batch at once into
// ranges sized by texel bytes and stores results through the indices.
#include <algorithm>
#include <mutex>

#include <cuda_runtime.h>

#include "lookup_kernels.cuh"
#include "aniso_launch.h"

namespace htex {

// ------------------------------------------------------------------ binning

constexpr int kBinThreads = 256;
constexpr int kBinPerThread = 8;
constexpr int kMaxBuckets = 4096;

__device__ __forceinline__ uint32_t bucket_of(int32_t h, int32_t H, int shift, uint32_t invalid) {
    return unsigned(h) < unsigned(H) ? uint32_t(h) >> shift : invalid;
}

// Pass 1: bucket sizes (shared-memory histogram per block, then global adds).
__global__ void __launch_bounds__(kBinThreads) k_bin_count(const htex_query* q, int64_t n, int32_t H, int shift,
                                                           uint32_t B, uint32_t* counts) {
    __shared__ uint32_t hist[kMaxBuckets + 1];
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t h = __ldcs(reinterpret_cast<const int32_t*>(q + i));
        atomicAdd(&hist[bucket_of(h, H, shift, B - 1)], 1u);
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x)
        if (hist[b]) atomicAdd(&counts[b], hist[b]);
}

// Pass 2: every block derives the bucket offsets from the counts (an
// exclusive scan of at most 4097 values), then places tiles of
// kBinThreads * kBinPerThread queries: a block-local histogram and ranks,
// one global reservation per (tile, bucket), and the writes of the
// queries and their original indices into their bucket's range.
__global__ void __launch_bounds__(kBinThreads) k_bin_scatter(const htex_query* q, int64_t n, int32_t H, int shift,
                                                             uint32_t B, const uint32_t* counts, uint32_t* taken,
                                                             htex_query* qs, int32_t* idx) {
    __shared__ uint32_t offset[kMaxBuckets + 1];
    __shared__ uint32_t cnt[kMaxBuckets + 1];
    __shared__ uint32_t base[kMaxBuckets + 1];
    __shared__ uint32_t warp_tot[kBinThreads / 32];
    // exclusive scan of counts: each thread a contiguous chunk
    const uint32_t per = (B + kBinThreads - 1) / kBinThreads;
    const uint32_t lo = min(B, threadIdx.x * per), hi = min(B, lo + per);
    uint32_t run = 0;
    for (uint32_t b = lo; b < hi; ++b) run += counts[b];
    uint32_t incl = run;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += o;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    uint32_t prefix = incl - run;
    for (int w = 0; w < warp; ++w) prefix += warp_tot[w];
    for (uint32_t b = lo; b < hi; ++b) {
        offset[b] = prefix;
        prefix += counts[b];
    }
    __syncthreads();

    constexpr int TILE = kBinThreads * kBinPerThread;
    for (int64_t t0 = int64_t(blockIdx.x) * TILE; t0 < n; t0 += int64_t(gridDim.x) * TILE) {
        for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) cnt[b] = 0;
        __syncthreads();
        int4 r[kBinPerThread];
        uint32_t bk[kBinPerThread], rank[kBinPerThread];
#pragma unroll
        for (int k = 0; k < kBinPerThread; ++k) {
            const int64_t i = t0 + int64_t(k) * kBinThreads + threadIdx.x;
            if (i < n) {
                r[k] = __ldcs(reinterpret_cast<const int4*>(q) + i);
                bk[k] = bucket_of(r[k].x, H, shift, B - 1);
                rank[k] = atomicAdd(&cnt[bk[k]], 1u);
            }
        }
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < B; b += blockDim.x)
            if (cnt[b]) base[b] = offset[b] + atomicAdd(&taken[b], cnt[b]);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kBinPerThread; ++k) {
            const int64_t i = t0 + int64_t(k) * kBinThreads + threadIdx.x;
            if (i < n) {
                const uint32_t pos = base[bk[k]] + rank[k];
                reinterpret_cast<int4*>(qs)[pos] = r[k];
                idx[pos] = int32_t(i);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------ chunk-local sort (HTEX_LOOKUP_BIN)
//
// One chunk of m queries at a time: a bucket histogram, then per tile of
// kSortThreads x kSortPer queries (fewer per thread for wider queries or a
// payload) a local counting sort in shared memory, so that every
// bucket's run of the tile is written to the sorted copy as one contiguous
// piece (whole sectors, not scattered 16-byte pieces), and each query's
// sorted position is recorded in query order.  The lookup then filters the
// sorted copy with coalesced result stores, and the gather puts every
// result back in query order through the recorded positions.

constexpr int kSortThreads = 256;
constexpr int kSortPer = 8;   // 16-byte query words per thread and tile (16: 8% slower sort, measured)
constexpr int kSortMaxBuckets = 256;

// QW: 16-byte words per query (1: htex_query, 2: htex_query_aniso); the
// halfedge id is the first word's first int.
template <int QW>
__global__ void __launch_bounds__(kSortThreads) k_chunk_count(const int4* q, int64_t m, int32_t H, int shift,
                                                              uint32_t B, uint32_t* counts) {
    constexpr int PER = kSortPer / QW, TILE = kSortThreads * PER;
    __shared__ uint32_t hist[kSortMaxBuckets];
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (int64_t t0 = int64_t(blockIdx.x) * TILE; t0 < m; t0 += int64_t(gridDim.x) * TILE) {
        int32_t h[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int64_t i = t0 + int64_t(k) * kSortThreads + threadIdx.x;
            h[k] = i < m ? __ldg(reinterpret_cast<const int32_t*>(q + i * QW)) : 0;
        }
#pragma unroll
        for (int k = 0; k < PER; ++k)
            if (t0 + int64_t(k) * kSortThreads + threadIdx.x < m) atomicAdd(&hist[bucket_of(h[k], H, shift, B - 1)], 1u);
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x)
        if (hist[b]) atomicAdd(&counts[b], hist[b]);
}

// Exclusive scan of x[0..B) into y (shared memory), each thread a
// contiguous piece; returns nothing, ends with a barrier.
__device__ __forceinline__ void block_scan_buckets(const uint32_t* x, uint32_t* y, uint32_t B, uint32_t* warp_tot) {
    const uint32_t per = (B + kSortThreads - 1) / kSortThreads;
    const uint32_t lo = min(B, threadIdx.x * per), hi = min(B, lo + per);
    uint32_t run = 0;
    for (uint32_t b = lo; b < hi; ++b) run += x[b];
    uint32_t incl = run;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += o;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    uint32_t prefix = incl - run;
    for (int w = 0; w < warp; ++w) prefix += warp_tot[w];
    for (uint32_t b = lo; b < hi; ++b) {
        const uint32_t c = x[b];
        y[b] = prefix;
        prefix += c;
    }
    __syncthreads();
}

// PC: floats of payload per query (rows of 'pay' in query order, moved to
// 'spay' in sorted order with their queries); pos nullable.
// Shared memory of k_chunk_scatter<QW, PC> (dynamic: a tile can exceed the
// 48 KiB of static shared memory): the tile's queries (QW words each) and
// payload rows, their buckets, and per bucket the first sorted position,
// the tile's count, local offset and global base.
template <int QW, int PC>
struct ScatterSmem {
    static constexpr int PER = kSortPer / QW / (PC > 0 ? 2 : 1), TILE = kSortThreads * PER;
    static constexpr size_t tile = 0;
    static constexpr size_t pay = tile + size_t(TILE) * QW * 16;
    static constexpr size_t bucket = pay + ((size_t(PC > 0 ? TILE * PC : 1) * 4 + 15) & ~size_t(15));
    static constexpr size_t arrays = bucket + ((size_t(TILE) * 2 + 15) & ~size_t(15));
    static constexpr size_t warps = arrays + size_t(4) * kSortMaxBuckets * 4;
    static constexpr size_t bytes = warps + (kSortThreads / 32) * 4;
};

template <int QW, int PC>
__global__ void __launch_bounds__(kSortThreads) k_chunk_scatter(const int4* q, int64_t m, int32_t H, int shift,
                                                                uint32_t B, const uint32_t* counts, uint32_t* taken,
                                                                int4* sq, int32_t* pos, int32_t pos_base,
                                                                const float* pay, float* spay) {
    using L = ScatterSmem<QW, PC>;
    constexpr int PER = L::PER, TILE = L::TILE;
    extern __shared__ __align__(16) uint8_t smem[];
    int4* tile = reinterpret_cast<int4*>(smem + L::tile);
    float* tile_pay = reinterpret_cast<float*>(smem + L::pay);
    uint16_t* tile_bucket = reinterpret_cast<uint16_t*>(smem + L::bucket);
    uint32_t* start = reinterpret_cast<uint32_t*>(smem + L::arrays);   // first sorted position of each bucket
    uint32_t* cnt = start + kSortMaxBuckets;                             // the tile's bucket sizes
    uint32_t* loff = cnt + kSortMaxBuckets;                              // the tile's local bucket offsets
    uint32_t* gbase = loff + kSortMaxBuckets;                            // where the tile's run of each bucket goes
    uint32_t* warp_tot = reinterpret_cast<uint32_t*>(smem + L::warps);
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) cnt[b] = counts[b];
    __syncthreads();
    block_scan_buckets(cnt, start, B, warp_tot);

    for (int64_t t0 = int64_t(blockIdx.x) * TILE; t0 < m; t0 += int64_t(gridDim.x) * TILE) {
        const int tm = int(min(int64_t(TILE), m - t0));
        for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) cnt[b] = 0;
        __syncthreads();
        int4 r[PER][QW];
        float pv[PER][PC > 0 ? PC : 1];
        uint32_t bk[PER], rank[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int j = k * kSortThreads + threadIdx.x;
#pragma unroll
            for (int w = 0; w < QW; ++w)
                if (j < tm) r[k][w] = __ldcs(q + (t0 + j) * QW + w);
#pragma unroll
            for (int c = 0; c < PC; ++c)
                if (j < tm) pv[k][c] = __ldcs(pay + (t0 + j) * PC + c);
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            if (k * kSortThreads + int(threadIdx.x) < tm) {
                bk[k] = bucket_of(r[k][0].x, H, shift, B - 1);
                rank[k] = atomicAdd(&cnt[bk[k]], 1u);
            }
        }
        __syncthreads();
        block_scan_buckets(cnt, loff, B, warp_tot);
        for (uint32_t b = threadIdx.x; b < B; b += blockDim.x)
            if (cnt[b]) gbase[b] = start[b] + atomicAdd(&taken[b], cnt[b]);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int j = k * kSortThreads + threadIdx.x;
            if (j < tm) {
                const uint32_t lp = loff[bk[k]] + rank[k];
#pragma unroll
                for (int w = 0; w < QW; ++w) tile[lp * QW + w] = r[k][w];
#pragma unroll
                for (int c = 0; c < PC; ++c) tile_pay[lp * PC + c] = pv[k][c];
                tile_bucket[lp] = uint16_t(bk[k]);
                if (pos) __stcs(pos + t0 + j, pos_base + int32_t(gbase[bk[k]] + rank[k]));
            }
        }
        __syncthreads();
        for (int x = threadIdx.x; x < tm * QW; x += kSortThreads) {   // one 16-byte word per thread
            const int j = x / QW, w = x - j * QW;
            const uint32_t b = tile_bucket[j];
            sq[int64_t(gbase[b] + (uint32_t(j) - loff[b])) * QW + w] = tile[x];
        }
        if constexpr (PC > 0) {
            for (int x = threadIdx.x; x < tm * PC; x += kSortThreads) {
                const int j = x / PC, c = x - j * PC;
                const uint32_t b = tile_bucket[j];
                spay[int64_t(gbase[b] + (uint32_t(j) - loff[b])) * PC + c] = tile_pay[x];
            }
        }
        __syncthreads();
    }
}

// Results back in query order: out[i] = sorted_out[pos[i]] (NaN where
// pos[i] is not in [0, m)).  Each thread has kGatherRows rows in flight:
// all their positions, then all their loads, then all their stores (a
// store between two loads would keep the second load from being issued
// early, since the compiler cannot prove the rows do not overlap).
constexpr int kGatherRows = 8;

template <int C>
__global__ void k_chunk_gather(const float* __restrict__ sout, const int32_t* __restrict__ pos, int64_t m,
                               float* __restrict__ out) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i0 < m; i0 += kGatherRows * stride) {
        int64_t p[kGatherRows];
#pragma unroll
        for (int k = 0; k < kGatherRows; ++k) {
            const int64_t i = i0 + k * stride;
            p[k] = i < m ? int64_t(__ldcs(pos + i)) : -1;
        }
        float v[kGatherRows][C];
#pragma unroll
        for (int k = 0; k < kGatherRows; ++k) {
            const bool ok = uint64_t(p[k]) < uint64_t(m);   // else not a position of this batch: NaN, no read
            if constexpr (C == 4) {
                const float4 r = ok ? __ldcg(reinterpret_cast<const float4*>(sout) + p[k])
                                    : make_float4(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000),
                                                  __int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
                v[k][0] = r.x; v[k][1] = r.y; v[k][2] = r.z; v[k][3] = r.w;
            } else if constexpr (C == 2) {
                const float2 r = ok ? __ldcg(reinterpret_cast<const float2*>(sout) + p[k])
                                    : make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
                v[k][0] = r.x; v[k][1] = r.y;
            } else {
#pragma unroll
                for (int c = 0; c < C; ++c) v[k][c] = ok ? __ldcg(sout + p[k] * C + c) : __int_as_float(0x7fc00000);
            }
        }
#pragma unroll
        for (int k = 0; k < kGatherRows; ++k) {
            const int64_t i = i0 + k * stride;
            if (i >= m) break;
            if constexpr (C == 4) {
                __stcs(reinterpret_cast<float4*>(out) + i, make_float4(v[k][0], v[k][1], v[k][2], v[k][3]));
            } else if constexpr (C == 2) {
                __stcs(reinterpret_cast<float2*>(out) + i, make_float2(v[k][0], v[k][1]));
            } else {
#pragma unroll
                for (int c = 0; c < C; ++c) __stcs(out + i * C + c, v[k][c]);
            }
        }
    }
}

}  // namespace htex

using namespace htex;

namespace {

#ifndef HTEX_SORT_CHUNK_LOG2
#define HTEX_SORT_CHUNK_LOG2 24
#endif
#ifndef HTEX_CHUNK_BUCKETS
#define HTEX_CHUNK_BUCKETS 128
#endif
constexpr int64_t kSortChunk = int64_t(1) << HTEX_SORT_CHUNK_LOG2;   // queries per L2-resident chunk
constexpr int64_t kChunkBuckets = HTEX_CHUNK_BUCKETS;                // halfedge ranges a chunk is sorted into

constexpr int64_t kBucketTexelBytes = int64_t(32) << 20;

template <bool BINNED>
htex_status launch_fwd_dt(const htex_textures* t, const FwdParams& p, uint32_t flags, cudaStream_t s) {
    switch (t->dtype) {
    case HTEX_F32: return launch_fwd_f32(t, p, flags, s, BINNED);
    case HTEX_U8: return launch_fwd_u8(t, p, flags, s, BINNED);
    case HTEX_F16: return launch_fwd_f16(t, p, flags, s, BINNED);
    case HTEX_BF16: return launch_fwd_bf16(t, p, flags, s, BINNED);
    case HTEX_E4M3: return launch_fwd_e4m3(t, p, flags, s, BINNED);
    }
    return HTEX_ERR_INVALID_ARG;
}

}  // namespace

cudaMemPool_t htex_scratch_pool(int device) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    std::lock_guard<std::mutex> g(mu);
    if (device < 0 || device >= 64) return nullptr;
    if (!pools[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        uint64_t keep = ~uint64_t(0);
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[device] = p;
    }
    return pools[device];
}

namespace {

}  // namespace

// Halfedges per bucket (log2) so one bucket's textures take about
// kBucketTexelBytes; returns -1 when the asset is too small to gain.
int htex_bin_shift(const htex_textures* t) {
    if (t->H <= 0 || t->pool_bytes <= 2 * kBucketTexelBytes) return -1;
    const int64_t buckets = std::min<int64_t>(kMaxBuckets, (t->pool_bytes + kBucketTexelBytes - 1) / kBucketTexelBytes);
    int shift = 0;
    while ((int64_t(t->H) >> shift) + 1 > buckets) ++shift;
    return shift;
}

namespace {

// Buckets of 2^shift consecutive halfedges, at most kChunkBuckets, plus the
// bucket of invalid queries.
struct SortPlan {
    int shift;
    uint32_t B;
};

SortPlan sort_plan(int32_t H) {
    static_assert(kChunkBuckets + 1 <= kSortMaxBuckets, "bucket arrays too small");
    SortPlan P{0, 0};
    while ((int64_t(H) >> P.shift) + 1 > kChunkBuckets) ++P.shift;
    P.B = uint32_t((int64_t(H) >> P.shift) + 2);
    return P;
}

size_t counter_bytes(const SortPlan& P) { return (size_t(2 * P.B) * 4 + 255) & ~size_t(255); }

// Sorts q[0..m) into sq within consecutive chunks of kSortChunk queries;
// pos[i] = where query i went (nullable); PC floats of payload per query
// follow their queries from pay to spay.  counters: counter_bytes(P) of
// scratch.  QW: 16-byte words per query.
template <int QW, int PC = 0>
htex_status launch_sort(const htex_textures* t, const SortPlan& P, const int4* q, int64_t m, uint32_t* counters,
                        int4* sq, int32_t* pos, cudaStream_t s, const float* pay = nullptr, float* spay = nullptr) {
    constexpr int64_t TILE = ScatterSmem<QW, PC>::TILE;
    constexpr size_t smem = ScatterSmem<QW, PC>::bytes;
    if (cudaFuncSetAttribute(k_chunk_scatter<QW, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
        cudaSuccess)
        return HTEX_ERR_CUDA;
    const int64_t blocks = int64_t(t->num_sms) * resident_blocks(k_chunk_scatter<QW, PC>, kSortThreads, smem);
    for (int64_t c0 = 0; c0 < m; c0 += kSortChunk) {
        const int64_t mc = std::min<int64_t>(kSortChunk, m - c0);
        const int64_t g = std::min<int64_t>((mc + TILE - 1) / TILE, blocks);
        if (cudaMemsetAsync(counters, 0, size_t(2 * P.B) * 4, s) != cudaSuccess) return HTEX_ERR_CUDA;
        k_chunk_count<QW><<<unsigned(g), kSortThreads, 0, s>>>(q + c0 * QW, mc, t->H, P.shift, P.B, counters);
        k_chunk_scatter<QW, PC><<<unsigned(g), kSortThreads, smem, s>>>(
            q + c0 * QW, mc, t->H, P.shift, P.B, counters, counters + P.B, sq + c0 * QW, pos ? pos + c0 : nullptr,
            int32_t(c0), PC ? pay + c0 * PC : nullptr, PC ? spay + c0 * PC : nullptr);
        if (cudaGetLastError() != cudaSuccess) return HTEX_ERR_CUDA;
    }
    return HTEX_OK;
}

inline const int4* words(const htex_query* q) { return reinterpret_cast<const int4*>(q); }
inline int4* words(htex_query* q) { return reinterpret_cast<int4*>(q); }

// Gathers the results of a chunk back into query order.  Positions are
// relative to the sorted chunk.
htex_status launch_gather(const float* sout, const int32_t* pos, int64_t m, int C, float* out, cudaStream_t s) {
    // one block per 256 x kGatherRows rows (no grid-stride pass: the last
    // wave balances better; 6% faster than 8 blocks per SM striding)
    const unsigned g = unsigned(std::max<int64_t>(1, (m + 256 * kGatherRows - 1) / (256 * kGatherRows)));
    switch (C) {
    case 1: k_chunk_gather<1><<<g, 256, 0, s>>>(sout, pos, m, out); break;
    case 2: k_chunk_gather<2><<<g, 256, 0, s>>>(sout, pos, m, out); break;
    case 3: k_chunk_gather<3><<<g, 256, 0, s>>>(sout, pos, m, out); break;
    case 4: k_chunk_gather<4><<<g, 256, 0, s>>>(sout, pos, m, out); break;
    default: return HTEX_ERR_INVALID_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? HTEX_OK : HTEX_ERR_CUDA;
}

}  // namespace

htex_status htex_launch_lookup(const htex_textures* t, const htex_query* q, int64_t n, float* out,
                               uint32_t flags, htex_stream stream, int32_t* d_status) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!(flags & HTEX_LOOKUP_BIN) || htex_bin_shift(t) < 0)
        return launch_fwd_dt<false>(t, FwdParams{q, n, out, d_status, nullptr}, flags, s);

    // one chunk at a time: sort, filter into the sorted copy, gather back
    // (storing each result straight to its query's row from the filter
    // instead was measured slower: scattered 16-byte stores leave partly
    // written sectors that DRAM has to merge)
    const SortPlan P = sort_plan(t->H);
    const int64_t M = std::min<int64_t>(n, kSortChunk);
    const size_t cnt_b = counter_bytes(P);
    const size_t sq_b = size_t(M) * 16, pos_b = (size_t(M) * 4 + 255) & ~size_t(255);
    const size_t sout_b = size_t(M) * 4 * size_t(t->C);
    cudaMemPool_t pool = htex_scratch_pool(t->device);
    if (!pool) return HTEX_ERR_CUDA;
    void* scratch = nullptr;
    if (cudaMallocFromPoolAsync(&scratch, cnt_b + sq_b + pos_b + sout_b, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    uint8_t* base = static_cast<uint8_t*>(scratch);
    uint32_t* counters = reinterpret_cast<uint32_t*>(base);
    htex_query* sq = reinterpret_cast<htex_query*>(base + cnt_b);
    int32_t* pos = reinterpret_cast<int32_t*>(base + cnt_b + sq_b);
    float* sout = reinterpret_cast<float*>(base + cnt_b + sq_b + pos_b);
    const uint32_t fwd_flags = flags & ~uint32_t(HTEX_LOOKUP_BIN);
    htex_status st = HTEX_OK;
    for (int64_t c0 = 0; c0 < n && st == HTEX_OK; c0 += M) {
        const int64_t m = std::min<int64_t>(M, n - c0);
        st = launch_sort<1>(t, P, words(q + c0), m, counters, words(sq), pos, s);
        if (st == HTEX_OK) st = launch_fwd_dt<false>(t, FwdParams{sq, m, sout, d_status, nullptr}, fwd_flags, s);
        if (st == HTEX_OK) st = launch_gather(sout, pos, m, t->C, out + c0 * t->C, s);
    }
    cudaFreeAsync(scratch, s);
    return st;
}

template <int C>
htex_status launch_sort_rows(const htex_textures* t, const SortPlan& P, const htex_query* q, int64_t m,
                             const float* g, uint32_t* counters, htex_query* sq, float* sg, cudaStream_t s) {
    return launch_sort<1, C>(t, P, words(q), m, counters, words(sq), nullptr, s, g, sg);
}

// The adjoint on sorted queries: each chunk sorted by halfedge range with
// its upstream gradient rows moving along (in the scatter's tiles, so they
// leave in whole runs like the queries), then the warp-aggregated adjoint
// over the sorted copy.
htex_status htex_launch_backward_sorted(const htex_textures* t, const htex_query* q, int64_t n,
                                        const float* grad_out, float* grad_texels, htex_stream stream,
                                        int32_t* d_status) {
    if (htex_bin_shift(t) < 0) return htex_launch_backward(t, q, n, grad_out, grad_texels, 0u, stream, d_status);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const SortPlan P = sort_plan(t->H);
    const int64_t M = std::min<int64_t>(n, kSortChunk);
    const size_t cnt_b = counter_bytes(P);
    const size_t sq_b = size_t(M) * 16, g_b = size_t(M) * 4 * size_t(t->C);
    cudaMemPool_t pool = htex_scratch_pool(t->device);
    if (!pool) return HTEX_ERR_CUDA;
    void* scratch = nullptr;
    if (cudaMallocFromPoolAsync(&scratch, cnt_b + sq_b + g_b, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    uint8_t* base = static_cast<uint8_t*>(scratch);
    uint32_t* counters = reinterpret_cast<uint32_t*>(base);
    htex_query* sq = reinterpret_cast<htex_query*>(base + cnt_b);
    float* gs = reinterpret_cast<float*>(base + cnt_b + sq_b);
    htex_status st = HTEX_OK;
    for (int64_t c0 = 0; c0 < n && st == HTEX_OK; c0 += M) {
        const int64_t m = std::min<int64_t>(M, n - c0);
        const float* gsrc = grad_out + c0 * t->C;
        switch (t->C) {
        case 1: st = launch_sort_rows<1>(t, P, q + c0, m, gsrc, counters, sq, gs, s); break;
        case 2: st = launch_sort_rows<2>(t, P, q + c0, m, gsrc, counters, sq, gs, s); break;
        case 3: st = launch_sort_rows<3>(t, P, q + c0, m, gsrc, counters, sq, gs, s); break;
        default: st = launch_sort_rows<4>(t, P, q + c0, m, gsrc, counters, sq, gs, s); break;
        }
        if (st == HTEX_OK)
            st = htex_launch_backward(t, sq, m, gs, grad_texels, kBackwardAggregate, stream, d_status);
    }
    cudaFreeAsync(scratch, s);
    return st;
}

htex_status htex_launch_aniso_sorted(const htex_textures* t, const htex_query_aniso* q, int64_t n, int32_t kmax,
                                     float* out, htex_stream stream, int32_t* d_status) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (htex_bin_shift(t) < 0) return htex_launch_aniso(t, q, n, kmax, out, stream, d_status);
    const SortPlan P = sort_plan(t->H);
    const int64_t M = std::min<int64_t>(n, kSortChunk);
    const size_t cnt_b = counter_bytes(P);
    const size_t sq_b = size_t(M) * sizeof(htex_query_aniso), pos_b = (size_t(M) * 4 + 255) & ~size_t(255);
    const size_t sout_b = size_t(M) * 4 * size_t(t->C);
    cudaMemPool_t pool = htex_scratch_pool(t->device);
    if (!pool) return HTEX_ERR_CUDA;
    void* scratch = nullptr;
    if (cudaMallocFromPoolAsync(&scratch, cnt_b + sq_b + pos_b + sout_b, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    uint8_t* base = static_cast<uint8_t*>(scratch);
    uint32_t* counters = reinterpret_cast<uint32_t*>(base);
    htex_query_aniso* sq = reinterpret_cast<htex_query_aniso*>(base + cnt_b);
    int32_t* pos = reinterpret_cast<int32_t*>(base + cnt_b + sq_b);
    float* sout = reinterpret_cast<float*>(base + cnt_b + sq_b + pos_b);
    htex_status st = HTEX_OK;
    for (int64_t c0 = 0; c0 < n && st == HTEX_OK; c0 += M) {
        const int64_t m = std::min<int64_t>(M, n - c0);
        st = launch_sort<2>(t, P, reinterpret_cast<const int4*>(q + c0), m, counters, reinterpret_cast<int4*>(sq),
                            pos, s);
        if (st == HTEX_OK) st = htex_launch_aniso(t, sq, m, kmax, sout, stream, d_status);
        if (st == HTEX_OK) st = launch_gather(sout, pos, m, t->C, out + c0 * t->C, s);
    }
    cudaFreeAsync(scratch, s);
    return st;
}

extern "C" htex_status htex_queries_sort(const htex_textures* t, const htex_query* q, int64_t n,
                                         htex_query* sorted, int32_t* pos, htex_stream stream) {
    if (!t || n < 0 || n > int64_t(INT32_MAX)) return HTEX_ERR_INVALID_ARG;
    if (n == 0) return HTEX_OK;
    if (!q || !sorted || !pos) return HTEX_ERR_INVALID_ARG;
    if (((reinterpret_cast<uintptr_t>(q) | reinterpret_cast<uintptr_t>(sorted)) & 15u) != 0 ||
        (reinterpret_cast<uintptr_t>(pos) & 3u) != 0)
        return HTEX_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const SortPlan P = sort_plan(t->H);
    cudaMemPool_t pool = htex_scratch_pool(t->device);
    if (!pool) return HTEX_ERR_CUDA;
    void* counters = nullptr;
    if (cudaMallocFromPoolAsync(&counters, counter_bytes(P), pool, s) != cudaSuccess) {
        cudaGetLastError();
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    const htex_status st =
        launch_sort<1>(t, P, words(q), n, static_cast<uint32_t*>(counters), words(sorted), pos, s);
    cudaFreeAsync(counters, s);
    return st;
}

extern "C" htex_status htex_results_gather(const float* sorted_out, const int32_t* pos, int64_t n, int32_t channels,
                                           float* out, htex_stream stream) {
    if (n < 0 || n > int64_t(INT32_MAX) || channels < 1 || channels > 4) return HTEX_ERR_INVALID_ARG;
    if (n == 0) return HTEX_OK;
    if (!sorted_out || !pos || !out) return HTEX_ERR_INVALID_ARG;
    const uintptr_t align = channels == 4 ? 16u : (channels == 2 ? 8u : 4u);
    if (((reinterpret_cast<uintptr_t>(sorted_out) | reinterpret_cast<uintptr_t>(out)) & (align - 1)) != 0 ||
        (reinterpret_cast<uintptr_t>(pos) & 3u) != 0)
        return HTEX_ERR_INVALID_ARG;
    return launch_gather(sorted_out, pos, n, channels, out, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" htex_status htex_lookup(const htex_textures* t, const htex_query* q, int64_t n, float* out,
                                   uint32_t flags, htex_stream stream, int32_t* d_status) {
    if (!t || n < 0) return HTEX_ERR_INVALID_ARG;
    if (flags & ~uint32_t(HTEX_LOOKUP_BIN | HTEX_LOOKUP_GLOBAL)) return HTEX_ERR_INVALID_ARG;
    if (n == 0) return HTEX_OK;
    if (!q || !out) return HTEX_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(q) & 15u) != 0) return HTEX_ERR_INVALID_ARG;
    const uintptr_t out_align = t->C == 4 ? 16u : (t->C == 2 ? 8u : 4u);
    if ((reinterpret_cast<uintptr_t>(out) & (out_align - 1)) != 0) return HTEX_ERR_INVALID_ARG;
    return htex_launch_lookup(t, q, n, out, flags, stream, d_status);
}

// ------------------------------------------------- allocation-free variant
//
// htex_lookup_noalloc: the binned lookup for callers that must not
// allocate device memory, e.g. a host application or engine that owns
// every device allocation and forbids its plug-ins to make their own, or a
// frame loop that cannot absorb the device-wide synchronisation cudaMalloc
// and cudaFree may cause.  Its scratch (sorted queries, their original
// indices, bucket counters) lives in one fixed file-scope device array
// that every device which loads this library holds until the process
// exits.  Host code cannot use the array's name as a device address, so
// the address is fetched once per device with cudaGetSymbolAddress.

namespace {

constexpr int64_t kNoAllocMaxQueries = int64_t(1) << 20;
constexpr size_t kNoAllocQueryBytes = size_t(kNoAllocMaxQueries) * 16;
constexpr size_t kNoAllocIndexBytes = size_t(kNoAllocMaxQueries) * 4;
constexpr size_t kNoAllocCountBytes = size_t(kMaxBuckets + 2) * 4;
constexpr size_t kNoAllocBytes = kNoAllocQueryBytes + kNoAllocIndexBytes + 2 * kNoAllocCountBytes;

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch for the current device, looked up on
// the first call made with that device current.
htex_status noalloc_scratch(int device, uint8_t** out) {
    static std::mutex mu;
    static void* addr[64] = {};
    if (device < 0 || device >= 64) return HTEX_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> g(mu);
    if (!addr[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HTEX_ERR_CUDA;
        }
        addr[device] = p;
    }
    *out = static_cast<uint8_t*>(addr[device]);
    return HTEX_OK;
}

}  // namespace

extern "C" int64_t htex_lookup_noalloc_max_queries(void) { return kNoAllocMaxQueries; }

extern "C" htex_status htex_lookup_noalloc(const htex_textures* t, const htex_query* q, int64_t n, float* out,
                                           htex_stream stream, int32_t* d_status) {
    if (!t || n < 0) return HTEX_ERR_INVALID_ARG;
    if (n == 0) return HTEX_OK;
    if (!q || !out) return HTEX_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(q) & 15u) != 0) return HTEX_ERR_INVALID_ARG;
    const uintptr_t out_align = t->C == 4 ? 16u : (t->C == 2 ? 8u : 4u);
    if ((reinterpret_cast<uintptr_t>(out) & (out_align - 1)) != 0) return HTEX_ERR_INVALID_ARG;
    if (n > kNoAllocMaxQueries) return HTEX_ERR_UNSUPPORTED;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) return HTEX_ERR_CUDA;
    if (device != t->device) return HTEX_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int shift = htex_bin_shift(t);
    if (shift < 0) return launch_fwd_dt<false>(t, FwdParams{q, n, out, d_status, nullptr}, 0u, s);

    uint8_t* base = nullptr;
    htex_status st = noalloc_scratch(device, &base);
    if (st != HTEX_OK) return st;
    const uint32_t B = uint32_t((int64_t(t->H) >> shift) + 2);
    htex_query* qs = reinterpret_cast<htex_query*>(base);
    int32_t* idx = reinterpret_cast<int32_t*>(base + kNoAllocQueryBytes);
    uint32_t* counts = reinterpret_cast<uint32_t*>(base + kNoAllocQueryBytes + kNoAllocIndexBytes);
    uint32_t* taken = counts + (kMaxBuckets + 2);
    // the array keeps the previous call's contents: clear both counter sets
    if (cudaMemsetAsync(counts, 0, 2 * kNoAllocCountBytes, s) != cudaSuccess) return HTEX_ERR_CUDA;
    const int64_t g1 = std::min<int64_t>((n + kBinThreads - 1) / kBinThreads, int64_t(t->num_sms) * 4);
    k_bin_count<<<unsigned(g1), kBinThreads, 0, s>>>(q, n, t->H, shift, B, counts);
    const int64_t tile = int64_t(kBinThreads) * kBinPerThread;
    const int64_t g2 = std::min<int64_t>((n + tile - 1) / tile, int64_t(t->num_sms) * 2);
    k_bin_scatter<<<unsigned(g2), kBinThreads, 0, s>>>(q, n, t->H, shift, B, counts, taken, qs, idx);
    if (cudaGetLastError() != cudaSuccess) return HTEX_ERR_CUDA;
    return launch_fwd_dt<true>(t, FwdParams{qs, n, out, d_status, idx}, 0u, s);
}
