// Filter kernels of htex_lookup (paper Section 4.4, Alg. 3 with Alg. 2)
// and their launchers, instantiated per texel format in lookup_<format>.cu
// so that the formats compile in parallel.  See lookup.cu for the paths.
#pragma once

#include <algorithm>

#include <cuda_runtime.h>

#include "lookup_core.cuh"

namespace htex {

template <bool BINNED, class I>
__device__ __forceinline__ int64_t dst_of(const FwdParams& p, I i) {
    return BINNED ? int64_t(__ldcs(p.idx + i)) : i;
}

// Grid-stride loop for the global path, software-pipelined: the query two
// iterations ahead and the record one iteration ahead are in flight while
// the current query's texels are gathered.  I: the index type (32-bit when
// n allows); UNI: every texture has one resolution.
template <int DT, int C, bool BINNED, bool DEFER, bool UNI, class I, class S>
__device__ __forceinline__ void lookup_loop(const Asset<S>& A, const FwdParams& p) {
    const I n = I(p.n);
    const I stride = I(gridDim.x) * I(blockDim.x);
    I i0 = I(blockIdx.x) * I(blockDim.x) + I(threadIdx.x);
    if (i0 >= n) return;
    I i1 = i0 + stride;
    int4 raw0 = ld_query(p.q, i0);
    int64_t dst0 = dst_of<BINNED>(p, i0);
    int4 raw1 = make_int4(-1, 0, 0, 0);
    int64_t dst1 = 0;
    if (i1 < n) {
        raw1 = ld_query(p.q, i1);
        dst1 = dst_of<BINNED>(p, i1);
    }
    uint4 rec0 = record_of(A, raw0);
    while (true) {
        const I i2 = i1 + stride;
        int4 raw2 = make_int4(-1, 0, 0, 0);
        int64_t dst2 = 0;
        if (i2 < n) {
            raw2 = ld_query(p.q, i2);
            dst2 = dst_of<BINNED>(p, i2);
        }
        uint4 rec1 = make_uint4(0, 0, 0, 0);
        if (i1 < n) rec1 = record_of(A, raw1);
        lookup_one<DT, C, DEFER, UNI>(A, p, raw0, rec0, dst0);
        if (i1 >= n) break;
        raw0 = raw1;
        dst0 = dst1;
        rec0 = rec1;
        raw1 = raw2;
        dst1 = dst2;
        i1 = i2;
    }
}

// Grid-stride loop for the shared-memory path, two queries per thread and
// iteration: both queries and both records are loaded before either is
// filtered, so their latencies overlap; the pair four strides ahead is
// prefetched into L2.  I: the index type (32-bit when n allows).
template <int DT, int C, bool BINNED, bool DEFER, bool UNI, class I, class S>
__device__ __forceinline__ void lookup_loop_pairs(const Asset<S>& A, const FwdParams& p) {
    const I n = I(p.n);
    const I stride = I(gridDim.x) * I(blockDim.x);
    for (I i = I(blockIdx.x) * I(blockDim.x) + I(threadIdx.x); i < n; i += 2 * stride) {
        const I j = i + stride;
        const int4 ra = ld_query(p.q, i);
        const int4 rb = j < n ? ld_query(p.q, j) : make_int4(-1, 0, 0, 0);
        if (i + 4 * stride < n) prefetch_query(p.q, i + 4 * stride);
        if (j + 4 * stride < n) prefetch_query(p.q, j + 4 * stride);
        const uint4 ca = record_of(A, ra), cb = record_of(A, rb);
        lookup_one<DT, C, DEFER, UNI>(A, p, ra, ca, dst_of<BINNED>(p, i));
        if (j < n) lookup_one<DT, C, DEFER, UNI>(A, p, rb, cb, dst_of<BINNED>(p, j));
    }
}

// One resident block of 640 threads per SM (20 warps, 5 per scheduler)
// under 102 registers: each SM's threads then filter a contiguous stretch
// of the (sorted) queries, so the texels of neighbouring queries meet in
// its L1.  Measured on the sorted asset batch: 1 x 640 0.525 ms; 1 x 512,
// 1 x 768 2-3% slower (1 x 896 and 1 x 1024 spill); 2 x 320 0.558 ms,
// 2 x 256 1.6% slower than that, 2 x 384 and 3 x 256 2.5-5% slower, odd
// warp counts per SM (2 x 224 / 288 / 352) slower still.
constexpr int kGlobalThreads = 640;
#ifndef HTEX_GLOBAL_MIN_BLOCKS
#define HTEX_GLOBAL_MIN_BLOCKS 1
#endif
// one block of 1024 threads per SM (the pool staged once per SM): measured
// against 384 x 3 / 512 x 2 / 576 x 2 / 640 x 2 blocks per SM, 2.3-4.6%
// faster on the cube stream
constexpr int kStagedThreads = 1024;

template <int DT, int C, bool BINNED, bool UNI>
__global__ void __launch_bounds__(kGlobalThreads, HTEX_GLOBAL_MIN_BLOCKS) k_lookup_global(Asset<GlobalSpace> A, FwdParams p) {
    if (p.n <= int64_t(INT32_MAX) - 2 * int64_t(gridDim.x) * blockDim.x)
        lookup_loop<DT, C, BINNED, Raw<DT, C>::PACKED, UNI, int32_t>(A, p);
    else
        lookup_loop<DT, C, BINNED, Raw<DT, C>::PACKED, UNI, int64_t>(A, p);
}

// Shared-memory layout of a staged asset: records, headers, scales, pool,
// each starting on a 16-byte boundary.
struct StageLayout {
    uint32_t rec, hdr, scale, pool, total;
};

__host__ __device__ inline StageLayout stage_layout(int32_t H, int32_t E, int64_t pool_bytes) {
    StageLayout s;
    s.rec = 0;
    s.hdr = s.rec + uint32_t(H) * 16u;
    s.scale = s.hdr + uint32_t(E) * 16u;
    s.pool = s.scale + ((uint32_t(E) * 4u + 15u) & ~15u);
    s.total = s.pool + uint32_t(pool_bytes);
    return s;
}

__device__ __forceinline__ void stage16(uint8_t* dst, const void* src, uint32_t bytes) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (uint32_t k = threadIdx.x; k < bytes / 16u; k += blockDim.x) d[k] = __ldg(s + k);
}

template <int DT, int C, bool BINNED, bool UNI>
__global__ void __launch_bounds__(kStagedThreads, 1) k_lookup_staged(Asset<GlobalSpace> G, int32_t E,
                                                                  int64_t pool_bytes, FwdParams p) {
    extern __shared__ __align__(16) uint8_t smem[];
    const StageLayout L = stage_layout(G.H, E, pool_bytes);
    stage16(smem + L.rec, G.rec.base, uint32_t(G.H) * 16u);
    stage16(smem + L.hdr, G.hdr.base, uint32_t(E) * 16u);
    stage16(smem + L.scale, G.scale.base, (uint32_t(E) * 4u + 15u) & ~15u);
    stage16(smem + L.pool, G.pool.base, uint32_t(pool_bytes));
    __syncthreads();
    Asset<SharedSpace> A;
    A.rec.base = smem + L.rec;
    A.hdr.base = smem + L.hdr;
    A.scale.base = smem + L.scale;
    A.pool.base = smem + L.pool;
    A.H = G.H;
    A.uniform_log2n = G.uniform_log2n;
    A.uniform_stride16 = G.uniform_stride16;
    if (p.n <= int64_t(INT32_MAX) - 4 * int64_t(gridDim.x) * blockDim.x)
        lookup_loop_pairs<DT, C, BINNED, false, UNI, int32_t>(A, p);
    else
        lookup_loop_pairs<DT, C, BINNED, false, UNI, int64_t>(A, p);
}

constexpr uint32_t kMaxStageBytes = 96u * 1024u;       // largest asset staged in shared memory
constexpr int64_t kMinStagedQueries = int64_t(1) << 20;  // fewest queries worth staging for

template <class K>
int resident_blocks(K kernel, int threads, size_t smem) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess) b = 1;
    return b > 0 ? b : 1;
}

template <int DT, int C, bool BINNED>
htex_status launch_fwd(const htex_textures* t, const FwdParams& p, uint32_t flags, cudaStream_t s) {
    const Asset<GlobalSpace> A = global_asset(t);
    const StageLayout L = stage_layout(t->H, t->E, t->pool_bytes);
    // (sorted-index launches never stage: they serve pools above the sort threshold)
    const bool staged = !BINNED && !(flags & HTEX_LOOKUP_GLOBAL) && int64_t(L.total) <= int64_t(kMaxStageBytes) &&
                        p.n >= kMinStagedQueries;
    if (staged) {
        if constexpr (!BINNED) {
            auto k = t->uniform_log2n >= 0 ? k_lookup_staged<DT, C, false, true> : k_lookup_staged<DT, C, false, false>;
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L.total)) != cudaSuccess)
                return HTEX_ERR_CUDA;
            const int64_t want = (p.n + kStagedThreads - 1) / kStagedThreads;
            const int64_t grid =
                std::min<int64_t>(want, int64_t(t->num_sms) * resident_blocks(k, kStagedThreads, L.total));
            k<<<unsigned(grid), kStagedThreads, L.total, s>>>(A, t->E, t->pool_bytes, p);
        }
    } else {
        auto k = t->uniform_log2n >= 0 ? k_lookup_global<DT, C, BINNED, true> : k_lookup_global<DT, C, BINNED, false>;
        const int64_t want = (p.n + kGlobalThreads - 1) / kGlobalThreads;
        const int64_t grid = std::min<int64_t>(want, int64_t(t->num_sms) * resident_blocks(k, kGlobalThreads, 0));
        k<<<unsigned(grid), kGlobalThreads, 0, s>>>(A, p);
    }
    return cudaGetLastError() == cudaSuccess ? HTEX_OK : HTEX_ERR_CUDA;
}

template <int DT, bool BINNED>
htex_status launch_fwd_c(const htex_textures* t, const FwdParams& p, uint32_t flags, cudaStream_t s) {
    switch (t->C) {
    case 1: return launch_fwd<DT, 1, BINNED>(t, p, flags, s);
    case 2: return launch_fwd<DT, 2, BINNED>(t, p, flags, s);
    case 3: return launch_fwd<DT, 3, BINNED>(t, p, flags, s);
    case 4: return launch_fwd<DT, 4, BINNED>(t, p, flags, s);
    }
    return HTEX_ERR_INVALID_ARG;
}

// One launcher per texel format (lookup_<format>.cu).
htex_status launch_fwd_f32(const htex_textures* t, const FwdParams& p, uint32_t flags, cudaStream_t s, bool binned);
htex_status launch_fwd_u8(const htex_textures* t, const FwdParams& p, uint32_t flags, cudaStream_t s, bool binned);
htex_status launch_fwd_f16(const htex_textures* t, const FwdParams& p, uint32_t flags, cudaStream_t s, bool binned);
htex_status launch_fwd_bf16(const htex_textures* t, const FwdParams& p, uint32_t flags, cudaStream_t s, bool binned);
htex_status launch_fwd_e4m3(const htex_textures* t, const FwdParams& p, uint32_t flags, cudaStream_t s, bool binned);

}  // namespace htex
