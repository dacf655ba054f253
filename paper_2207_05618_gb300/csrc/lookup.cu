// Forward filtered lookup (paper Section 4.4, Alg. 3 with Alg. 2) and the
// htex_lookup entry point.
//
// One thread per query in a grid-stride loop over a persistent grid.  Per
// query: one streaming 16-byte query load, one 16-byte packed record
// (edges and Alg. 2 reflections of h, Next(h), Prev(h)), then up to three
// fetches, each one or two levels of 2x2 border-aware taps; fetches whose
// taps all fall outside their texture load nothing.  Two memory paths: the
// pool staged in shared memory (small assets, many queries) or read
// through the read-only cache from global memory.
#include <cuda_runtime.h>

#include "fetch.cuh"

namespace htex {

struct FwdParams {
    const htex_query* q;
    int64_t n;
    float* out;
    int32_t* status;
};

template <int DT, int C, class S>
__device__ __forceinline__ void sample_acc(const Asset<S>& A, const TexRef& t, int l, float x, float y,
                                           float wl, float (&acc)[C], float& W) {
    Taps k;
    if (!taps(x, y, 1 << (t.n - l), k)) return;
    constexpr int TB = C * Fmt<DT>::ES;
    using off_t = typename S::off_t;
    const off_t lvl = off_t(t.off + level_bytes(t.n, l, TB));
    float t00[C], t10[C], t01[C], t11[C];
    load_texel<DT, C>(A.pool, lvl + off_t(k.j0 * k.N + k.i0) * TB, t00);
    load_texel<DT, C>(A.pool, lvl + off_t(k.j0 * k.N + k.i1) * TB, t10);
    load_texel<DT, C>(A.pool, lvl + off_t(k.j1 * k.N + k.i0) * TB, t01);
    load_texel<DT, C>(A.pool, lvl + off_t(k.j1 * k.N + k.i1) * TB, t11);
    const float sc = wl * t.scale;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float r0 = fmaf(k.wx0, t00[c], k.wx1 * t10[c]);
        const float r1 = fmaf(k.wx0, t01[c], k.wx1 * t11[c]);
        acc[c] = fmaf(sc, fmaf(k.wy0, r0, k.wy1 * r1), acc[c]);
    }
    W = fmaf(wl, (k.wx0 + k.wx1) * (k.wy0 + k.wy1), W);
}

template <int DT, int C, class S>
__device__ __forceinline__ void fetch_acc(const Asset<S>& A, uint32_t code, float a, float b, float lf,
                                          float (&acc)[C], float& W) {
    float x, y;
    quad_coords(code, a, b, x, y);
    const TexRef t = tex_ref<DT>(A, code & ~kFlipBit);
    const Lod d = select_lod(lf, t.n);
    sample_acc<DT, C>(A, t, d.l0, x, y, d.w0, acc, W);
    if (d.l1 >= 0) sample_acc<DT, C>(A, t, d.l1, x, y, d.w1, acc, W);
}

template <int C>
__device__ __forceinline__ void store_out(float* out, int64_t i, const float (&r)[C]) {
    if constexpr (C == 4) {
        __stcs(reinterpret_cast<float4*>(out) + i, make_float4(r[0], r[1], r[2], r[3]));
    } else if constexpr (C == 2) {
        __stcs(reinterpret_cast<float2*>(out) + i, make_float2(r[0], r[1]));
    } else {
#pragma unroll
        for (int c = 0; c < C; ++c) __stcs(out + i * C + c, r[c]);
    }
}

template <int DT, int C, class S>
__device__ __forceinline__ void lookup_one(const Asset<S>& A, const FwdParams& p, int64_t i) {
    int h;
    float u, v, f;
    float r[C];
    if (!decode_query(ld_query(p.q, i), A.H, h, u, v, f)) {
#pragma unroll
        for (int c = 0; c < C; ++c) r[c] = __int_as_float(0x7fc00000);
        if (p.status) atomicAdd(p.status, 1);
    } else {
        const uint4 rec = A.rec.ld16(typename S::off_t(h) * 16u);
        const float lf = footprint_log2(f);
        float acc[C];
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = 0.0f;
        float W = 0.0f;
        fetch_acc<DT, C>(A, rec.x, u, v, lf, acc, W);    // own quad at (u, v)
        fetch_acc<DT, C>(A, rec.y, v, -u, lf, acc, W);   // Next(h)'s quad at (v, -u)
        fetch_acc<DT, C>(A, rec.z, -v, u, lf, acc, W);   // Prev(h)'s quad at (-v, u)
        const float inv = 1.0f / W;
#pragma unroll
        for (int c = 0; c < C; ++c) r[c] = acc[c] * inv;
    }
    store_out<C>(p.out, i, r);
}

template <int DT, int C>
__global__ void __launch_bounds__(256) k_lookup_global(Asset<GlobalSpace> A, FwdParams p) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < p.n; i += stride)
        lookup_one<DT, C>(A, p, i);
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

template <int DT, int C>
__global__ void __launch_bounds__(256) k_lookup_staged(Asset<GlobalSpace> G, int32_t E, int64_t pool_bytes,
                                                       FwdParams p) {
    extern __shared__ __align__(16) uint8_t smem[];
    const StageLayout L = stage_layout(G.H, E, pool_bytes);
    stage16(smem + L.rec, G.rec.base, uint32_t(G.H) * 16u);
    stage16(smem + L.hdr, G.hdr.base, uint32_t(E) * 16u);
    stage16(smem + L.scale, G.scale.base, (uint32_t(E) * 4u + 15u) & ~15u);
    stage16(smem + L.pool, G.pool.base, uint32_t(pool_bytes));
    __syncthreads();
    const uint32_t base = uint32_t(__cvta_generic_to_shared(smem));
    Asset<SharedSpace> A;
    A.rec.base = base + L.rec;
    A.hdr.base = base + L.hdr;
    A.scale.base = base + L.scale;
    A.pool.base = base + L.pool;
    A.H = G.H;
    A.uniform_log2n = G.uniform_log2n;
    A.uniform_stride16 = G.uniform_stride16;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < p.n; i += stride)
        lookup_one<DT, C>(A, p, i);
}

}  // namespace htex

using namespace htex;

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kMaxStageBytes = 96u * 1024u;
constexpr int64_t kMinStagedQueries = int64_t(1) << 20;

Asset<GlobalSpace> global_asset(const htex_textures* t) {
    Asset<GlobalSpace> A;
    A.rec.base = static_cast<const uint8_t*>(t->d_rec);
    A.hdr.base = static_cast<const uint8_t*>(t->d_hdr);
    A.scale.base = static_cast<const uint8_t*>(t->d_scale);
    A.pool.base = static_cast<const uint8_t*>(t->d_pool);
    A.H = t->H;
    A.uniform_log2n = t->uniform_log2n;
    A.uniform_stride16 = uint32_t(t->uniform_stride / 16);
    return A;
}

template <class K>
int resident_blocks(K kernel, size_t smem) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kThreads, smem) != cudaSuccess) b = 1;
    return b > 0 ? b : 1;
}

template <int DT, int C>
htex_status launch_fwd(const htex_textures* t, const FwdParams& p, uint32_t flags, cudaStream_t s) {
    const Asset<GlobalSpace> A = global_asset(t);
    const int64_t want = (p.n + kThreads - 1) / kThreads;
    const StageLayout L = stage_layout(t->H, t->E, t->pool_bytes);
    const bool staged = !(flags & HTEX_LOOKUP_GLOBAL) && int64_t(L.total) <= int64_t(kMaxStageBytes) &&
                        p.n >= kMinStagedQueries;
    if (staged) {
        auto k = k_lookup_staged<DT, C>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L.total)) != cudaSuccess)
            return HTEX_ERR_CUDA;
        const int64_t grid = std::min<int64_t>(want, int64_t(t->num_sms) * resident_blocks(k, L.total));
        k<<<unsigned(grid), kThreads, L.total, s>>>(A, t->E, t->pool_bytes, p);
    } else {
        auto k = k_lookup_global<DT, C>;
        const int64_t grid = std::min<int64_t>(want, int64_t(t->num_sms) * resident_blocks(k, 0));
        k<<<unsigned(grid), kThreads, 0, s>>>(A, p);
    }
    return cudaGetLastError() == cudaSuccess ? HTEX_OK : HTEX_ERR_CUDA;
}

template <int DT>
htex_status launch_fwd_c(const htex_textures* t, const FwdParams& p, uint32_t flags, cudaStream_t s) {
    switch (t->C) {
    case 1: return launch_fwd<DT, 1>(t, p, flags, s);
    case 2: return launch_fwd<DT, 2>(t, p, flags, s);
    case 3: return launch_fwd<DT, 3>(t, p, flags, s);
    case 4: return launch_fwd<DT, 4>(t, p, flags, s);
    }
    return HTEX_ERR_INVALID_ARG;
}

}  // namespace

htex_status htex_launch_lookup(const htex_textures* t, const htex_query* q, int64_t n, float* out,
                               uint32_t flags, htex_stream stream, int32_t* d_status) {
    const FwdParams p{q, n, out, d_status};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (t->dtype) {
    case HTEX_F32: return launch_fwd_c<HTEX_F32>(t, p, flags, s);
    case HTEX_U8: return launch_fwd_c<HTEX_U8>(t, p, flags, s);
    case HTEX_F16: return launch_fwd_c<HTEX_F16>(t, p, flags, s);
    case HTEX_BF16: return launch_fwd_c<HTEX_BF16>(t, p, flags, s);
    case HTEX_E4M3: return launch_fwd_c<HTEX_E4M3>(t, p, flags, s);
    }
    return HTEX_ERR_INVALID_ARG;
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
    if (flags & HTEX_LOOKUP_BIN) return HTEX_ERR_UNSUPPORTED;
    return htex_launch_lookup(t, q, n, out, flags, stream, d_status);
}
