// Adjoint of the filtered lookup and the htex_lookup_backward entry point.
//
// The lookup is linear in the stored texels: out_c = sum_k w_k T_k,c / W
// with W the sum of the in-bounds weights of all taps of the three fetches
// (Alg. 3).  So dL/dT_k,c = sum over queries of grad_out_c * w_k / W.  Per
// query the kernel first recomputes W from the coordinates alone (no texel
// loads), then scatter-adds grad_out * w_k / W into every in-bounds tap
// with nonzero weight: float4/float2 atomics where a texel's channels are
// contiguous and aligned (three-channel texels: one float2 and one scalar
// atomic), scalar atomics otherwise.
//
// Every lane of a warp runs every iteration of the grid-stride loop (lanes
// past the end carry no query), so warp-wide collectives always see all 32
// lanes; the query two iterations ahead and the record and upstream
// gradient one iteration ahead are in flight while the current query is
// scattered.
//
// Warp-aggregated variant (AGG, used after the queries are sorted by
// halfedge range, HTEX_LOOKUP_BIN): a query's taps come in parts -- the own fetch's 2x2
// block at each of its levels, and the two-texel row or column of the
// Next and Prev fetches at each level.  A part's taps are fixed by (texture,
// level, first tap index, side), so lanes whose parts have equal keys
// (__match_any_sync) add into the same texels: their values are summed
// across the group with shuffles and only the group's lowest lane issues
// the atomics.  Lanes on the same coarse level of one texture collapse to
// one atomic per texel; a warp with no shared part pays one match and one
// vote per part.
#include <algorithm>
#include <cmath>

#include <cuda_runtime.h>

#include "fetch.cuh"

namespace htex {

constexpr unsigned kFull = 0xffffffffu;

struct BwdParams {
    const htex_query* q;
    int64_t n;
    const float* gout;
    float* grad;
    int32_t* status;
    int32_t vec;    // grad's alignment in floats (4: 16 bytes, 2: 8 bytes, else 1): the widest atomics three-channel texels may take
};

// The forward weights, recomputed: each fetch decomposed as in the forward
// kernel (own 2x2 block, Next/Prev one texel row or column per level).
__device__ __forceinline__ float own_weight(int n, int l, float x, float y) {
    const int N = 1 << (n - l);
    const Taps1 tx = taps1(x, N), ty = taps1(y, N);
    return (tx.w0 + tx.w1) * (ty.w0 + ty.w1);
}

__device__ __forceinline__ float edge_weight(int n, int l, float dist, float along, bool flip) {
    const int N = 1 << (n - l);
    const float wa = across_weight(dist, N);
    if (!(wa > 0.0f)) return 0.0f;
    const Taps1 ta = taps1(flip ? 1.0f - along : along, N);
    return wa * (ta.w0 + ta.w1);
}

// One texel's C values added into the gradient at element index elem.  A
// three-channel texel with a 16-byte aligned gradient: the three values lie
// in one 16-byte block for half the texels (elem = 0 or 1 mod 4), which
// take one four-float atomic (+0.0 added to the block's fourth element,
// which keeps its value); the others a float2 and a scalar atomic.  This
// takes about a quarter of the atomic requests off (measured: the adjoint
// in the given query order 27% faster, sorted 3-8%).
template <int C>
__device__ __forceinline__ void red_texel(float* grad, uint64_t elem, const float* x, int vec) {
    if constexpr (C == 4) {
        atomicAdd(reinterpret_cast<float4*>(grad + elem), make_float4(x[0], x[1], x[2], x[3]));
    } else if constexpr (C == 2) {
        atomicAdd(reinterpret_cast<float2*>(grad + elem), make_float2(x[0], x[1]));
    } else if constexpr (C == 3) {
        if (vec == 4) {
            const uint32_t r = uint32_t(elem & 3u);
            float* c = grad + (elem - r);   // the 16-byte block holding the first value
            if (r == 0) {
                atomicAdd(reinterpret_cast<float4*>(c), make_float4(x[0], x[1], x[2], 0.0f));
            } else if (r == 1) {
                atomicAdd(reinterpret_cast<float4*>(c), make_float4(0.0f, x[0], x[1], x[2]));
            } else if (r == 2) {
                atomicAdd(reinterpret_cast<float2*>(c + 2), make_float2(x[0], x[1]));
                atomicAdd(c + 4, x[2]);
            } else {
                atomicAdd(c + 3, x[0]);
                atomicAdd(reinterpret_cast<float2*>(c + 4), make_float2(x[1], x[2]));
            }
        } else if (vec == 2) {   // the 8-byte-aligned pair of the three channels, then the third alone
            const bool even = (elem & 1u) == 0;
            atomicAdd(reinterpret_cast<float2*>(grad + elem + (even ? 0 : 1)),
                      even ? make_float2(x[0], x[1]) : make_float2(x[1], x[2]));
            atomicAdd(grad + elem + (even ? 2 : 0), even ? x[2] : x[0]);
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) atomicAdd(grad + elem + c, x[c]);
        }
    } else {
        atomicAdd(grad + elem, x[0]);
    }
}

// Two horizontally adjacent texels (elements elem and elem + C), each added
// when its flag is set.  Both set, with a 16-byte aligned gradient: three
// channels take 2 atomics for half the pairs and 3 for the rest (the six
// values cover 2 or 3 16-byte blocks; zeros pad the blocks' other
// elements), against 3 on average texel by texel; two channels with elem a
// multiple of 4 take one float4; one channel with elem even one float2.
template <int C>
__device__ __forceinline__ void red_pair(float* grad, uint64_t elem, const float* x, bool a0, bool a1, int vec) {
    if (a0 && a1 && vec == 4) {
        const uint32_t r = uint32_t(elem & 3u);
        float* c = grad + (elem - r);
        if constexpr (C == 3) {
            const float* y = x + 3;
            if (r == 0) {
                atomicAdd(reinterpret_cast<float4*>(c), make_float4(x[0], x[1], x[2], y[0]));
                atomicAdd(reinterpret_cast<float2*>(c + 4), make_float2(y[1], y[2]));
            } else if (r == 1) {
                atomicAdd(reinterpret_cast<float4*>(c), make_float4(0.0f, x[0], x[1], x[2]));
                atomicAdd(reinterpret_cast<float4*>(c + 4), make_float4(y[0], y[1], y[2], 0.0f));
            } else if (r == 2) {
                atomicAdd(reinterpret_cast<float2*>(c + 2), make_float2(x[0], x[1]));
                atomicAdd(reinterpret_cast<float4*>(c + 4), make_float4(x[2], y[0], y[1], y[2]));
            } else {
                atomicAdd(c + 3, x[0]);
                atomicAdd(reinterpret_cast<float4*>(c + 4), make_float4(x[1], x[2], y[0], y[1]));
                atomicAdd(c + 8, y[2]);
            }
            return;
        } else if constexpr (C == 2) {
            if (r == 0) {
                atomicAdd(reinterpret_cast<float4*>(c), make_float4(x[0], x[1], x[2], x[3]));
                return;
            }
        } else if constexpr (C == 1) {
            if ((r & 1u) == 0) {
                atomicAdd(reinterpret_cast<float2*>(grad + elem), make_float2(x[0], x[1]));
                return;
            }
        }
    }
    if (a0) red_texel<C>(grad, elem, x, vec);
    if (a1) red_texel<C>(grad, elem + C, x + C, vec);
}

// Sum of x over the lanes of the calling lane's group (peers: the lanes with
// an equal key, from __match_any_sync); the group's lowest lane ends up
// holding the total.  All 32 lanes call it together.  A tree over group
// ranks: at step s, the lane of rank r adds the partial sum of rank r + s.
template <int K>
__device__ __forceinline__ void group_sum(unsigned peers, float (&x)[K]) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned most = __reduce_max_sync(kFull, unsigned(__popc(peers)));
    unsigned above = peers & ~((2u << lane) - 1u);   // group members above this lane
    int dropped = 0;
    for (unsigned s = 1; s < most; s <<= 1) {
        while (dropped < int(s) - 1) {   // keep the members from rank + s up
            above &= above - 1u;
            ++dropped;
        }
        const bool has = above != 0u;
        const int src = has ? __ffs(above) - 1 : int(lane);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float o = __shfl_sync(kFull, x[k], src);
            if (has) x[k] += o;
        }
    }
}

__device__ __forceinline__ bool lowest_of(unsigned peers) {
    return (peers & ((1u << (threadIdx.x & 31u)) - 1u)) == 0u;
}

// The own fetch's 2x2 block at level l: taps (i, j), (i + 1, j), (i, j + 1),
// (i + 1, j + 1) of weight wl * w_x * w_y, into element index
// level start + (row * N + column) * C.
template <int DT, int C, bool AGG>
__device__ __forceinline__ void own_part(const BwdParams& p, const TexRef& t, uint32_t e, int l, float x, float y,
                                         float wl, bool on, const float (&g)[C]) {
    const int N = 1 << (t.n - l);
    const TapsU tx = taps_u(x, N), ty = taps_u(y, N);
    const float w[4] = {wl * ty.w0 * tx.w0, wl * ty.w0 * tx.w1, wl * ty.w1 * tx.w0, wl * ty.w1 * tx.w1};
    const bool inb[4] = {tx.i >= 0 && ty.i >= 0, tx.i + 1 < N && ty.i >= 0, tx.i >= 0 && ty.i + 1 < N,
                         tx.i + 1 < N && ty.i + 1 < N};
    float v[4 * C];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < C; ++c) v[k * C + c] = w[k] * g[c];
    bool summed = false;
    if constexpr (AGG) {
        const unsigned long long key =
            on ? (uint64_t(e) << 32) | (uint32_t(l) << 28) | (uint32_t(ty.i + 1) << 14) | uint32_t(tx.i + 1)
               : ~0ull;
        const unsigned peers = __match_any_sync(kFull, key);
        if (__any_sync(kFull, on && peers != (1u << (threadIdx.x & 31u)))) {
            group_sum<4 * C>(peers, v);
            summed = true;
            on = on && lowest_of(peers);
        }
    }
    if (!on) return;
    const int64_t b = int64_t(t.off / Fmt<DT>::ES + uint64_t(level_texels(t.n, l)) * C) +
                      (int64_t(ty.i) * N + tx.i) * C;
    bool act[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) act[k] = inb[k] && (summed || w[k] != 0.0f);
    red_pair<C>(p.grad, uint64_t(b), v, act[0], act[1], p.vec);                       // row j
    red_pair<C>(p.grad, uint64_t(b + int64_t(N) * C), v + 2 * C, act[2], act[3], p.vec);   // row j + 1
}

// A Next (row) or Prev (column) fetch at level l: the two texels of row or
// column k (0, or N - 1 when Alg. 2 reflects the quad) on the shared side,
// at positions i and i + 1 along it.
template <int DT, int C, bool AGG>
__device__ __forceinline__ void edge_part(const BwdParams& p, const TexRef& t, uint32_t e, int l, float dist,
                                          float along, bool flip, bool row, float wl, bool on,
                                          const float (&g)[C]) {
    const int N = 1 << (t.n - l);
    const float wa = across_weight(dist, N);
    on = on && wa > 0.0f;
    const TapsU ta = taps_u(flip ? 1.0f - along : along, N);
    const float w[2] = {wl * wa * ta.w0, wl * wa * ta.w1};
    const bool inb[2] = {ta.i >= 0, ta.i + 1 < N};
    float v[2 * C];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int c = 0; c < C; ++c) v[k * C + c] = w[k] * g[c];
    bool summed = false;
    if constexpr (AGG) {
        const unsigned long long key =
            on ? (uint64_t(e) << 32) | (uint32_t(l) << 28) | (uint32_t(row) << 27) | (uint32_t(flip) << 26) |
                     uint32_t(ta.i + 1)
               : ~0ull;
        const unsigned peers = __match_any_sync(kFull, key);
        if (__any_sync(kFull, on && peers != (1u << (threadIdx.x & 31u)))) {
            group_sum<2 * C>(peers, v);
            summed = true;
            on = on && lowest_of(peers);
        }
    }
    if (!on) return;
    const int k = flip ? N - 1 : 0;
    const int64_t step = row ? 1 : N;
    const int64_t b = int64_t(t.off / Fmt<DT>::ES + uint64_t(level_texels(t.n, l)) * C) +
                      ((row ? int64_t(k) * N : int64_t(k)) + int64_t(ta.i) * step) * C;
    const bool act0 = inb[0] && (summed || w[0] != 0.0f), act1 = inb[1] && (summed || w[1] != 0.0f);
    if (row) {
        red_pair<C>(p.grad, uint64_t(b), v, act0, act1, p.vec);
    } else {
        if (act0) red_texel<C>(p.grad, uint64_t(b), v, p.vec);
        if (act1) red_texel<C>(p.grad, uint64_t(b + step * C), v + C, p.vec);
    }
}

// One query's three fetches: their textures, level choices and coordinates.
struct Fetches {
    TexRef t[3];
    Lod d[3];
    bool flip[3];
    uint32_t e[3];
};

template <int DT, class S>
__device__ __forceinline__ Fetches plan(const Asset<S>& A, uint4 rec, float lf) {
    Fetches F;
    const uint32_t code[3] = {rec.x, rec.y, rec.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        F.e[k] = code[k] & ~kFlipBit;
        F.t[k] = tex_ref<DT>(A, F.e[k]);
        F.d[k] = select_lod(lf, F.t[k].n);
        F.flip[k] = code[k] & kFlipBit;
    }
    return F;
}

template <int C>
__device__ __forceinline__ void load_gout(const BwdParams& p, int64_t i, bool valid, float (&g)[C]) {
    if constexpr (C == 4) {
        const float4 r = valid ? __ldcs(reinterpret_cast<const float4*>(p.gout) + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        g[0] = r.x; g[1] = r.y; g[2] = r.z; g[3] = r.w;
    } else {
#pragma unroll
        for (int c = 0; c < C; ++c) g[c] = valid ? __ldcs(p.gout + i * C + c) : 0.0f;
    }
}

// The adjoint of one query (valid: the lane holds a query of the batch).
template <int DT, int C, bool AGG>
__device__ __forceinline__ void scatter_one(const Asset<GlobalSpace>& A, const BwdParams& p, bool valid, int4 raw,
                                            uint4 rec, const float (&gin)[C]) {
    int h;
    float u, v, f;
    bool ok = valid && decode_query(raw, A.H, h, u, v, f);
    if (valid && !ok && p.status) atomicAdd(p.status, 1);
    if (!ok) {
        u = 0.0f;
        v = 0.0f;
        f = 0.0f;
        rec = make_uint4(0u, 0u, 0u, 0u);
    }
    const Fetches F = plan<DT>(A, rec, footprint_log2(f));
    const float x = F.flip[0] ? 1.0f - u : u, y = F.flip[0] ? 1.0f - v : v;
    float W = 0.0f;
    W = fmaf(F.d[0].w0, own_weight(F.t[0].n, F.d[0].l0, x, y), W);
    if (F.d[0].l1 >= 0) W = fmaf(F.d[0].w1, own_weight(F.t[0].n, F.d[0].l1, x, y), W);
    W = fmaf(F.d[1].w0, edge_weight(F.t[1].n, F.d[1].l0, u, v, F.flip[1]), W);
    if (F.d[1].l1 >= 0) W = fmaf(F.d[1].w1, edge_weight(F.t[1].n, F.d[1].l1, u, v, F.flip[1]), W);
    W = fmaf(F.d[2].w0, edge_weight(F.t[2].n, F.d[2].l0, v, u, F.flip[2]), W);
    if (F.d[2].l1 >= 0) W = fmaf(F.d[2].w1, edge_weight(F.t[2].n, F.d[2].l1, v, u, F.flip[2]), W);
    const float inv = ok ? __frcp_rn(W) : 0.0f;
    float g[C];
#pragma unroll
    for (int c = 0; c < C; ++c) g[c] = gin[c] * inv;

    // own fetch (one or two levels), then Next (row, distance u, along v) and
    // Prev (column, distance v, along u); parts no lane needs are skipped
    own_part<DT, C, AGG>(p, F.t[0], F.e[0], F.d[0].l0, x, y, F.d[0].w0, ok, g);
    const bool own2 = ok && F.d[0].l1 >= 0;
    if (__any_sync(kFull, own2))
        own_part<DT, C, AGG>(p, F.t[0], F.e[0], own2 ? F.d[0].l1 : F.d[0].l0, x, y, F.d[0].w1, own2, g);
#pragma unroll
    for (int k = 1; k < 3; ++k) {
        const bool row = k == 1;
        const float dist = row ? u : v, along = row ? v : u;
        const int cl = F.d[k].l1 >= 0 ? F.d[k].l1 : F.d[k].l0;   // coarsest level: the widest reach
        const bool near = ok && across_weight(dist, 1 << (F.t[k].n - cl)) > 0.0f;
        if (!__any_sync(kFull, near)) continue;
        edge_part<DT, C, AGG>(p, F.t[k], F.e[k], F.d[k].l0, dist, along, F.flip[k], row, F.d[k].w0, near, g);
        const bool two = near && F.d[k].l1 >= 0;
        if (__any_sync(kFull, two))
            edge_part<DT, C, AGG>(p, F.t[k], F.e[k], two ? F.d[k].l1 : F.d[k].l0, dist, along, F.flip[k], row,
                                  F.d[k].w1, two, g);
    }
}

template <int DT, int C, bool AGG>
__global__ void __launch_bounds__(256, 3) k_backward(Asset<GlobalSpace> A, BwdParams p) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t base = i - int64_t(threadIdx.x & 31u);   // the warp's first query: the loop is warp-uniform
    if (base >= p.n) return;
    const int4 none = make_int4(-1, 0, 0, 0);
    int4 raw0 = i < p.n ? ld_query(p.q, i) : none;
    int4 raw1 = i + stride < p.n ? ld_query(p.q, i + stride) : none;
    uint4 rec0 = i < p.n ? A.rec.ld16(uint64_t(unsigned(raw0.x) < unsigned(A.H) ? raw0.x : 0) * 16u)
                         : make_uint4(0u, 0u, 0u, 0u);
    float g0[C];
    load_gout<C>(p, i, i < p.n, g0);
    for (; base < p.n; base += stride, i += stride) {
        const int64_t i1 = i + stride, i2 = i + 2 * stride;
        const int4 raw2 = i2 < p.n ? ld_query(p.q, i2) : none;
        const uint4 rec1 = i1 < p.n ? A.rec.ld16(uint64_t(unsigned(raw1.x) < unsigned(A.H) ? raw1.x : 0) * 16u)
                                    : make_uint4(0u, 0u, 0u, 0u);
        float g1[C];
        load_gout<C>(p, i1, i1 < p.n, g1);
        scatter_one<DT, C, AGG>(A, p, i < p.n, raw0, rec0, g0);
        raw0 = raw1;
        raw1 = raw2;
        rec0 = rec1;
#pragma unroll
        for (int c = 0; c < C; ++c) g0[c] = g1[c];
    }
}

}  // namespace htex

using namespace htex;

namespace {

constexpr int kThreads = 256;

template <int DT, int C, bool AGG>
htex_status launch_bwd(const htex_textures* t, const BwdParams& p, cudaStream_t s) {
    const Asset<GlobalSpace> A = global_asset(t);
    auto k = k_backward<DT, C, AGG>;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, kThreads, 0) != cudaSuccess || b < 1) b = 1;
    const int64_t want = (p.n + kThreads - 1) / kThreads;
    const int64_t grid = std::min<int64_t>(want, int64_t(t->num_sms) * b);
    k<<<unsigned(grid), kThreads, 0, s>>>(A, p);
    return cudaGetLastError() == cudaSuccess ? HTEX_OK : HTEX_ERR_CUDA;
}

template <int DT, bool AGG>
htex_status launch_bwd_c(const htex_textures* t, const BwdParams& p, cudaStream_t s) {
    switch (t->C) {
    case 1: return launch_bwd<DT, 1, AGG>(t, p, s);
    case 2: return launch_bwd<DT, 2, AGG>(t, p, s);
    case 3: return launch_bwd<DT, 3, AGG>(t, p, s);
    case 4: return launch_bwd<DT, 4, AGG>(t, p, s);
    }
    return HTEX_ERR_INVALID_ARG;
}

template <bool AGG>
htex_status launch_bwd_dt(const htex_textures* t, const BwdParams& p, cudaStream_t s) {
    switch (t->dtype) {
    case HTEX_F32: return launch_bwd_c<HTEX_F32, AGG>(t, p, s);
    case HTEX_U8: return launch_bwd_c<HTEX_U8, AGG>(t, p, s);
    case HTEX_F16: return launch_bwd_c<HTEX_F16, AGG>(t, p, s);
    case HTEX_BF16: return launch_bwd_c<HTEX_BF16, AGG>(t, p, s);
    case HTEX_E4M3: return launch_bwd_c<HTEX_E4M3, AGG>(t, p, s);
    }
    return HTEX_ERR_INVALID_ARG;
}

}  // namespace

htex_status htex_launch_backward(const htex_textures* t, const htex_query* q, int64_t n, const float* grad_out,
                                 float* grad_texels, uint32_t flags, htex_stream stream, int32_t* d_status) {
    const uintptr_t ga = reinterpret_cast<uintptr_t>(grad_texels);
    const BwdParams p{q, n, grad_out, grad_texels, d_status, (ga & 15u) == 0 ? 4 : ((ga & 7u) == 0 ? 2 : 1)};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (flags & kBackwardAggregate) return launch_bwd_dt<true>(t, p, s);
    return launch_bwd_dt<false>(t, p, s);
}

// ------------------------------------------------------ Adam on the pool
//
// One Adam step (Kingma & Ba) on an FP32 asset's texels, fused with what a
// texture fit needs around it: the updated values go to the master copy
// and straight into the resident pool, and the gradient is cleared for the
// next accumulation.  Per element, with t the step number:
//   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
//   p = p - (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps).
struct AdamParams {
    float* master;   // the values being optimised (the pool itself when no separate copy is kept)
    float* grad;
    float* m;
    float* v;
    float* pool;     // null when master is the pool
    int64_t n;
    float b1, b2, eps, step_size, inv_sqrt_bc2;
};

__device__ __forceinline__ float adam_one(float& p, float g, float& m, float& v, const AdamParams& a) {
    m = fmaf(a.b1, m, (1.0f - a.b1) * g);
    v = fmaf(a.b2, v, ((1.0f - a.b2) * g) * g);
    const float denom = sqrtf(v) * a.inv_sqrt_bc2 + a.eps;
    p = p - a.step_size * (m / denom);
    return p;
}

__global__ void __launch_bounds__(256) k_adam(AdamParams a) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t n4 = a.n / 4;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 p = reinterpret_cast<float4*>(a.master)[i];
        const float4 g = __ldcs(reinterpret_cast<const float4*>(a.grad) + i);
        float4 m = reinterpret_cast<float4*>(a.m)[i];
        float4 v = reinterpret_cast<float4*>(a.v)[i];
        adam_one(p.x, g.x, m.x, v.x, a);
        adam_one(p.y, g.y, m.y, v.y, a);
        adam_one(p.z, g.z, m.z, v.z, a);
        adam_one(p.w, g.w, m.w, v.w, a);
        reinterpret_cast<float4*>(a.master)[i] = p;
        reinterpret_cast<float4*>(a.m)[i] = m;
        reinterpret_cast<float4*>(a.v)[i] = v;
        if (a.pool) __stcs(reinterpret_cast<float4*>(a.pool) + i, p);
        __stcs(reinterpret_cast<float4*>(a.grad) + i, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
    }
    for (int64_t i = 4 * n4 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        float p = a.master[i], m = a.m[i], v = a.v[i];
        adam_one(p, a.grad[i], m, v, a);
        a.master[i] = p;
        a.m[i] = m;
        a.v[i] = v;
        if (a.pool) a.pool[i] = p;
        a.grad[i] = 0.0f;
    }
}

extern "C" htex_status htex_textures_adam_step(htex_textures* t, float* master, float* grad, float* m, float* v,
                                               int64_t n, float lr, float beta1, float beta2, float eps,
                                               int32_t step, htex_stream stream) {
    if (!t || t->dtype != HTEX_F32) return HTEX_ERR_INVALID_ARG;
    if (n != t->pool_bytes / 4 || step < 1) return HTEX_ERR_INVALID_ARG;
    if (!grad || !m || !v) return HTEX_ERR_INVALID_ARG;
    float* pool = static_cast<float*>(t->d_pool);
    if (!master) {   // the pool holds the values: one stream less, no copy to keep
        master = pool;
        pool = nullptr;
    }
    const uintptr_t all = reinterpret_cast<uintptr_t>(master) | reinterpret_cast<uintptr_t>(grad) |
                          reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v);
    if ((all & 15u) != 0) return HTEX_ERR_INVALID_ARG;
    if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps > 0.0f)) return HTEX_ERR_INVALID_ARG;
    const double bc1 = 1.0 - std::pow(double(beta1), double(step));
    const double bc2 = 1.0 - std::pow(double(beta2), double(step));
    const AdamParams a{master, grad, m, v, pool, n, beta1, beta2, eps,
                       float(double(lr) / bc1), float(1.0 / std::sqrt(bc2))};
    const int64_t want = (n / 4 + 255) / 256 + 1;
    const unsigned grid = unsigned(std::min<int64_t>(want, int64_t(t->num_sms) * 8));
    k_adam<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? HTEX_OK : HTEX_ERR_CUDA;
}

extern "C" htex_status htex_lookup_backward(const htex_textures* t, const htex_query* q, int64_t n,
                                            const float* grad_out, float* grad_texels, uint32_t flags,
                                            htex_stream stream, int32_t* d_status) {
    if (!t || n < 0) return HTEX_ERR_INVALID_ARG;
    if (flags & ~uint32_t(HTEX_LOOKUP_BIN | HTEX_LOOKUP_GLOBAL)) return HTEX_ERR_INVALID_ARG;
    if (n == 0) return HTEX_OK;
    if (!q || !grad_out || !grad_texels) return HTEX_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(q) & 15u) != 0) return HTEX_ERR_INVALID_ARG;
    // vector atomics need the gradient's texel groups aligned to their size
    const uintptr_t ga = t->C == 4 ? 16u : (t->C == 2 ? 8u : 4u);
    if ((reinterpret_cast<uintptr_t>(grad_texels) & (ga - 1)) != 0) return HTEX_ERR_INVALID_ARG;
    if (flags & HTEX_LOOKUP_BIN) return htex_launch_backward_sorted(t, q, n, grad_out, grad_texels, stream, d_status);
    return htex_launch_backward(t, q, n, grad_out, grad_texels, flags, stream, d_status);
}
