// Adjoint of the filtered lookup and the htex_lookup_backward entry point.
//
// The lookup is linear in the stored texels: out_c = sum_k w_k T_k,c / W
// with W the sum of the in-bounds weights of all taps of the three fetches
// (Alg. 3).  So dL/dT_k,c = sum over queries of grad_out_c * w_k / W.  Per
// query the kernel first recomputes W from the coordinates alone (no texel
// loads), then scatter-adds grad_out * w_k / W into every in-bounds tap
// with nonzero weight: float4/float2 atomics where a texel's channels are
// contiguous and aligned, scalar atomics otherwise.
#include <algorithm>
#include <cmath>

#include <cuda_runtime.h>

#include "fetch.cuh"

namespace htex {

struct BwdParams {
    const htex_query* q;
    int64_t n;
    const float* gout;
    float* grad;
    int32_t* status;
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

template <int C>
__device__ __forceinline__ void add_texel(float* grad, uint64_t elem, float w, const float (&g)[C]) {
    if (w == 0.0f) return;
    if constexpr (C == 4) {
        atomicAdd(reinterpret_cast<float4*>(grad + elem), make_float4(w * g[0], w * g[1], w * g[2], w * g[3]));
    } else if constexpr (C == 2) {
        atomicAdd(reinterpret_cast<float2*>(grad + elem), make_float2(w * g[0], w * g[1]));
    } else {
#pragma unroll
        for (int c = 0; c < C; ++c) atomicAdd(grad + elem + c, w * g[c]);
    }
}

template <int DT, int C>
__device__ __forceinline__ void own_scatter(float* grad, const TexRef& t, int l, float x, float y, float wl,
                                            const float (&g)[C]) {
    constexpr int ES = Fmt<DT>::ES;
    const int N = 1 << (t.n - l);
    const Taps1 tx = taps1(x, N), ty = taps1(y, N);
    const uint64_t lvl = t.off / ES + uint64_t(level_texels(t.n, l)) * C;   // element index
    add_texel<C>(grad, lvl + uint64_t(ty.i0 * N + tx.i0) * C, wl * ty.w0 * tx.w0, g);
    add_texel<C>(grad, lvl + uint64_t(ty.i0 * N + tx.i1) * C, wl * ty.w0 * tx.w1, g);
    add_texel<C>(grad, lvl + uint64_t(ty.i1 * N + tx.i0) * C, wl * ty.w1 * tx.w0, g);
    add_texel<C>(grad, lvl + uint64_t(ty.i1 * N + tx.i1) * C, wl * ty.w1 * tx.w1, g);
}

template <int DT, int C, bool ROW>
__device__ __forceinline__ void edge_scatter(float* grad, const TexRef& t, int l, float dist, float along, bool flip,
                                             float wl, const float (&g)[C]) {
    constexpr int ES = Fmt<DT>::ES;
    const int N = 1 << (t.n - l);
    const float wa = across_weight(dist, N);
    if (!(wa > 0.0f)) return;
    const Taps1 ta = taps1(flip ? 1.0f - along : along, N);
    const int k = flip ? N - 1 : 0;
    const uint64_t lvl = t.off / ES + uint64_t(level_texels(t.n, l)) * C;
    const uint64_t e0 = ROW ? uint64_t(k * N + ta.i0) : uint64_t(ta.i0 * N + k);
    const uint64_t e1 = ROW ? uint64_t(k * N + ta.i1) : uint64_t(ta.i1 * N + k);
    add_texel<C>(grad, lvl + e0 * C, wl * wa * ta.w0, g);
    add_texel<C>(grad, lvl + e1 * C, wl * wa * ta.w1, g);
}

// One query's three fetches: their textures, level choices and coordinates.
struct Fetches {
    TexRef t[3];
    Lod d[3];
    bool flip[3];
};

template <int DT, class S>
__device__ __forceinline__ Fetches plan(const Asset<S>& A, uint4 rec, float lf) {
    Fetches F;
    const uint32_t code[3] = {rec.x, rec.y, rec.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        F.t[k] = tex_ref<DT>(A, code[k] & ~kFlipBit);
        F.d[k] = select_lod(lf, F.t[k].n);
        F.flip[k] = code[k] & kFlipBit;
    }
    return F;
}

template <int DT, int C>
__global__ void __launch_bounds__(256) k_backward(Asset<GlobalSpace> A, BwdParams p) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < p.n; i += stride) {
        int h;
        float u, v, f;
        if (!decode_query(ld_query(p.q, i), A.H, h, u, v, f)) {
            if (p.status) atomicAdd(p.status, 1);
            continue;
        }
        const uint4 rec = A.rec.ld16(uint64_t(h) * 16u);
        const Fetches F = plan<DT>(A, rec, footprint_log2(f));
        const float x = F.flip[0] ? 1.0f - u : u, y = F.flip[0] ? 1.0f - v : v;
        float W = 0.0f;
        W = fmaf(F.d[0].w0, own_weight(F.t[0].n, F.d[0].l0, x, y), W);
        if (F.d[0].l1 >= 0) W = fmaf(F.d[0].w1, own_weight(F.t[0].n, F.d[0].l1, x, y), W);
        W = fmaf(F.d[1].w0, edge_weight(F.t[1].n, F.d[1].l0, u, v, F.flip[1]), W);
        if (F.d[1].l1 >= 0) W = fmaf(F.d[1].w1, edge_weight(F.t[1].n, F.d[1].l1, u, v, F.flip[1]), W);
        W = fmaf(F.d[2].w0, edge_weight(F.t[2].n, F.d[2].l0, v, u, F.flip[2]), W);
        if (F.d[2].l1 >= 0) W = fmaf(F.d[2].w1, edge_weight(F.t[2].n, F.d[2].l1, v, u, F.flip[2]), W);
        const float inv = __frcp_rn(W);
        float g[C];
#pragma unroll
        for (int c = 0; c < C; ++c) g[c] = __ldcs(p.gout + i * C + c) * inv;
        own_scatter<DT, C>(p.grad, F.t[0], F.d[0].l0, x, y, F.d[0].w0, g);
        if (F.d[0].l1 >= 0) own_scatter<DT, C>(p.grad, F.t[0], F.d[0].l1, x, y, F.d[0].w1, g);
        edge_scatter<DT, C, true>(p.grad, F.t[1], F.d[1].l0, u, v, F.flip[1], F.d[1].w0, g);
        if (F.d[1].l1 >= 0) edge_scatter<DT, C, true>(p.grad, F.t[1], F.d[1].l1, u, v, F.flip[1], F.d[1].w1, g);
        edge_scatter<DT, C, false>(p.grad, F.t[2], F.d[2].l0, v, u, F.flip[2], F.d[2].w0, g);
        if (F.d[2].l1 >= 0) edge_scatter<DT, C, false>(p.grad, F.t[2], F.d[2].l1, v, u, F.flip[2], F.d[2].w1, g);
    }
}

}  // namespace htex

using namespace htex;

namespace {

constexpr int kThreads = 256;

template <int DT, int C>
htex_status launch_bwd(const htex_textures* t, const BwdParams& p, cudaStream_t s) {
    Asset<GlobalSpace> A;
    A.rec.base = static_cast<const uint8_t*>(t->d_rec);
    A.hdr.base = static_cast<const uint8_t*>(t->d_hdr);
    A.scale.base = static_cast<const uint8_t*>(t->d_scale);
    A.pool.base = static_cast<const uint8_t*>(t->d_pool);
    A.H = t->H;
    A.uniform_log2n = t->uniform_log2n;
    A.uniform_stride16 = uint32_t(t->uniform_stride / 16);
    auto k = k_backward<DT, C>;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, kThreads, 0) != cudaSuccess || b < 1) b = 1;
    const int64_t want = (p.n + kThreads - 1) / kThreads;
    const int64_t grid = std::min<int64_t>(want, int64_t(t->num_sms) * b);
    k<<<unsigned(grid), kThreads, 0, s>>>(A, p);
    return cudaGetLastError() == cudaSuccess ? HTEX_OK : HTEX_ERR_CUDA;
}

template <int DT>
htex_status launch_bwd_c(const htex_textures* t, const BwdParams& p, cudaStream_t s) {
    switch (t->C) {
    case 1: return launch_bwd<DT, 1>(t, p, s);
    case 2: return launch_bwd<DT, 2>(t, p, s);
    case 3: return launch_bwd<DT, 3>(t, p, s);
    case 4: return launch_bwd<DT, 4>(t, p, s);
    }
    return HTEX_ERR_INVALID_ARG;
}

}  // namespace

htex_status htex_launch_backward(const htex_textures* t, const htex_query* q, int64_t n, const float* grad_out,
                                 float* grad_texels, uint32_t flags, htex_stream stream, int32_t* d_status) {
    (void)flags;
    const BwdParams p{q, n, grad_out, grad_texels, d_status};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (t->dtype) {
    case HTEX_F32: return launch_bwd_c<HTEX_F32>(t, p, s);
    case HTEX_U8: return launch_bwd_c<HTEX_U8>(t, p, s);
    case HTEX_F16: return launch_bwd_c<HTEX_F16>(t, p, s);
    case HTEX_BF16: return launch_bwd_c<HTEX_BF16>(t, p, s);
    case HTEX_E4M3: return launch_bwd_c<HTEX_E4M3>(t, p, s);
    }
    return HTEX_ERR_INVALID_ARG;
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
    float* master;
    float* grad;
    float* m;
    float* v;
    float* pool;
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
        __stcs(reinterpret_cast<float4*>(a.pool) + i, p);
        __stcs(reinterpret_cast<float4*>(a.grad) + i, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
    }
    for (int64_t i = 4 * n4 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        float p = a.master[i], m = a.m[i], v = a.v[i];
        adam_one(p, a.grad[i], m, v, a);
        a.master[i] = p;
        a.m[i] = m;
        a.v[i] = v;
        a.pool[i] = p;
        a.grad[i] = 0.0f;
    }
}

extern "C" htex_status htex_textures_adam_step(htex_textures* t, float* master, float* grad, float* m, float* v,
                                               int64_t n, float lr, float beta1, float beta2, float eps,
                                               int32_t step, htex_stream stream) {
    if (!t || t->dtype != HTEX_F32) return HTEX_ERR_INVALID_ARG;
    if (n != t->pool_bytes / 4 || step < 1) return HTEX_ERR_INVALID_ARG;
    if (!master || !grad || !m || !v) return HTEX_ERR_INVALID_ARG;
    const uintptr_t all = reinterpret_cast<uintptr_t>(master) | reinterpret_cast<uintptr_t>(grad) |
                          reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v);
    if ((all & 15u) != 0) return HTEX_ERR_INVALID_ARG;
    if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps > 0.0f)) return HTEX_ERR_INVALID_ARG;
    const double bc1 = 1.0 - std::pow(double(beta1), double(step));
    const double bc2 = 1.0 - std::pow(double(beta2), double(step));
    const AdamParams a{master, grad, m, v, static_cast<float*>(t->d_pool), n, beta1, beta2, eps,
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
