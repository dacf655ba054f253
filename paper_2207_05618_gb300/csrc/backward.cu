// Adjoint of the filtered lookup and the htex_lookup_backward entry point.
//
// The lookup is linear in the stored texels: out_c = sum_k w_k T_k,c / W
// with W the sum of the in-bounds weights of all taps of the three fetches.
// So dL/dT_k,c = sum over queries of grad_out_c * w_k / W.  Per query the
// kernel first recomputes W from the coordinates alone (no texel loads),
// then scatter-adds grad_out * w_k / W into every in-bounds tap with
// nonzero weight: float4/float2 atomics where a texel's channels are
// contiguous and aligned, scalar atomics otherwise.
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

template <int DT, class S>
__device__ __forceinline__ float level_weight(const TexRef& t, int l, float x, float y) {
    Taps k;
    if (!taps(x, y, 1 << (t.n - l), k)) return 0.0f;
    return (k.wx0 + k.wx1) * (k.wy0 + k.wy1);
}

template <int DT, class S>
__device__ __forceinline__ float fetch_weight(const Asset<S>& A, uint32_t code, float a, float b, float lf) {
    float x, y;
    quad_coords(code, a, b, x, y);
    const TexRef t = tex_ref<DT>(A, code & ~kFlipBit);
    const Lod d = select_lod(lf, t.n);
    float w = d.w0 * level_weight<DT, S>(t, d.l0, x, y);
    if (d.l1 >= 0) w = fmaf(d.w1, level_weight<DT, S>(t, d.l1, x, y), w);
    return w;
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
__device__ __forceinline__ void scatter_level(float* grad, const TexRef& t, int l, float x, float y, float wl,
                                              const float (&g)[C]) {
    Taps k;
    if (!taps(x, y, 1 << (t.n - l), k)) return;
    constexpr int ES = Fmt<DT>::ES;
    const uint64_t lvl = (t.off + level_bytes(t.n, l, C * ES)) / ES;   // element index
    add_texel<C>(grad, lvl + uint64_t(k.j0 * k.N + k.i0) * C, wl * k.wy0 * k.wx0, g);
    add_texel<C>(grad, lvl + uint64_t(k.j0 * k.N + k.i1) * C, wl * k.wy0 * k.wx1, g);
    add_texel<C>(grad, lvl + uint64_t(k.j1 * k.N + k.i0) * C, wl * k.wy1 * k.wx0, g);
    add_texel<C>(grad, lvl + uint64_t(k.j1 * k.N + k.i1) * C, wl * k.wy1 * k.wx1, g);
}

template <int DT, int C, class S>
__device__ __forceinline__ void scatter_fetch(const Asset<S>& A, float* grad, uint32_t code, float a, float b,
                                              float lf, const float (&g)[C]) {
    float x, y;
    quad_coords(code, a, b, x, y);
    const TexRef t = tex_ref<DT>(A, code & ~kFlipBit);
    const Lod d = select_lod(lf, t.n);
    scatter_level<DT, C>(grad, t, d.l0, x, y, d.w0, g);
    if (d.l1 >= 0) scatter_level<DT, C>(grad, t, d.l1, x, y, d.w1, g);
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
        const float lf = footprint_log2(f);
        const float W = fetch_weight<DT>(A, rec.x, u, v, lf) + fetch_weight<DT>(A, rec.y, v, -u, lf) +
                        fetch_weight<DT>(A, rec.z, -v, u, lf);
        const float inv = 1.0f / W;
        float g[C];
#pragma unroll
        for (int c = 0; c < C; ++c) g[c] = __ldcs(p.gout + i * C + c) * inv;
        scatter_fetch<DT, C>(A, p.grad, rec.x, u, v, lf, g);
        scatter_fetch<DT, C>(A, p.grad, rec.y, v, -u, lf, g);
        scatter_fetch<DT, C>(A, p.grad, rec.z, -v, u, lf, g);
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
    if (flags & HTEX_LOOKUP_BIN) return HTEX_ERR_UNSUPPORTED;
    return htex_launch_backward(t, q, n, grad_out, grad_texels, flags, stream, d_status);
}
