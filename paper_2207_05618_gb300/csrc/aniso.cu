// Anisotropic filtered lookup and the htex_lookup_aniso entry point.
//
// Section 5.1 renders Htex through the GPU's anisotropic filter, applied to
// each of Alg. 3's three texture fetches; the paper states no formula, so
// this follows one reading, the same as the FP64 oracle's:
//   - the footprint is given by the screen derivatives of the barycentrics,
//     ax = (du/dx, dv/dx) and ay = (du/dy, dv/dy), in quad-uv units;
//   - px2 = |ax|^2, py2 = |ay|^2 (each product and sum rounded to float);
//     the major axis m is ay when py2 > px2, else ax; the probe count K is 1
//     when both are zero, else min(ceil(sqrt(max / min)), kmax), computed
//     with correctly rounded float division and square root so that the
//     integer K is decided exactly as the oracle decides it;
//   - each probe is an isotropic trilinear sample with footprint Pmax / K;
//   - probe k sits at c + m * s * ((k + 1/2) / K - 1/2) with s = min(1,
//     K / Pmax) (the probes never span more than K quad widths);
//   - every probe samples all three fetches at its own (u', v'): own quad
//     at (u', v'), Next's at (v', -u'), Prev's at (-v', u'), each through
//     Alg. 2, with full 2x2 zero-bordered taps (a probe off the triangle can
//     reach any texel of the neighbouring quads); the result is the summed
//     data over the summed normalisation weight.
// Work distribution: a warp takes 32 queries at a time and works through
// all of their probes together, 32 (query, probe) pairs per round, so a
// warp whose lanes need 1 to 16 probes runs ceil(sum K / 32) rounds instead
// of its largest K.  Each query's constants (centre, scaled major axis, K,
// and for each fetch its two levels' offsets, sizes and weights, code
// factor and reflection) are computed once by its own lane and kept in
// shared memory for the lanes that run its probes; each round's probe
// results (data and weight sums) go through shared memory back to the
// lanes of their queries, which add them in probe order, so that a query's
// result does not depend on which other queries share its warp.  A fetch whose
// quad no probe of the round can reach (more than half a coarsest-level
// texel outside it) is skipped warp-uniformly.
#include <cuda_runtime.h>

#include "lookup_core.cuh"
#include "aniso_launch.h"

namespace htex {

struct AnisoParams {
    const htex_query_aniso* q;
    int64_t n;
    int32_t kmax;
    float* out;
    int32_t* status;
};

// Two taps along one axis for an arbitrary coordinate: index i = floor(s)
// unclamped, in-bounds weights (zero for a tap outside [0, N)).
struct TapsG {
    int i;
    float w0, w1;
};

__device__ __forceinline__ TapsG taps_g(float p, int N) {
    const float s = fmaf(p, float(N), -0.5f);
    const float fi = floorf(s);
    const float a = s - fi;
    const int i = int(fi);
    return TapsG{i, (i >= 0 && i < N) ? 1.0f - a : 0.0f, (i + 1 >= 0 && i + 1 < N) ? a : 0.0f};
}

// Per-query constants of one fetch, fixed over its probes: where its two
// levels start, their sizes and weights, the code factor and the Alg. 2
// reflection.
struct FetchConst {
    int64_t base0;          // byte offset of texel (0, 0) of level l0
    int32_t d1;             // byte offset of level l1 from level l0 (0 when one level is read)
    int16_t n0, n1;         // log2 of their sizes (l1 = l0 when one level is read)
    float w0, w1;           // their weights (w1 = 0 when one level is read)
    float sc;               // code factor
    uint32_t flip;          // Alg. 2 reflection
};

template <int DT, int C>
__device__ __forceinline__ FetchConst fetch_const(const TexRef& t, const Lod& d, uint32_t code) {
    constexpr int TB = C * Fmt<DT>::ES;
    FetchConst f;
    const int l1 = d.l1 >= 0 ? d.l1 : d.l0;
    f.n0 = int16_t(t.n - d.l0);
    f.n1 = int16_t(t.n - l1);
    f.base0 = int64_t(t.off) + int64_t(level_texels(t.n, d.l0)) * TB;
    f.d1 = int32_t(int64_t(level_texels(t.n, l1) - level_texels(t.n, d.l0)) * TB);
    f.w0 = d.w0;
    f.w1 = d.l1 >= 0 ? d.w1 : 0.0f;
    f.sc = code_factor<DT>(t);
    f.flip = code & kFlipBit;
    return f;
}

// One level of one fetch at quad coordinates (x, y) with level weight wl.
template <int DT, int C>
__device__ __forceinline__ void aniso_level(const Asset<GlobalSpace>& A, int64_t base, int N, float x, float y,
                                            float wl, float sc, float (&acc)[C], float& W) {
    constexpr int TB = C * Fmt<DT>::ES;
    const TapsG tx = taps_g(x, N), ty = taps_g(y, N);
    W += wl * (tx.w0 + tx.w1) * (ty.w0 + ty.w1);
    const float y0 = ty.w0 * wl, y1 = ty.w1 * wl;
    const float w[4] = {y0 * tx.w0, y0 * tx.w1, y1 * tx.w0, y1 * tx.w1};
    const int64_t o = base + (int64_t(ty.i) * N + tx.i) * TB;
    const int64_t d[4] = {0, TB, int64_t(N) * TB, int64_t(N) * TB + TB};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float v[C];
        load_texel_if<DT, C>(A.pool, w[k] != 0.0f, uint64_t(o + d[k]), v);
        const float wd = w[k] * sc;
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = fmaf(wd, v[c], acc[c]);
    }
}

// One fetch of one probe (one or two levels), skipped when no lane of the
// warp has a tap in bounds.
template <int DT, int C>
__device__ __forceinline__ void aniso_fetch(const Asset<GlobalSpace>& A, bool on, const FetchConst& f, float a,
                                            float b, float (&acc)[C], float& W) {
    const float x = f.flip ? 1.0f - a : a, y = f.flip ? 1.0f - b : b;
    const float half = __int_as_float((126 - f.n1) << 23);   // 2^-(n1 + 1): half a texel of the coarser level
    const bool near = on && x > -half && x < 1.0f + half && y > -half && y < 1.0f + half;
    if (!__any_sync(0xffffffffu, near)) return;
    aniso_level<DT, C>(A, f.base0, 1 << f.n0, x, y, near ? f.w0 : 0.0f, f.sc, acc, W);
    const bool two = near && f.w1 != 0.0f;
    if (__any_sync(0xffffffffu, two))
        aniso_level<DT, C>(A, f.base0 + f.d1, 1 << f.n1, x, y, two ? f.w1 : 0.0f, f.sc, acc, W);
}

// Probe count (see the file comment): same float operations as the oracle.
__device__ __forceinline__ int aniso_probes(float px2, float py2, int kmax) {
    const float mx = fmaxf(px2, py2), mn = fminf(px2, py2);
    if (mx == 0.0f) return 1;
    const float r = __fsqrt_rn(__fdiv_rn(mx, mn));
    if (!(r < float(kmax))) return kmax;
    return max(1, int(ceilf(r)));
}

// One block of 1024 threads per SM (156 KiB of per-warp shared state):
// measured 7% faster than four blocks of 256 per SM on the asset-scale
// anisotropic batch
constexpr int kAnisoThreads = 1024;
constexpr int kAnisoWarps = kAnisoThreads / 32;
constexpr int kAnisoMaxK = 16;

// One query's constants, written by its lane, read by the lanes that run
// its probes.  120 bytes (30 words), so that lanes reading the same field
// of different queries hit different shared-memory banks (a size of 32
// words put them all in one bank).
struct AnisoQuery {
    float u, v, mu, mv;     // centre and the probe spacing axis (major axis times s)
    int32_t K;              // probes (0: the lane holds no query)
    float inv2K;            // +-1 / (2K), negative for an invalid query: probe k sits at t = (2k + 1 - K) / (2K)
    FetchConst f[3];        // own, Next, Prev
};
static_assert(sizeof(AnisoQuery) == 120, "AnisoQuery: 30 words (bank spread)");

template <int DT, int C>
__global__ void __launch_bounds__(kAnisoThreads) k_lookup_aniso(Asset<GlobalSpace> A, AnisoParams p) {
    __shared__ AnisoQuery sq[kAnisoWarps][32];
    __shared__ uint8_t owner[kAnisoWarps][32 * kAnisoMaxK];   // the query lane of each of the warp's probes
    __shared__ float pr[kAnisoWarps][C + 1][32];             // one round's probe results: data and weight sums
    const unsigned lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    const int64_t warps = int64_t(gridDim.x) * kAnisoWarps;
    for (int64_t base = (int64_t(blockIdx.x) * kAnisoWarps + wib) * 32; base < p.n; base += warps * 32) {
        // ---- this lane's query: decode, probe count, per-fetch constants
        const int64_t i = base + lane;
        const bool valid = i < p.n;
        const int4 r0 = valid ? ld_query(reinterpret_cast<const htex_query*>(p.q), 2 * i) : make_int4(-1, 0, 0, 0);
        const int4 r1 = valid ? ld_query(reinterpret_cast<const htex_query*>(p.q), 2 * i + 1) : make_int4(0, 0, 0, 0);
        const float dudx = __int_as_float(r1.x), dvdx = __int_as_float(r1.y);
        const float dudy = __int_as_float(r1.z), dvdy = __int_as_float(r1.w);
        const float px2 = __fadd_rn(__fmul_rn(dudx, dudx), __fmul_rn(dvdx, dvdx));
        const float py2 = __fadd_rn(__fmul_rn(dudy, dudy), __fmul_rn(dvdy, dvdy));
        int h;
        float u, v, f;
        bool ok = valid && decode_query(make_int4(r0.x, r0.y, r0.z, 0), A.H, h, u, v, f);
        ok = ok && isfinite(dudx) && isfinite(dvdx) && isfinite(dudy) && isfinite(dvdy) && isfinite(px2) &&
             isfinite(py2);
        if (!ok) {
            u = 0.0f;
            v = 0.0f;
            if (valid && p.status) atomicAdd(p.status, 1);
        }
        const int K = valid ? (ok ? aniso_probes(px2, py2, p.kmax) : 1) : 0;
        const bool major_y = py2 > px2;
        const float pmax = sqrtf(fmaxf(px2, py2));
        const float s = pmax > float(max(K, 1)) ? float(K) / pmax : 1.0f;
        const float lf = footprint_log2(ok ? pmax / float(K) : 0.0f);
        const uint4 rec = ok ? A.rec.ld16(uint64_t(h) * 16u) : make_uint4(0, 0, 0, 0);
        const TexRef to = tex_ref<DT>(A, rec.x & ~kFlipBit);
        const TexRef tn = tex_ref<DT>(A, rec.y & ~kFlipBit);
        const TexRef tp = tex_ref<DT>(A, rec.z & ~kFlipBit);
        AnisoQuery& Q = sq[wib][lane];
        Q.u = u;
        Q.v = v;
        Q.mu = (major_y ? dudy : dudx) * s;
        Q.mv = (major_y ? dvdy : dvdx) * s;
        Q.K = K;
        Q.inv2K = (ok ? 1.0f : -1.0f) / float(2 * max(K, 1));
        Q.f[0] = fetch_const<DT, C>(to, select_lod(lf, to.n), rec.x);
        Q.f[1] = fetch_const<DT, C>(tn, select_lod(lf, tn.n), rec.y);
        Q.f[2] = fetch_const<DT, C>(tp, select_lod(lf, tp.n), rec.z);
        float qacc[C];
#pragma unroll
        for (int c = 0; c < C; ++c) qacc[c] = 0.0f;
        float qW = 0.0f;

        // ---- the warp's probes in order: query lane by lane, probe by probe
        int incl = K;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= unsigned(d)) incl += o;
        }
        const int first = incl - K;                          // this lane's first probe
        const int P = __shfl_sync(0xffffffffu, incl, 31);     // the warp's probes
        for (int k = 0; k < K; ++k) owner[wib][first + k] = uint8_t(lane);
        __syncwarp();

        for (int r0p = 0; r0p < P; r0p += 32) {
            const int j = r0p + int(lane);
            const bool has = j < P;
            const int q = has ? owner[wib][j] : int(owner[wib][P - 1]);
            const int qfirst = __shfl_sync(0xffffffffu, first, q);
            const AnisoQuery& R = sq[wib][q];
            const bool on = has && R.inv2K > 0.0f;
            const int KR = R.K, k = j - qfirst;
            const float t = float(2 * k + 1 - KR) * R.inv2K;
            const float pu = fmaf(R.mu, t, R.u), pv = fmaf(R.mv, t, R.v);
            float acc[C];
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = 0.0f;
            float W = 0.0f;
            aniso_fetch<DT, C>(A, on, R.f[0], pu, pv, acc, W);
            aniso_fetch<DT, C>(A, on, R.f[1], pv, -pu, acc, W);
            aniso_fetch<DT, C>(A, on, R.f[2], -pv, pu, acc, W);
#pragma unroll
            for (int c = 0; c < C; ++c) pr[wib][c][lane] = acc[c];
            pr[wib][C][lane] = W;
            __syncwarp();
            // each lane adds the probes of its own query that this round
            // computed, in probe order: the same sums whatever the other
            // queries of the warp are
            const int a = max(first, r0p) - r0p, b = min(first + K, r0p + 32) - r0p;
            for (int m = a; m < b; ++m) {
#pragma unroll
                for (int c = 0; c < C; ++c) qacc[c] += pr[wib][c][m];
                qW += pr[wib][C][m];
            }
            __syncwarp();
        }

        // ---- normalise and store (invalid queries: W = 0, data 0, 0 * inf = NaN)
        if (valid) {
            const float inv = __frcp_rn(qW);
            float res[C];
#pragma unroll
            for (int c = 0; c < C; ++c) res[c] = qacc[c] * inv;
            store_out<C>(p.out, i, res);
        }
        __syncwarp();
    }
}

template <int DT, int C>
htex_status launch_aniso_c(const htex_textures* t, const AnisoParams& p, cudaStream_t s) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_lookup_aniso<DT, C>, kAnisoThreads, 0) != cudaSuccess ||
        b < 1)
        b = 1;
    const int64_t want = (p.n + kAnisoThreads - 1) / kAnisoThreads;
    const int64_t grid = std::min<int64_t>(want, int64_t(t->num_sms) * b);
    k_lookup_aniso<DT, C><<<unsigned(grid), kAnisoThreads, 0, s>>>(global_asset(t), p);
    return cudaGetLastError() == cudaSuccess ? HTEX_OK : HTEX_ERR_CUDA;
}

template <int DT>
htex_status launch_aniso_dt(const htex_textures* t, const AnisoParams& p, cudaStream_t s) {
    switch (t->C) {
    case 1: return launch_aniso_c<DT, 1>(t, p, s);
    case 2: return launch_aniso_c<DT, 2>(t, p, s);
    case 3: return launch_aniso_c<DT, 3>(t, p, s);
    case 4: return launch_aniso_c<DT, 4>(t, p, s);
    }
    return HTEX_ERR_INVALID_ARG;
}

}  // namespace htex

using namespace htex;

htex_status htex_launch_aniso(const htex_textures* t, const htex_query_aniso* q, int64_t n, int32_t kmax,
                              float* out, htex_stream stream, int32_t* d_status) {
    const AnisoParams p{q, n, kmax, out, d_status};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (t->dtype) {
    case HTEX_F32: return launch_aniso_dt<HTEX_F32>(t, p, s);
    case HTEX_U8: return launch_aniso_dt<HTEX_U8>(t, p, s);
    case HTEX_F16: return launch_aniso_dt<HTEX_F16>(t, p, s);
    case HTEX_BF16: return launch_aniso_dt<HTEX_BF16>(t, p, s);
    case HTEX_E4M3: return launch_aniso_dt<HTEX_E4M3>(t, p, s);
    }
    return HTEX_ERR_INVALID_ARG;
}

extern "C" htex_status htex_lookup_aniso(const htex_textures* t, const htex_query_aniso* q, int64_t n,
                                         int32_t max_aniso, uint32_t flags, float* out, htex_stream stream,
                                         int32_t* d_status) {
    if (!t || n < 0 || max_aniso < 1 || max_aniso > 16) return HTEX_ERR_INVALID_ARG;
    if (flags & ~uint32_t(HTEX_LOOKUP_BIN)) return HTEX_ERR_INVALID_ARG;
    if (n == 0) return HTEX_OK;
    if (!q || !out) return HTEX_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(q) & 15u) != 0) return HTEX_ERR_INVALID_ARG;
    const uintptr_t out_align = t->C == 4 ? 16u : (t->C == 2 ? 8u : 4u);
    if ((reinterpret_cast<uintptr_t>(out) & (out_align - 1)) != 0) return HTEX_ERR_INVALID_ARG;
    if (flags & HTEX_LOOKUP_BIN) return htex_launch_aniso_sorted(t, q, n, max_aniso, out, stream, d_status);
    return htex_launch_aniso(t, q, n, max_aniso, out, stream, d_status);
}
