// Per-query device code of the filtered lookup (paper Section 4.4, Alg. 3
// with Alg. 2), shared by the lookup kernels and the serving kernels.
#pragma once

#include "fetch.cuh"

namespace htex {

struct FwdParams {
    const htex_query* q;
    int64_t n;
    float* out;
    int32_t* status;
    const int32_t* idx;   // binned: original index of each sorted query
};

// Levels of at most 2^kCoarseLog2 texels a side are read with an L2
// keep hint (about 84 bytes of RGBA8 per texture: L2-resident for assets of
// hundreds of thousands of textures), finer ones with a leave-first hint.
constexpr int kCoarseLog2 = 2;

// Coarsest level a fetch reads (its texels are the widest).
__device__ __forceinline__ int coarsest(const Lod& d) { return d.l1 >= 0 ? d.l1 : d.l0; }

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

// The record of a query's halfedge (zeros when the id is out of range;
// such a query is rejected before the record is used).
template <class S>
__device__ __forceinline__ uint4 record_of(const Asset<S>& A, int4 raw) {
    if (unsigned(raw.x) >= unsigned(A.H)) return make_uint4(0, 0, 0, 0);
    return A.rec.ld16(typename S::off_t(raw.x) * 16u);
}

// The taps of one query, gathered in slots: up to 4 + 4 (own, two levels)
// and 2 + 2 for each of Next and Prev.  With DEFER (packed texel formats
// read from global memory) every load of nonzero weight is issued into a
// raw register first and the decoding and weighting happen after all of
// them are in flight; otherwise each slot is weighted as it is loaded.
template <int DT, int C, bool DEFER>
struct Gather {
    static constexpr int K = 16;
    Raw<DT, C> raw[DEFER ? K : 1];
    float w[DEFER ? K : 1];
    float acc[C];
    float W = 0.0f;

    __device__ __forceinline__ Gather() {
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = 0.0f;
        // slots of parts the warp skips keep weight zero
#pragma unroll
        for (int k = 0; k < (DEFER ? K : 1); ++k) w[k] = 0.0f;
    }

    // slot k: when 'on', load the texel at byte offset o; data weight wd
    // (W += ws done by the caller)
    template <int k, class S>
    __device__ __forceinline__ void tap(const S& pool, typename S::off_t o, bool on, float wd, uint64_t pol) {
        if constexpr (DEFER) {
            w[k] = wd;
            raw[k].load_if(pool, on, o, pol);
        } else {
            float t[C];
            load_texel_if<DT, C>(pool, on, o, t);
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = fmaf(wd, t[c], acc[c]);
        }
    }

    __device__ __forceinline__ void finish() {
        if constexpr (DEFER) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float t[C];
                raw[k].decode(t);
#pragma unroll
                for (int c = 0; c < C; ++c) acc[c] = fmaf(w[k], t[c], acc[c]);
            }
        }
    }
};

// Data weight factor of a texture's decoded codes: its scale (scaled
// formats) times the format's unit (1/255 for RGBA8).
template <int DT>
__device__ __forceinline__ float code_factor(const TexRef& t) {
    return (Fmt<DT>::SCALED ? t.scale : 1.0f) * Fmt<DT>::UNIT;
}

// Taps are loaded only where their weight (before the code factor) is
// nonzero: exactly the taps inside the texture.
template <int DT, int C, int k0, bool DEFER, class S>
__device__ __forceinline__ void own_taps(const Asset<S>& A, const TexRef& t, int l, float x, float y, float wl,
                                         Gather<DT, C, DEFER>& g) {
    using off_t = typename S::off_t;
    constexpr int TB = C * Fmt<DT>::ES;
    const OwnPlan q = own_plan<TB>(t.n, l, x, y, wl);
    const uint64_t pol = t.n - l <= kCoarseLog2 ? l2_keep_policy() : l2_leave_policy();
    const float sc = code_factor<DT>(t);
    g.W += q.ws;
    const off_t b = off_t(t.off) + off_t(int64_t(q.o)), r = off_t(q.row);
    g.template tap<k0 + 0>(A.pool, b, q.w[0] != 0.0f, q.w[0] * sc, pol);
    g.template tap<k0 + 1>(A.pool, b + TB, q.w[1] != 0.0f, q.w[1] * sc, pol);
    g.template tap<k0 + 2>(A.pool, b + r, q.w[2] != 0.0f, q.w[2] * sc, pol);
    g.template tap<k0 + 3>(A.pool, b + r + TB, q.w[3] != 0.0f, q.w[3] * sc, pol);
}

template <int DT, int C, int k0, bool DEFER, class S>
__device__ __forceinline__ void edge_taps(const Asset<S>& A, const TexRef& t, int l, float dist, float along,
                                          bool flip, bool row, float wl, Gather<DT, C, DEFER>& g) {
    using off_t = typename S::off_t;
    constexpr int TB = C * Fmt<DT>::ES;
    const EdgePlan e = edge_plan<TB>(t.n, l, dist, along, flip, row, wl);
    const uint64_t pol = t.n - l <= kCoarseLog2 ? l2_keep_policy() : l2_leave_policy();
    const float sc = code_factor<DT>(t);
    g.W += e.ws;
    const off_t b = off_t(t.off) + off_t(int64_t(e.o));
    g.template tap<k0 + 0>(A.pool, b, e.w[0] != 0.0f, e.w[0] * sc, pol);
    g.template tap<k0 + 1>(A.pool, b + off_t(e.step), e.w[1] != 0.0f, e.w[1] * sc, pol);
}

// One edge fetch (Next: row, dist u, along v; Prev: column, dist v, along
// u), one or two levels, for the lanes with 'on' set.
template <int DT, int C, int k0, bool L0, bool DEFER, class S>
__device__ __forceinline__ void edge_fetch(const Asset<S>& A, unsigned act, bool on, const TexRef& t, const Lod& d,
                                           float dist, float along, bool flip, bool row, Gather<DT, C, DEFER>& g) {
    edge_taps<DT, C, k0>(A, t, L0 ? 0 : d.l0, dist, along, flip, row, on ? (L0 ? 1.0f : d.w0) : 0.0f, g);
    if constexpr (!L0) {
        const bool two = on && d.l1 >= 0;
        if (__any_sync(act, two))
            edge_taps<DT, C, k0 + 2>(A, t, two ? d.l1 : d.l0, dist, along, flip, row, two ? d.w1 : 0.0f, g);
    }
}

// Alg. 3 for one query: the own fetch (one or two levels), then the Next
// and Prev fetches (one texel row / column per level).  A lane needs both
// edge fetches only within half a texel of the face centroid, so the lanes
// of a warp share one edge pass, each running the edge it needs (Next if
// any, else Prev); a second pass runs Prev for the lanes that need both.
// Every load of nonzero weight is issued without branching; parts no lane
// of the warp needs are skipped warp-uniformly.  L0: no lane of the warp
// has a positive footprint, so every fetch is level 0 only.
template <int DT, int C, bool L0, bool DEFER, bool UNI, class S>
__device__ __forceinline__ void lookup_body(const Asset<S>& A, const FwdParams& p, unsigned act, bool ok, float u,
                                            float v, float f, uint4 rec, int64_t dst) {
    const bool uni = UNI || A.uniform_log2n >= 0;
    const float lf = L0 ? -__int_as_float(0x7f800000) : footprint_log2(f);
    Gather<DT, C, DEFER> g;

    // own quad at (u, v), through Alg. 2
    const TexRef to = tex_ref<DT, UNI>(A, rec.x & ~kFlipBit);
    const Lod d = L0 ? Lod{0, -1, 1.0f, 0.0f} : select_lod(lf, to.n);
    const bool fo = rec.x & kFlipBit;
    const float x = fo ? 1.0f - u : u, y = fo ? 1.0f - v : v;
    own_taps<DT, C, 0>(A, to, L0 ? 0 : d.l0, x, y, ok ? (L0 ? 1.0f : d.w0) : 0.0f, g);
    if constexpr (!L0) {
        const bool two = ok && d.l1 >= 0;
        if (__any_sync(act, two)) own_taps<DT, C, 4>(A, to, two ? d.l1 : d.l0, x, y, two ? d.w1 : 0.0f, g);
    }

    // which edge fetches have taps in bounds (at the coarsest level read)
    const TexRef tn = tex_ref<DT, UNI>(A, rec.y & ~kFlipBit);
    const TexRef tp = tex_ref<DT, UNI>(A, rec.z & ~kFlipBit);
    const Lod dn = (L0 || uni) ? d : select_lod(lf, tn.n);
    const Lod dp = (L0 || uni) ? d : select_lod(lf, tp.n);
    const bool nn = ok && across_weight(u, 1 << (tn.n - coarsest(dn))) > 0.0f;
    const bool pp = ok && across_weight(v, 1 << (tp.n - coarsest(dp))) > 0.0f;

    if (__any_sync(act, nn || pp)) {   // first edge pass: Next where needed, else Prev
        const bool row = nn;
        edge_fetch<DT, C, 8, L0>(A, act, nn || pp, row ? tn : tp, row ? dn : dp, row ? u : v, row ? v : u,
                                 ((row ? rec.y : rec.z) & kFlipBit) != 0, row, g);
    }
    if (__any_sync(act, nn && pp))     // second pass: Prev for lanes that need both
        edge_fetch<DT, C, 12, L0>(A, act, nn && pp, tp, dp, v, u, (rec.z & kFlipBit) != 0, false, g);

    g.finish();
    // an invalid query has every weight zero: W = 0, 1/W = inf, 0 * inf = NaN
    const float inv = __frcp_rn(g.W);
    float r[C];
#pragma unroll
    for (int c = 0; c < C; ++c) r[c] = g.acc[c] * inv;
    store_out<C>(p.out, dst, r);
}

template <int DT, int C, bool DEFER, bool UNI = false, class S>
__device__ __forceinline__ void lookup_one(const Asset<S>& A, const FwdParams& p, int4 raw, uint4 rec,
                                           int64_t dst) {
    int h;
    float u, v, f;
    const bool ok = decode_query(raw, A.H, h, u, v, f);
    if (!ok) {
        u = 0.0f;
        v = 0.0f;
        f = 0.0f;
        if (p.status) atomicAdd(p.status, 1);
    }
    const unsigned act = __activemask();
    if (__any_sync(act, f > 0.0f)) lookup_body<DT, C, false, DEFER, UNI>(A, p, act, ok, u, v, f, rec, dst);
    else lookup_body<DT, C, true, DEFER, UNI>(A, p, act, ok, u, v, f, rec, dst);
}

}  // namespace htex
