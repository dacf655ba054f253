// Device-side pieces of the Htex lookup shared by the forward and backward
// kernels: memory spaces (global or shared), texel decoding, the packed
// per-halfedge record, level selection and the border-aware bilinear taps.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "htex_internal.h"

namespace htex {

// ------------------------------------------------------------ memory spaces

// Read-only global memory: texels and records through the non-coherent
// (read-only) cache path.  The *_if loads touch memory only when p holds
// and return zero otherwise (the compiler predicates them).
struct GlobalSpace {
    using off_t = uint64_t;
    const uint8_t* base;
    template <class T>
    __device__ __forceinline__ T at(off_t o) const { return __ldg(reinterpret_cast<const T*>(base + o)); }
    __device__ __forceinline__ uint4 ld16(off_t o) const { return at<uint4>(o); }
    __device__ __forceinline__ uint2 ld8(off_t o) const { return at<uint2>(o); }
    __device__ __forceinline__ uint32_t ld4(off_t o) const { return at<unsigned int>(o); }
    __device__ __forceinline__ uint32_t ld2(off_t o) const { return at<unsigned short>(o); }
    __device__ __forceinline__ uint32_t ld1(off_t o) const { return at<unsigned char>(o); }
    __device__ __forceinline__ uint4 ld16_if(bool p, off_t o) const { return p ? ld16(o) : make_uint4(0u, 0u, 0u, 0u); }
    __device__ __forceinline__ uint2 ld8_if(bool p, off_t o) const { return p ? ld8(o) : make_uint2(0u, 0u); }
    __device__ __forceinline__ uint32_t ld4_if(bool p, off_t o) const { return p ? ld4(o) : 0u; }
    __device__ __forceinline__ uint32_t ld2_if(bool p, off_t o) const { return p ? ld2(o) : 0u; }
    __device__ __forceinline__ uint32_t ld1_if(bool p, off_t o) const { return p ? ld1(o) : 0u; }
    // 4-byte predicated load with an L2 eviction policy (l2_keep_policy or
    // l2_leave_policy).
    __device__ __forceinline__ uint32_t ld4_if_pol(bool p, off_t o, uint64_t pol) const {
        uint32_t r = 0u;
        asm("{\n\t.reg .pred q;\n\t"
            "setp.ne.u32 q, %2, 0;\n\t"
            "@q ld.global.nc.L2::cache_hint.u32 %0, [%1], %3;\n\t}"
            : "+r"(r) : "l"(base + o), "r"(uint32_t(p)), "l"(pol));
        return r;
    }
};

// L2 eviction policies: lines to keep (evict_last) and lines to leave first
// (evict_first).  The asm has no side effects, so the compiler creates each
// policy once and reuses it.
__device__ __forceinline__ uint64_t l2_keep_policy() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t l2_leave_policy() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Shared memory: 'base' points into the kernel's dynamic shared buffer (the
// compiler sees where it comes from and emits shared-window loads); offsets
// are 32-bit.
struct SharedSpace {
    using off_t = uint32_t;
    const uint8_t* base;
    template <class T>
    __device__ __forceinline__ T at(off_t o) const { return *reinterpret_cast<const T*>(base + o); }
    __device__ __forceinline__ uint4 ld16(off_t o) const { return at<uint4>(o); }
    __device__ __forceinline__ uint2 ld8(off_t o) const { return at<uint2>(o); }
    __device__ __forceinline__ uint32_t ld4(off_t o) const { return at<unsigned int>(o); }
    __device__ __forceinline__ uint32_t ld2(off_t o) const { return at<unsigned short>(o); }
    __device__ __forceinline__ uint32_t ld1(off_t o) const { return at<unsigned char>(o); }
    __device__ __forceinline__ uint4 ld16_if(bool p, off_t o) const { return p ? ld16(o) : make_uint4(0u, 0u, 0u, 0u); }
    __device__ __forceinline__ uint2 ld8_if(bool p, off_t o) const { return p ? ld8(o) : make_uint2(0u, 0u); }
    __device__ __forceinline__ uint32_t ld4_if(bool p, off_t o) const { return p ? ld4(o) : 0u; }
    __device__ __forceinline__ uint32_t ld2_if(bool p, off_t o) const { return p ? ld2(o) : 0u; }
    __device__ __forceinline__ uint32_t ld1_if(bool p, off_t o) const { return p ? ld1(o) : 0u; }
};

// ---------------------------------------------------------------- decoding

// ES: bytes per channel; SCALED: decoded codes are multiplied by the
// texture's scale; UNIT: constant factor of every decoded code (applied to
// the tap weights).
template <int DT> struct Fmt;
template <> struct Fmt<HTEX_F32> { static constexpr int ES = 4; static constexpr bool SCALED = false; static constexpr float UNIT = 1.0f; };
template <> struct Fmt<HTEX_U8> { static constexpr int ES = 1; static constexpr bool SCALED = false; static constexpr float UNIT = 1.0f / 255.0f; };
template <> struct Fmt<HTEX_F16> { static constexpr int ES = 2; static constexpr bool SCALED = true; static constexpr float UNIT = 1.0f; };
template <> struct Fmt<HTEX_BF16> { static constexpr int ES = 2; static constexpr bool SCALED = true; static constexpr float UNIT = 1.0f; };
template <> struct Fmt<HTEX_E4M3> { static constexpr int ES = 1; static constexpr bool SCALED = true; static constexpr float UNIT = 1.0f; };

// RGBA8 UNORM: the code b stands for b / 255; the lookup kernels apply the
// 1/255 to the tap weight (Fmt<HTEX_U8>::UNIT) rather than to each channel.
__device__ __forceinline__ float dec_u8(uint32_t b) { return float(b); }
__device__ __forceinline__ float dec_f16(uint32_t b) { return __half2float(__ushort_as_half((unsigned short)b)); }
__device__ __forceinline__ float dec_bf16(uint32_t b) { return __uint_as_float(b << 16); }
__device__ __forceinline__ float dec_e4m3(uint32_t b) {
    __half_raw r = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
    return __half2float(__half(r));
}
__device__ __forceinline__ float2 dec_e4m3x2(uint32_t b2) {
    __half2_raw r = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)b2, __NV_E4M3);
    return __half22float2(__half2(r));
}

template <int DT>
__device__ __forceinline__ float dec1(uint32_t b) {
    if constexpr (DT == HTEX_U8) return dec_u8(b);
    else if constexpr (DT == HTEX_F16) return dec_f16(b);
    else if constexpr (DT == HTEX_BF16) return dec_bf16(b);
    else if constexpr (DT == HTEX_E4M3) return dec_e4m3(b);
    else return __uint_as_float(b);
}

// Byte c of a packed word as a float, exactly: the byte placed in the low
// mantissa bits of 2^23 (one byte permute) minus 2^23 (one add), instead of
// an integer-to-float conversion on the slower conversion pipe.
__device__ __forceinline__ float byte_as_float(uint32_t word, int c) {
    return __uint_as_float(__byte_perm(word, 0x4B000000u, 0x7540u | uint32_t(c))) - 8388608.0f;
}

// Channel c of a packed 8-bit-per-channel texel word, decoded.
template <int DT>
__device__ __forceinline__ float dec_byte(uint32_t word, int c) {
    if constexpr (DT == HTEX_U8) return byte_as_float(word, c);
    else return dec1<DT>((word >> (8 * c)) & 0xffu);
}

// One texel: C decoded (unscaled) channels from byte offset o.
template <int DT, int C, class S>
__device__ __forceinline__ void load_texel(const S& s, typename S::off_t o, float (&t)[C]) {
    constexpr int ES = Fmt<DT>::ES;
    if constexpr (DT == HTEX_F32) {
        if constexpr (C == 4) {
            const uint4 r = s.ld16(o);
            t[0] = __uint_as_float(r.x); t[1] = __uint_as_float(r.y);
            t[2] = __uint_as_float(r.z); t[3] = __uint_as_float(r.w);
        } else if constexpr (C == 2) {
            const uint2 r = s.ld8(o);
            t[0] = __uint_as_float(r.x); t[1] = __uint_as_float(r.y);
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) t[c] = __uint_as_float(s.ld4(o + 4 * c));
        }
    } else if constexpr (ES == 1) {
        if constexpr (C == 4) {
            const uint32_t r = s.ld4(o);
            if constexpr (DT == HTEX_E4M3) {
                const float2 lo = dec_e4m3x2(r & 0xffffu), hi = dec_e4m3x2(r >> 16);
                t[0] = lo.x; t[1] = lo.y; t[2] = hi.x; t[3] = hi.y;
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) t[c] = dec_byte<DT>(r, c);
            }
        } else if constexpr (C == 2) {
            const uint32_t r = s.ld2(o);
            t[0] = dec1<DT>(r & 0xffu); t[1] = dec1<DT>(r >> 8);
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) t[c] = dec1<DT>(s.ld1(o + c));
        }
    } else {  // 16-bit codes
        if constexpr (C == 4) {
            const uint2 r = s.ld8(o);
            t[0] = dec1<DT>(r.x & 0xffffu); t[1] = dec1<DT>(r.x >> 16);
            t[2] = dec1<DT>(r.y & 0xffffu); t[3] = dec1<DT>(r.y >> 16);
        } else if constexpr (C == 2) {
            const uint32_t r = s.ld4(o);
            t[0] = dec1<DT>(r & 0xffffu); t[1] = dec1<DT>(r >> 16);
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) t[c] = dec1<DT>(s.ld2(o + 2 * c));
        }
    }
}

// One texel, loaded only when p (else all channels zero).
template <int DT, int C, class S>
__device__ __forceinline__ void load_texel_if(const S& s, bool p, typename S::off_t o, float (&t)[C]) {
    constexpr int ES = Fmt<DT>::ES;
    if constexpr (DT == HTEX_F32) {
        if constexpr (C == 4) {
            const uint4 r = s.ld16_if(p, o);
            t[0] = __uint_as_float(r.x); t[1] = __uint_as_float(r.y);
            t[2] = __uint_as_float(r.z); t[3] = __uint_as_float(r.w);
        } else if constexpr (C == 2) {
            const uint2 r = s.ld8_if(p, o);
            t[0] = __uint_as_float(r.x); t[1] = __uint_as_float(r.y);
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) t[c] = __uint_as_float(s.ld4_if(p, o + 4 * c));
        }
    } else if constexpr (ES == 1) {
        if constexpr (C == 4) {
            const uint32_t r = s.ld4_if(p, o);
            if constexpr (DT == HTEX_E4M3) {
                const float2 lo = dec_e4m3x2(r & 0xffffu), hi = dec_e4m3x2(r >> 16);
                t[0] = lo.x; t[1] = lo.y; t[2] = hi.x; t[3] = hi.y;
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) t[c] = dec_byte<DT>(r, c);
            }
        } else if constexpr (C == 2) {
            const uint32_t r = s.ld2_if(p, o);
            t[0] = dec1<DT>(r & 0xffu); t[1] = dec1<DT>(r >> 8);
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) t[c] = dec1<DT>(s.ld1_if(p, o + c));
        }
    } else {
        if constexpr (C == 4) {
            const uint2 r = s.ld8_if(p, o);
            t[0] = dec1<DT>(r.x & 0xffffu); t[1] = dec1<DT>(r.x >> 16);
            t[2] = dec1<DT>(r.y & 0xffffu); t[3] = dec1<DT>(r.y >> 16);
        } else if constexpr (C == 2) {
            const uint32_t r = s.ld4_if(p, o);
            t[0] = dec1<DT>(r & 0xffffu); t[1] = dec1<DT>(r >> 16);
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) t[c] = dec1<DT>(s.ld2_if(p, o + 2 * c));
        }
    }
}

// Raw storage of one texel as loaded (decoded later), for the formats whose
// texel fits 8 bytes: one or two registers instead of C floats.
template <int DT, int C>
struct Raw {
    static constexpr int TB = C * Fmt<DT>::ES;
    static constexpr bool PACKED = (TB == 1 || TB == 2 || TB == 4);   // one register per texel
    uint32_t a = 0u, b = 0u;

    template <class S>
    __device__ __forceinline__ void load_if(const S& s, bool p, typename S::off_t o, uint64_t pol) {
        if constexpr (TB == 4 && std::is_same<S, GlobalSpace>::value) {
            a = s.ld4_if_pol(p, o, pol);   // coarse levels stay in L2 across queries
        } else if constexpr (TB == 8) {
            const uint2 r = s.ld8_if(p, o);
            a = r.x;
            b = r.y;
        } else if constexpr (TB == 4) {
            a = s.ld4_if(p, o);
        } else if constexpr (TB == 2) {
            a = s.ld2_if(p, o);
        } else {
            a = s.ld1_if(p, o);
        }
    }

    __device__ __forceinline__ void decode(float (&t)[C]) const {
        if constexpr (DT == HTEX_F32) {
            t[0] = __uint_as_float(a);
            if constexpr (C == 2) t[1] = __uint_as_float(b);
        } else if constexpr (Fmt<DT>::ES == 1) {
            if constexpr (DT == HTEX_E4M3 && C >= 2) {
                const float2 lo = dec_e4m3x2(a & 0xffffu);
                t[0] = lo.x;
                t[1] = lo.y;
                if constexpr (C == 4) {
                    const float2 hi = dec_e4m3x2(a >> 16);
                    t[2] = hi.x;
                    t[3] = hi.y;
                }
            } else {
#pragma unroll
                for (int c = 0; c < C; ++c) t[c] = dec_byte<DT>(a, c);
            }
        } else {
            t[0] = dec1<DT>(a & 0xffffu);
            if constexpr (C >= 2) t[1] = dec1<DT>(a >> 16);
            if constexpr (C == 4) {
                t[2] = dec1<DT>(b & 0xffffu);
                t[3] = dec1<DT>(b >> 16);
            }
        }
    }
};

// ---------------------------------------------------------------- asset

// A resident asset seen from one memory space.
template <class S>
struct Asset {
    S rec;      // int4 per halfedge
    S hdr;      // int4 per edge (unused when uniform)
    S scale;    // float per edge
    S pool;     // texel bytes
    int32_t H;
    int32_t uniform_log2n;      // >= 0: every texture has this resolution
    uint32_t uniform_stride16;  // texture stride / 16 bytes when uniform
};

// The resident asset of a textures handle, seen from global memory.
inline Asset<GlobalSpace> global_asset(const htex_textures* t) {
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

struct TexRef {
    uint64_t off;   // byte offset of the texture in the pool
    int n;          // log2 of the resolution
    float scale;    // code scale (1 for unscaled formats)
};

// UNI: the caller knows every texture of the asset has one resolution
// (uniform_log2n >= 0), so the resolution is the same kernel-wide value for
// every lane and everything derived from it stays warp-uniform.
template <int DT, bool UNI = false, class S>
__device__ __forceinline__ TexRef tex_ref(const Asset<S>& A, uint32_t e) {
    TexRef t;
    if (UNI || A.uniform_log2n >= 0) {
        t.off = uint64_t(e) * A.uniform_stride16 * 16u;
        t.n = A.uniform_log2n;
        t.scale = Fmt<DT>::SCALED ? __uint_as_float(A.scale.ld4(typename S::off_t(e) * 4u)) : 1.0f;
    } else {
        const uint4 h = A.hdr.ld16(typename S::off_t(e) * 16u);
        t.off = uint64_t(h.x) * 16u;
        t.n = int(h.y);
        t.scale = Fmt<DT>::SCALED ? __uint_as_float(h.z) : 1.0f;
    }
    return t;
}

// Texels before level l in a chain of base 2^n: sum_{k<l} 4^(n-k)
// = 4^(n-l+1) (4^l - 1) / 3, where (4^l - 1) / 3 is the bit pattern 0101..01
// (l pairs).  Fits 32 bits for n <= 15.
__device__ __forceinline__ uint32_t level_texels(int n, int l) {
    return l ? ((0x55555555u & ((1u << (2 * l)) - 1u)) << (2 * (n - l + 1))) : 0u;
}

// Level choice of one fetch: levels l0 (weight w0) and l1 (weight w1, l1 < 0
// when a single level is used).  lam = log2(footprint) + n; level 0 unless
// lam > 0; the last level once floor(lam) reaches it.
struct Lod {
    int l0, l1;
    float w0, w1;
};

__device__ __forceinline__ Lod select_lod(float log2f_fp, int n) {
    Lod d{0, -1, 1.0f, 0.0f};
    const float lam = log2f_fp + float(n);
    if (lam > 0.0f) {
        const float fl = floorf(lam);
        if (fl >= float(n)) {
            d.l0 = n;
        } else {
            d.l0 = int(fl);
            d.l1 = d.l0 + 1;
            d.w1 = lam - fl;
            d.w0 = 1.0f - d.w1;
        }
    }
    return d;
}

// Two taps along one axis at coordinate p in [0, 1] on a level of N
// texels with a zero border: texel centres at (i + 1/2) / N, so
// s = p N - 1/2, taps floor(s) and floor(s) + 1 with weights 1 - a and a
// (a = s - floor(s)); floor(s) >= -1 and floor(s) + 1 <= N for p in [0, 1],
// so only the two end texels can fall outside (weight zero).
struct Taps1 {
    int i0, i1;     // clamped indices
    float w0, w1;   // in-bounds weights
};

__device__ __forceinline__ Taps1 taps1(float p, int N) {
    const float s = fmaf(p, float(N), -0.5f);
    const float fi = floorf(s);
    const float a = s - fi;
    const int i = int(fi);
    Taps1 t;
    t.w0 = (i >= 0) ? 1.0f - a : 0.0f;
    t.w1 = (i + 1 < N) ? a : 0.0f;
    t.i0 = max(i, 0);
    t.i1 = min(i + 1, N - 1);
    return t;
}

// The same two taps for the forward fetches: the first index i = floor(s)
// unclamped (in [-1, N - 1]; the second tap is i + 1) and the same weights.
// A tap outside [0, N) has weight exactly zero and is never loaded, so the
// offsets can be formed from i without clamping.
struct TapsU {
    int i;
    float w0, w1;
};

__device__ __forceinline__ TapsU taps_u(float p, int N) {
    const float s = fmaf(p, float(N), -0.5f);
    const float fi = floorf(s);
    const float a = s - fi;
    const int i = int(fi);
    return TapsU{i, i >= 0 ? 1.0f - a : 0.0f, i + 1 < N ? a : 0.0f};
}

// Alg. 3's three fetches, after the query is clamped onto its triangle
// (u, v >= 0, u + v <= 1):
//   own    quad of h at (u, v) or (1 - u, 1 - v): inside [0, 1]^2, a 2x2 tap
//          block per level;
//   Next   quad of Next(h) at (v, -u) or (1 - v, 1 + u): the y coordinate lies
//          u outside the quad, so only row 0 (row N - 1 when reflected) can
//          be in bounds, with weight max(0, 1/2 - u N), and x = v (1 - v) is
//          in [0, 1]: two taps per level;
//   Prev   quad of Prev(h) at (-v, u) or (1 + v, 1 - u): only column 0
//          (column N - 1) with weight max(0, 1/2 - v N), y = u (1 - u):
//          two taps per level.
// These are the bilinear taps of a zero-bordered sample written out for
// the coordinates Alg. 3 produces; no tap with nonzero in-bounds weight is
// left out.
__device__ __forceinline__ float across_weight(float dist, int N) {
    return fmaf(-dist, float(N), 0.5f);
}

// Taps of the own fetch at one level: the byte offset o (from the texture
// start) of tap (i, j), the others at o + TB, o + row and o + row + TB;
// their weights (level weight included) in the order (i, j), (i + 1, j),
// (i, j + 1), (i + 1, j + 1), and the level's share of the normalisation
// sum.  A tap of weight zero is never loaded (its offset may lie outside
// the texture).
struct OwnPlan {
    int32_t o, row;
    float w[4];
    float ws;
};

template <int TB>
__device__ __forceinline__ OwnPlan own_plan(int n, int l, float x, float y, float wl) {
    const int N = 1 << (n - l);
    const TapsU tx = taps_u(x, N), ty = taps_u(y, N);
    OwnPlan q;
    q.row = N * TB;
    q.o = int32_t(level_texels(n, l)) * TB + (ty.i * N + tx.i) * TB;
    const float y0 = ty.w0 * wl, y1 = ty.w1 * wl;
    q.w[0] = y0 * tx.w0;
    q.w[1] = y0 * tx.w1;
    q.w[2] = y1 * tx.w0;
    q.w[3] = y1 * tx.w1;
    q.ws = wl * (tx.w0 + tx.w1) * (ty.w0 + ty.w1);
    return q;
}

// Taps of a Next (row = true) or Prev fetch at one level: the two texels of
// the row or column on the shared side, at o and o + step, with weights
// including the across weight and the level weight (all zero when the
// query lies too far away).
struct EdgePlan {
    int32_t o, step;
    float w[2];
    float ws;
};

template <int TB>
__device__ __forceinline__ EdgePlan edge_plan(int n, int l, float dist, float along, bool flip, bool row,
                                              float wl) {
    const int N = 1 << (n - l);
    const float wa = across_weight(dist, N);
    const float waw = wa > 0.0f ? wa * wl : 0.0f;
    const TapsU ta = taps_u(flip ? 1.0f - along : along, N);
    const int k = flip ? N - 1 : 0;
    // texel (i, k) of the row or (k, i) of the column, row-major j * N + i
    const int stride_i = row ? 1 : N, fixed = row ? k * N : k;
    EdgePlan e;
    e.step = stride_i * TB;
    e.o = int32_t(level_texels(n, l)) * TB + (fixed + ta.i * stride_i) * TB;
    e.w[0] = ta.w0 * waw;
    e.w[1] = ta.w1 * waw;
    e.ws = waw * (ta.w0 + ta.w1);
    return e;
}

// Coordinates of one of Alg. 3's fetches in its quad (Alg. 2): reflected
// when the halfedge is the smaller id of its pair.
__device__ __forceinline__ void quad_coords(uint32_t code, float a, float b, float& x, float& y) {
    const bool flip = code & kFlipBit;
    x = flip ? 1.0f - a : a;
    y = flip ? 1.0f - b : b;
}

// Query decode: invalid when h is out of range or u, v are not finite;
// finite (u, v) are clamped onto the closed triangle.
__device__ __forceinline__ bool decode_query(int4 raw, int32_t H, int& h, float& u, float& v, float& f) {
    h = raw.x;
    u = __int_as_float(raw.y);
    v = __int_as_float(raw.z);
    f = __int_as_float(raw.w);
    if (unsigned(h) >= unsigned(H) || !(fabsf(u) <= 3.402823466e38f) || !(fabsf(v) <= 3.402823466e38f))
        return false;
    u = fmaxf(u, 0.0f);
    v = fmaxf(v, 0.0f);
    float s = u + v;
    if (s > 3.402823466e38f) {  // both huge: halve first so the sum stays finite
        u *= 0.5f;
        v *= 0.5f;
        s = u + v;
    }
    if (s > 1.0f) {
        u = u / s;
        v = v / s;
    }
    return true;
}

// log2 of the footprint, or -inf when level 0 is forced (footprint <= 0 or NaN).
__device__ __forceinline__ float footprint_log2(float f) {
    return (f > 0.0f) ? log2f(f) : -__int_as_float(0x7f800000);
}

// Bring a future query's line into L2 (no register, no wait).
template <class I>
__device__ __forceinline__ void prefetch_query(const htex_query* q, I i) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const int4*>(q) + i));
}

// Streaming 16-byte query load: bypasses L1 and is marked first to leave L2.
template <class I>
__device__ __forceinline__ int4 ld_query(const htex_query* q, I i) {
    int4 r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(reinterpret_cast<const int4*>(q) + i), "l"(l2_leave_policy()));
    return r;
}

}  // namespace htex
