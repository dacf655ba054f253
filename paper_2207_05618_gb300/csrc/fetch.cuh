// Device-side pieces of the Htex lookup shared by the forward and backward
// kernels: memory spaces (global or shared), texel decoding, the packed
// per-halfedge record, level selection and the border-aware bilinear taps.
#pragma once

#include <cstdint>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "htex_internal.h"

namespace htex {

// ------------------------------------------------------------ memory spaces

// Read-only global memory: texels and records through the non-coherent
// (read-only) cache path.
struct GlobalSpace {
    using off_t = uint64_t;
    const uint8_t* base;
    __device__ __forceinline__ uint4 ld16(off_t o) const { return __ldg(reinterpret_cast<const uint4*>(base + o)); }
    __device__ __forceinline__ uint2 ld8(off_t o) const { return __ldg(reinterpret_cast<const uint2*>(base + o)); }
    __device__ __forceinline__ uint32_t ld4(off_t o) const { return __ldg(reinterpret_cast<const unsigned int*>(base + o)); }
    __device__ __forceinline__ uint32_t ld2(off_t o) const { return __ldg(reinterpret_cast<const unsigned short*>(base + o)); }
    __device__ __forceinline__ uint32_t ld1(off_t o) const { return __ldg(reinterpret_cast<const unsigned char*>(base + o)); }
};

// Shared memory addressed by 32-bit shared-window addresses.
struct SharedSpace {
    using off_t = uint32_t;
    uint32_t base;
    __device__ __forceinline__ uint4 ld16(off_t o) const {
        uint4 r;
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "r"(base + o));
        return r;
    }
    __device__ __forceinline__ uint2 ld8(off_t o) const {
        uint2 r;
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "r"(base + o));
        return r;
    }
    __device__ __forceinline__ uint32_t ld4(off_t o) const {
        uint32_t r;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(r) : "r"(base + o));
        return r;
    }
    __device__ __forceinline__ uint32_t ld2(off_t o) const {
        unsigned short r;
        asm volatile("ld.shared.u16 %0, [%1];" : "=h"(r) : "r"(base + o));
        return r;
    }
    __device__ __forceinline__ uint32_t ld1(off_t o) const {
        unsigned short r;
        asm volatile("ld.shared.u8 %0, [%1];" : "=h"(r) : "r"(base + o));
        return r & 0xffu;
    }
};

// ---------------------------------------------------------------- decoding

template <int DT> struct Fmt;
template <> struct Fmt<HTEX_F32> { static constexpr int ES = 4; static constexpr bool SCALED = false; };
template <> struct Fmt<HTEX_U8> { static constexpr int ES = 1; static constexpr bool SCALED = false; };
template <> struct Fmt<HTEX_F16> { static constexpr int ES = 2; static constexpr bool SCALED = true; };
template <> struct Fmt<HTEX_BF16> { static constexpr int ES = 2; static constexpr bool SCALED = true; };
template <> struct Fmt<HTEX_E4M3> { static constexpr int ES = 1; static constexpr bool SCALED = true; };

__device__ __forceinline__ float dec_u8(uint32_t b) { return float(b) * (1.0f / 255.0f); }
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
                for (int c = 0; c < 4; ++c) t[c] = dec1<DT>((r >> (8 * c)) & 0xffu);
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

struct TexRef {
    uint64_t off;   // byte offset of the texture in the pool
    int n;          // log2 of the resolution
    float scale;    // code scale (1 for unscaled formats)
};

template <int DT, class S>
__device__ __forceinline__ TexRef tex_ref(const Asset<S>& A, uint32_t e) {
    TexRef t;
    if (A.uniform_log2n >= 0) {
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

// Byte offset of level l inside a chain of base 2^n with 'tb' bytes per texel.
__device__ __forceinline__ uint64_t level_bytes(int n, int l, int tb) {
    const uint64_t t = ((uint64_t(1) << (2 * n + 2)) - (uint64_t(1) << (2 * (n - l) + 2))) / 3u;
    return t * uint64_t(tb);
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

// Bilinear taps of one level with a zero border: texel centres at
// (i + 1/2) / N; the 1-D weights of out-of-range taps are zero, so
// (wx0 + wx1) (wy0 + wy1) is this level's share of the normalisation sum.
struct Taps {
    int N;
    int i0, i1, j0, j1;     // clamped texel indices
    float wx0, wx1, wy0, wy1;
};

__device__ __forceinline__ bool taps(float x, float y, int N, Taps& t) {
    const float fN = float(N);
    const float s = fmaf(x, fN, -0.5f), r = fmaf(y, fN, -0.5f);
    const float fi = floorf(s), fj = floorf(r);
    const float a = s - fi, b = r - fj;
    const int i = int(fi), j = int(fj);
    t.N = N;
    t.wx0 = (unsigned(i) < unsigned(N)) ? 1.0f - a : 0.0f;
    t.wx1 = (unsigned(i + 1) < unsigned(N)) ? a : 0.0f;
    t.wy0 = (unsigned(j) < unsigned(N)) ? 1.0f - b : 0.0f;
    t.wy1 = (unsigned(j + 1) < unsigned(N)) ? b : 0.0f;
    t.i0 = max(i, 0);
    t.i1 = min(i + 1, N - 1);
    t.j0 = max(j, 0);
    t.j1 = min(j + 1, N - 1);
    return (t.wx0 + t.wx1) * (t.wy0 + t.wy1) != 0.0f;
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

__device__ __forceinline__ int4 ld_query(const htex_query* q, int64_t i) {
    int4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(reinterpret_cast<const int4*>(q) + i));
    return r;
}

}  // namespace htex
