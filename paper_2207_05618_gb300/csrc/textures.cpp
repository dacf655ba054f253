// Texture storage: pool layout, host-side preparation (mips, boundary
// mirroring, corner pre-processing, reduced-precision codes) and device
// residency.  Paper Section 4.3 (one square texture per edge, boundary
// mirroring) and Section 4.4 (corner pre-processing); mip generation and
// reduced-precision storage fill in what the paper leaves to the graphics
// API.  Compiled without FMA contraction so prepared pools are identical on
// every host architecture.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "htex_internal.h"

int htex_elem_size(htex_dtype d) {
    switch (d) {
    case HTEX_F32: return 4;
    case HTEX_U8: return 1;
    case HTEX_F16: return 2;
    case HTEX_BF16: return 2;
    case HTEX_E4M3: return 1;
    }
    return 0;
}

bool htex_dtype_valid(int32_t d) { return d >= HTEX_F32 && d <= HTEX_E4M3; }

int64_t htex_pool_offsets(int32_t E, const int32_t* log2n, int32_t C, htex_dtype dt,
                          int64_t* offsets) {
    const int64_t es = htex_elem_size(dt);
    int64_t at = 0;
    for (int32_t e = 0; e < E; ++e) {
        if (offsets) offsets[e] = at;
        const int64_t bytes = htex_chain_texels(log2n[e]) * C * es;
        at += (bytes + 15) & ~int64_t(15);
    }
    if (offsets) offsets[E] = at;
    return at;
}

namespace {

bool is_scaled(htex_dtype d) { return d == HTEX_F16 || d == HTEX_BF16 || d == HTEX_E4M3; }

// Round a double to a binary format with 'ebits' exponent and 'mbits'
// fraction bits, to nearest with ties to even, by integer manipulation of
// the double's significand.  'fn' selects the E4M3 variant without
// infinities that saturates at its largest finite value; otherwise
// overflow gives infinity.  Returns the code.
uint32_t encode_code(double x, int ebits, int mbits, bool fn) {
    uint64_t bits;
    std::memcpy(&bits, &x, 8);
    const uint32_t sign = uint32_t(bits >> 63) << (ebits + mbits);
    const int dexp = int((bits >> 52) & 0x7ff);
    const uint64_t dman = bits & ((uint64_t(1) << 52) - 1);
    const int bias = (1 << (ebits - 1)) - 1;
    const int emin = 1 - bias;
    if (dexp == 0) return sign;  // zero, or a double subnormal far below every code
    int e = dexp - 1023;
    const uint64_t sig = dman | (uint64_t(1) << 52);
    int te = e < emin ? emin : e;
    const int drop = 52 - mbits + (te - e);
    uint64_t q = 0;
    if (drop < 64) {
        q = sig >> drop;
        const uint64_t rem = sig & ((uint64_t(1) << drop) - 1);
        const uint64_t half = uint64_t(1) << (drop - 1);
        if (rem > half || (rem == half && (q & 1))) ++q;
    }
    if (q >= (uint64_t(2) << mbits)) {  // rounded up into the next binade
        q >>= 1;
        ++te;
    }
    uint32_t E, M;
    if (q < (uint64_t(1) << mbits)) {
        E = 0;
        M = uint32_t(q);
    } else {
        E = uint32_t(te + bias);
        M = uint32_t(q - (uint64_t(1) << mbits));
    }
    const uint32_t emax_field = (1u << ebits) - 1;
    if (fn) {
        // E4M3: the all-ones pattern is NaN; largest finite is E=15, M=6 (448)
        if (E > emax_field || (E == emax_field && M == (1u << mbits) - 1)) {
            E = emax_field;
            M = (1u << mbits) - 2;
        }
    } else if (E >= emax_field) {
        E = emax_field;
        M = 0;
    }
    return sign | (E << mbits) | M;
}

// Texture element views over a contiguous work buffer in pool element order.
template <class T>
struct Work {
    T* base;
    const int64_t* eoff;  // element offset of each texture
    int32_t C;
    T* level(int32_t e, int n, int l) const { return base + eoff[e] + htex_level_texels(n, l) * C; }
};

template <class T>
void mirror_level(T* L, int N, int C) {
    for (int j = 0; j < N; ++j)
        for (int i = N - j; i < N; ++i)  // i + j > N - 1
            for (int c = 0; c < C; ++c) L[(int64_t(j) * N + i) * C + c] = L[(int64_t(N - 1 - i) * N + (N - 1 - j)) * C + c];
}

void mip_down(const float* src, float* dst, int Nd, int C) {
    const int Ns = 2 * Nd;
    for (int j = 0; j < Nd; ++j)
        for (int i = 0; i < Nd; ++i)
            for (int c = 0; c < C; ++c) {
                const double a = src[(int64_t(2 * j) * Ns + 2 * i) * C + c];
                const double b = src[(int64_t(2 * j) * Ns + 2 * i + 1) * C + c];
                const double d0 = src[(int64_t(2 * j + 1) * Ns + 2 * i) * C + c];
                const double d1 = src[(int64_t(2 * j + 1) * Ns + 2 * i + 1) * C + c];
                dst[(int64_t(j) * Nd + i) * C + c] = float((((a + b) + d0) + d1) * 0.25);
            }
}

void mip_down(const uint8_t* src, uint8_t* dst, int Nd, int C) {
    const int Ns = 2 * Nd;
    for (int j = 0; j < Nd; ++j)
        for (int i = 0; i < Nd; ++i)
            for (int c = 0; c < C; ++c) {
                const unsigned s = src[(int64_t(2 * j) * Ns + 2 * i) * C + c] +
                                   src[(int64_t(2 * j) * Ns + 2 * i + 1) * C + c] +
                                   src[(int64_t(2 * j + 1) * Ns + 2 * i) * C + c] +
                                   src[(int64_t(2 * j + 1) * Ns + 2 * i + 1) * C + c];
                dst[(int64_t(j) * Nd + i) * C + c] = uint8_t((s + 2) >> 2);
            }
}

inline float group_mean(double s, int64_t cnt, float*) { return float(s / double(cnt)); }
inline uint8_t group_mean(double s, int64_t cnt, uint8_t*) {
    const int64_t si = int64_t(s);  // exact: a sum of bytes
    return uint8_t((2 * si + cnt) / (2 * cnt));
}

struct UnionFind {
    std::vector<int32_t> p;
    explicit UnionFind(int32_t n) : p(size_t(n)) {
        for (int32_t i = 0; i < n; ++i) p[i] = i;
    }
    int32_t root(int32_t x) {
        while (p[x] != x) x = p[x] = p[p[x]];
        return x;
    }
    void join(int32_t a, int32_t b) {
        a = root(a);
        b = root(b);
        if (a != b) p[a] = b;
    }
};

// Corner pre-processing (Section 4.4).  For every resolution R, each
// texture with a level of size R contributes its corner texels, each tied
// to the surface point it sits on (mesh vertex or face centroid); texels
// meeting at one point take the group mean, groups joined through texels
// that are several corners at once (R = 1).
template <class T>
void fix_corners(const htex_mesh& m, const int32_t* log2n, const std::vector<int32_t>& owner,
                 const Work<T>& w, bool mirrored) {
    int maxn = 0;
    for (int32_t e = 0; e < m.E; ++e) maxn = log2n[e] > maxn ? log2n[e] : maxn;
    const int32_t P = m.V + m.F;
    const int C = w.C;
    struct Slot {
        T* texel;
        int32_t point;
    };
    std::vector<Slot> slots;
    std::vector<double> sum;
    std::vector<int64_t> cnt;
    for (int r = 0; r <= maxn; ++r) {
        const int64_t R = int64_t(1) << r;
        slots.clear();
        for (int32_t e = 0; e < m.E; ++e) {
            const int n = log2n[e];
            if (n < r) continue;
            const int32_t h = owner[e];
            T* L = w.level(e, n, n - r);
            slots.push_back({L + (R - 1) * C, m.vert[h]});                      // (R-1, 0)
            slots.push_back({L + (R - 1) * R * C, m.vert[m.next[h]]});          // (0, R-1)
            slots.push_back({L, m.V + m.face[h]});                              // (0, 0)
            if (m.twin[h] >= 0)
                slots.push_back({L + ((R - 1) * R + R - 1) * C, m.V + m.face[m.twin[h]]});
            else if (mirrored)
                slots.push_back({L + ((R - 1) * R + R - 1) * C, m.V + m.face[h]});
            else
                slots.push_back({nullptr, -1});
        }
        UnionFind uf(P);
        if (r == 0)
            for (size_t k = 0; k < slots.size(); k += 4)
                for (size_t a = 1; a < 4; ++a)
                    if (slots[k + a].texel) uf.join(slots[k].point, slots[k + a].point);
        sum.assign(size_t(P) * C, 0.0);
        cnt.assign(size_t(P), 0);
        auto first_in_texture = [&](size_t k) {
            const size_t base = k - k % 4;
            for (size_t b = base; b < k; ++b)
                if (slots[b].texel == slots[k].texel) return false;
            return true;
        };
        for (size_t k = 0; k < slots.size(); ++k) {
            if (!slots[k].texel || !first_in_texture(k)) continue;
            const int32_t g = uf.root(slots[k].point);
            ++cnt[g];
            for (int c = 0; c < C; ++c) sum[size_t(g) * C + c] += double(slots[k].texel[c]);
        }
        for (size_t k = 0; k < slots.size(); ++k) {
            if (!slots[k].texel || !first_in_texture(k)) continue;
            const int32_t g = uf.root(slots[k].point);
            for (int c = 0; c < C; ++c)
                slots[k].texel[c] = group_mean(sum[size_t(g) * C + c], cnt[g], (T*)nullptr);
        }
    }
}

template <class T>
void prepare_work(const htex_mesh& m, const int32_t* log2n, const Work<T>& w, uint32_t flags) {
    std::vector<int32_t> owner(size_t(m.E), -1);
    for (int32_t h = 0; h < m.H; ++h)
        if (m.twin[h] < h) owner[m.edge[h]] = h;
    const bool mirror = flags & HTEX_MIRROR_BOUNDARY;
    const bool given = flags & HTEX_LEVELS_GIVEN;
    if (!given) {
        if (mirror)
            for (int32_t e = 0; e < m.E; ++e)
                if (m.twin[owner[e]] < 0) mirror_level(w.level(e, log2n[e], 0), 1 << log2n[e], w.C);
        for (int32_t e = 0; e < m.E; ++e)
            for (int l = 0; l < log2n[e]; ++l)
                mip_down(w.level(e, log2n[e], l), w.level(e, log2n[e], l + 1), 1 << (log2n[e] - l - 1), w.C);
    }
    if (mirror)
        for (int32_t e = 0; e < m.E; ++e)
            if (m.twin[owner[e]] < 0)
                for (int l = 0; l <= log2n[e]; ++l) mirror_level(w.level(e, log2n[e], l), 1 << (log2n[e] - l), w.C);
    if (flags & HTEX_FIX_CORNERS) fix_corners(m, log2n, owner, w, mirror);
}

htex_status check_texture_args(const htex_mesh* m, int32_t C, int32_t dt, const int32_t* log2n,
                               const void* texels, uint32_t flags) {
    if (!m || !log2n || !texels) return HTEX_ERR_INVALID_ARG;
    if (C < 1 || C > 4 || !htex_dtype_valid(dt)) return HTEX_ERR_INVALID_ARG;
    if (flags & ~uint32_t(HTEX_BUILD_MIPS | HTEX_MIRROR_BOUNDARY | HTEX_FIX_CORNERS | HTEX_LEVELS_GIVEN))
        return HTEX_ERR_INVALID_ARG;
    if (!(flags & HTEX_LEVELS_GIVEN) && !(flags & HTEX_BUILD_MIPS)) return HTEX_ERR_INVALID_ARG;
    for (int32_t e = 0; e < m->E; ++e)
        if (log2n[e] < 0 || log2n[e] > kMaxLog2Res) return HTEX_ERR_BAD_TEXTURE;
    return HTEX_OK;
}

template <class T>
void fill_work(const htex_mesh& m, const int32_t* log2n, const T* src, const Work<T>& w, bool given) {
    int64_t at = 0;
    for (int32_t e = 0; e < m.E; ++e) {
        const int n = log2n[e];
        const int64_t cnt = (given ? htex_chain_texels(n) : (int64_t(1) << (2 * n))) * w.C;
        std::memcpy(w.base + w.eoff[e], src + at, size_t(cnt) * sizeof(T));
        at += cnt;
    }
}

}  // namespace

extern "C" htex_status htex_textures_layout(const htex_mesh* m, int32_t channels, htex_dtype dtype,
                                            const int32_t* log2_res, int64_t* pool_bytes,
                                            int64_t* texture_offsets) {
    if (!m || !log2_res || !pool_bytes || channels < 1 || channels > 4 || !htex_dtype_valid(dtype))
        return HTEX_ERR_INVALID_ARG;
    for (int32_t e = 0; e < m->E; ++e)
        if (log2_res[e] < 0 || log2_res[e] > kMaxLog2Res) return HTEX_ERR_BAD_TEXTURE;
    *pool_bytes = htex_pool_offsets(m->E, log2_res, channels, dtype, texture_offsets);
    return HTEX_OK;
}

extern "C" htex_status htex_textures_prepare(const htex_mesh* m, int32_t channels, htex_dtype dtype,
                                             const int32_t* log2_res, const void* texels,
                                             uint32_t flags, void* pool_out, float* scales_out) {
    htex_status st = check_texture_args(m, channels, dtype, log2_res, texels, flags);
    if (st != HTEX_OK) return st;
    if (!pool_out) return HTEX_ERR_INVALID_ARG;
    const int32_t E = m->E, C = channels;
    const bool given = flags & HTEX_LEVELS_GIVEN;
    try {
        std::vector<int64_t> boff(size_t(E) + 1);
        const int64_t pool_bytes = htex_pool_offsets(E, log2_res, C, dtype, boff.data());
        const int es = htex_elem_size(dtype);
        std::vector<int64_t> eoff(size_t(E) + 1);
        for (int32_t e = 0; e <= E; ++e) eoff[e] = boff[e] / es;
        std::memset(pool_out, 0, size_t(pool_bytes));
        if (dtype == HTEX_U8) {
            Work<uint8_t> w{static_cast<uint8_t*>(pool_out), eoff.data(), C};
            fill_work(*m, log2_res, static_cast<const uint8_t*>(texels), w, given);
            prepare_work(*m, log2_res, w, flags);
            if (scales_out)
                for (int32_t e = 0; e < E; ++e) scales_out[e] = 1.0f;
            return HTEX_OK;
        }
        if (dtype == HTEX_F32) {
            Work<float> w{static_cast<float*>(pool_out), eoff.data(), C};
            fill_work(*m, log2_res, static_cast<const float*>(texels), w, given);
            prepare_work(*m, log2_res, w, flags);
            if (scales_out)
                for (int32_t e = 0; e < E; ++e) scales_out[e] = 1.0f;
            return HTEX_OK;
        }
        // scaled formats: prepare in float with float element offsets, then encode
        std::vector<int64_t> foff(size_t(E) + 1);
        {
            int64_t at = 0;
            for (int32_t e = 0; e < E; ++e) {
                foff[e] = at;
                at += htex_chain_texels(log2_res[e]) * C;
            }
            foff[E] = at;
        }
        std::vector<float> work(size_t(foff[E]));
        Work<float> w{work.data(), foff.data(), C};
        fill_work(*m, log2_res, static_cast<const float*>(texels), w, given);
        prepare_work(*m, log2_res, w, flags);
        uint8_t* pool = static_cast<uint8_t*>(pool_out);
        for (int32_t e = 0; e < E; ++e) {
            const float* src = work.data() + foff[e];
            const int64_t cnt = foff[e + 1] - foff[e];
            double mx = 0.0;
            for (int64_t k = 0; k < cnt; ++k) mx = std::fabs(double(src[k])) > mx ? std::fabs(double(src[k])) : mx;
            double s;
            if (mx == 0.0) s = 1.0;
            else if (dtype == HTEX_E4M3) s = double(float(mx / 448.0));
            else s = double(float(mx));
            if (scales_out) scales_out[e] = float(s);
            uint8_t* dst = pool + boff[e];
            for (int64_t k = 0; k < cnt; ++k) {
                const double x = double(src[k]) / s;
                if (dtype == HTEX_E4M3) {
                    dst[k] = uint8_t(encode_code(x, 4, 3, true));
                } else {
                    const uint16_t code = uint16_t(dtype == HTEX_F16 ? encode_code(x, 5, 10, false)
                                                                     : encode_code(x, 8, 7, false));
                    std::memcpy(dst + 2 * k, &code, 2);
                }
            }
        }
    } catch (const std::bad_alloc&) {
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    return HTEX_OK;
}

namespace {

htex_status cuda_fail(htex_textures* t) {
    if (t) {
        cudaFree(t->d_rec);
        cudaFree(t->d_hdr);
        cudaFree(t->d_scale);
        cudaFree(t->d_pool);
        delete t;
    }
    cudaGetLastError();
    return HTEX_ERR_CUDA;
}

}  // namespace

htex_status htex_asset_arrays(const htex_mesh* m, int32_t C, htex_dtype dtype, const int32_t* log2n,
                              const float* scales, HtexAssetArrays* out) {
    HtexAssetArrays& A = *out;
    const int32_t H = m->H, E = m->E;
    std::vector<int64_t> boff(size_t(E) + 1);
    A.pool_bytes = htex_pool_offsets(E, log2n, C, dtype, boff.data());
    if (boff[E] / 16 >= (int64_t(1) << 32)) return HTEX_ERR_UNSUPPORTED;  // header offsets are 32-bit x 16 B
    A.H = H;
    A.E = E;
    A.C = C;
    A.dtype = dtype;
    // per-halfedge lookup records: the edge and Alg. 2 reflection of h, Next(h), Prev(h)
    A.rec.assign(size_t(H) * 4, 0);
    auto code = [&](int32_t g) { return uint32_t(m->edge[g]) | (g < m->twin[g] ? kFlipBit : 0u); };
    for (int32_t h = 0; h < H; ++h) {
        A.rec[4 * size_t(h) + 0] = int32_t(code(h));
        A.rec[4 * size_t(h) + 1] = int32_t(code(m->next[h]));
        A.rec[4 * size_t(h) + 2] = int32_t(code(m->prev[h]));
        A.rec[4 * size_t(h) + 3] = m->face[h];
    }
    A.hdr.assign(size_t(E) * 4, 0);
    A.scale.assign((size_t(E) + 3) & ~size_t(3), 1.0f);   // whole 16-byte words (shared-memory staging)
    int32_t uniform = E > 0 ? log2n[0] : 0, maxn = 0;
    for (int32_t e = 0; e < E; ++e) {
        if (scales) A.scale[e] = scales[e];
        const float sv = A.scale[e];
        A.hdr[4 * size_t(e) + 0] = int32_t(uint32_t(boff[e] / 16));
        A.hdr[4 * size_t(e) + 1] = log2n[e];
        std::memcpy(&A.hdr[4 * size_t(e) + 2], &sv, 4);
        if (log2n[e] != uniform) uniform = -1;
        maxn = log2n[e] > maxn ? log2n[e] : maxn;
    }
    A.uniform_log2n = uniform;
    A.max_log2n = maxn;
    A.uniform_stride = (uniform >= 0 && E > 0) ? boff[1] - boff[0] : 0;
    return HTEX_OK;
}

int64_t htex_asset_device_bytes(const HtexAssetArrays& a) {
    return int64_t(a.rec.size() + a.hdr.size() + a.scale.size()) * 4 + a.pool_bytes;
}

htex_status htex_asset_allocate(const HtexAssetArrays& a, htex_textures** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_fail(nullptr);
    htex_textures* t = new (std::nothrow) htex_textures;
    if (!t) return HTEX_ERR_OUT_OF_MEMORY;
    t->H = a.H;
    t->E = a.E;
    t->C = a.C;
    t->dtype = a.dtype;
    t->uniform_log2n = a.uniform_log2n;
    t->uniform_stride = a.uniform_stride;
    t->pool_bytes = a.pool_bytes;
    t->max_log2n = a.max_log2n;
    t->has_scales = is_scaled(a.dtype);
    t->device = dev;
    cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t rec_b = a.rec.size() * 4, hdr_b = a.hdr.size() * 4, sc_b = a.scale.size() * 4;
    if (cudaMalloc(&t->d_rec, rec_b ? rec_b : 16) != cudaSuccess ||
        cudaMalloc(&t->d_hdr, hdr_b ? hdr_b : 16) != cudaSuccess ||
        cudaMalloc(&t->d_scale, sc_b ? sc_b : 16) != cudaSuccess ||
        cudaMalloc(&t->d_pool, size_t(a.pool_bytes > 0 ? a.pool_bytes : 16)) != cudaSuccess) {
        cuda_fail(t);
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    t->device_bytes = htex_asset_device_bytes(a);
    *out = t;
    return HTEX_OK;
}

htex_status htex_asset_allocate_async(const HtexAssetArrays& a, cudaMemPool_t pool, cudaStream_t stream,
                                      htex_textures** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cuda_fail(nullptr);
    htex_textures* t = new (std::nothrow) htex_textures;
    if (!t) return HTEX_ERR_OUT_OF_MEMORY;
    t->H = a.H;
    t->E = a.E;
    t->C = a.C;
    t->dtype = a.dtype;
    t->uniform_log2n = a.uniform_log2n;
    t->uniform_stride = a.uniform_stride;
    t->pool_bytes = a.pool_bytes;
    t->max_log2n = a.max_log2n;
    t->has_scales = is_scaled(a.dtype);
    t->device = dev;
    t->free_stream = stream;
    cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t rec_b = a.rec.size() * 4, hdr_b = a.hdr.size() * 4, sc_b = a.scale.size() * 4;
    void** bufs[4] = {&t->d_rec, &t->d_hdr, &t->d_scale, &t->d_pool};
    const size_t sizes[4] = {rec_b ? rec_b : 16, hdr_b ? hdr_b : 16, sc_b ? sc_b : 16,
                             size_t(a.pool_bytes > 0 ? a.pool_bytes : 16)};
    for (int k = 0; k < 4; ++k) {
        if (cudaMallocFromPoolAsync(bufs[k], sizes[k], pool, stream) != cudaSuccess) {
            cudaGetLastError();
            htex_textures_destroy(t);
            return HTEX_ERR_OUT_OF_MEMORY;
        }
    }
    t->device_bytes = htex_asset_device_bytes(a);
    *out = t;
    return HTEX_OK;
}

htex_status htex_asset_copy_async(const HtexAssetArrays& a, const void* pool, htex_textures* t, cudaStream_t stream) {
    const size_t rec_b = a.rec.size() * 4, hdr_b = a.hdr.size() * 4, sc_b = a.scale.size() * 4;
    if ((rec_b && cudaMemcpyAsync(t->d_rec, a.rec.data(), rec_b, cudaMemcpyHostToDevice, stream) != cudaSuccess) ||
        (hdr_b && cudaMemcpyAsync(t->d_hdr, a.hdr.data(), hdr_b, cudaMemcpyHostToDevice, stream) != cudaSuccess) ||
        (sc_b && cudaMemcpyAsync(t->d_scale, a.scale.data(), sc_b, cudaMemcpyHostToDevice, stream) != cudaSuccess) ||
        (a.pool_bytes && cudaMemcpyAsync(t->d_pool, pool, size_t(a.pool_bytes), cudaMemcpyHostToDevice, stream) != cudaSuccess)) {
        cudaGetLastError();
        return HTEX_ERR_CUDA;
    }
    return HTEX_OK;
}

namespace {

htex_status upload_prepared(const htex_mesh* m, int32_t C, htex_dtype dtype, const int32_t* log2n,
                            const void* pool, const float* scales, cudaStream_t stream,
                            htex_textures** out) {
    HtexAssetArrays a;
    htex_status st = htex_asset_arrays(m, C, dtype, log2n, scales, &a);
    if (st != HTEX_OK) return st;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return cuda_fail(nullptr);
    if (htex_asset_device_bytes(a) + (int64_t(64) << 20) > int64_t(free_b)) return HTEX_ERR_OUT_OF_MEMORY;
    htex_textures* t = nullptr;
    st = htex_asset_allocate(a, &t);
    if (st != HTEX_OK) return st;
    if (htex_asset_copy_async(a, pool, t, stream) != HTEX_OK || cudaStreamSynchronize(stream) != cudaSuccess)
        return cuda_fail(t);
    *out = t;
    return HTEX_OK;
}

htex_status upload_from_texels(const htex_mesh* m, int32_t C, htex_dtype dtype, const int32_t* log2n,
                               const void* texels, uint32_t flags, htex_stream stream,
                               htex_textures** out) {
    if (!out) return HTEX_ERR_INVALID_ARG;
    *out = nullptr;
    htex_status st = check_texture_args(m, C, dtype, log2n, texels, flags);
    if (st != HTEX_OK) return st;
    try {
        const int64_t bytes = htex_pool_offsets(m->E, log2n, C, dtype, nullptr);
        std::vector<uint8_t> pool(size_t(bytes > 0 ? bytes : 1));
        std::vector<float> scales(size_t(m->E) + 1);
        st = htex_textures_prepare(m, C, dtype, log2n, texels, flags, pool.data(), scales.data());
        if (st != HTEX_OK) return st;
        return upload_prepared(m, C, dtype, log2n, pool.data(), scales.data(),
                               reinterpret_cast<cudaStream_t>(stream), out);
    } catch (const std::bad_alloc&) {
        return HTEX_ERR_OUT_OF_MEMORY;
    }
}

}  // namespace

extern "C" htex_status htex_textures_upload(const htex_mesh* m, int32_t channels, htex_dtype dtype,
                                            const int32_t* log2_res, const void* texels,
                                            uint32_t flags, htex_stream stream, htex_textures** out) {
    return upload_from_texels(m, channels, dtype, log2_res, texels, flags, stream, out);
}

extern "C" htex_status htex_textures_upload_levels(const htex_mesh* m, int32_t channels,
                                                   htex_dtype dtype, const int32_t* log2_res,
                                                   const void* texels, uint32_t flags,
                                                   htex_stream stream, htex_textures** out) {
    return upload_from_texels(m, channels, dtype, log2_res, texels,
                              (flags & ~uint32_t(HTEX_BUILD_MIPS)) | HTEX_LEVELS_GIVEN, stream, out);
}

extern "C" htex_status htex_textures_upload_pool(const htex_mesh* m, int32_t channels,
                                                 htex_dtype dtype, const int32_t* log2_res,
                                                 const void* pool, const float* scales,
                                                 htex_stream stream, htex_textures** out) {
    if (!out) return HTEX_ERR_INVALID_ARG;
    *out = nullptr;
    if (!m || !log2_res || !pool || channels < 1 || channels > 4 || !htex_dtype_valid(dtype))
        return HTEX_ERR_INVALID_ARG;
    if (is_scaled(dtype) && !scales) return HTEX_ERR_INVALID_ARG;
    for (int32_t e = 0; e < m->E; ++e)
        if (log2_res[e] < 0 || log2_res[e] > kMaxLog2Res) return HTEX_ERR_BAD_TEXTURE;
    try {
        return upload_prepared(m, channels, dtype, log2_res, pool, scales,
                               reinterpret_cast<cudaStream_t>(stream), out);
    } catch (const std::bad_alloc&) {
        return HTEX_ERR_OUT_OF_MEMORY;
    }
}

extern "C" htex_status htex_textures_info(const htex_textures* t, int32_t* channels,
                                          htex_dtype* dtype, int32_t* H, int32_t* E,
                                          int64_t* pool_bytes, int64_t* device_bytes) {
    if (!t) return HTEX_ERR_INVALID_ARG;
    if (channels) *channels = t->C;
    if (dtype) *dtype = t->dtype;
    if (H) *H = t->H;
    if (E) *E = t->E;
    if (pool_bytes) *pool_bytes = t->pool_bytes;
    if (device_bytes) *device_bytes = t->device_bytes;
    return HTEX_OK;
}

extern "C" htex_status htex_textures_download_pool(const htex_textures* t, void* pool, float* scales,
                                                   htex_stream stream) {
    if (!t || !pool) return HTEX_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (t->pool_bytes && cudaMemcpyAsync(pool, t->d_pool, size_t(t->pool_bytes), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return HTEX_ERR_CUDA;
    if (scales && t->E && cudaMemcpyAsync(scales, t->d_scale, sizeof(float) * size_t(t->E), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return HTEX_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return HTEX_ERR_CUDA;
    return HTEX_OK;
}

extern "C" htex_status htex_textures_write_pool(const htex_textures* t, int64_t offset, int64_t bytes,
                                                const void* src, htex_stream stream) {
    if (!t || offset < 0 || bytes < 0 || offset > t->pool_bytes || bytes > t->pool_bytes - offset)
        return HTEX_ERR_INVALID_ARG;
    if (bytes == 0) return HTEX_OK;
    if (!src) return HTEX_ERR_INVALID_ARG;
    if (cudaMemcpyAsync(static_cast<uint8_t*>(t->d_pool) + offset, src, size_t(bytes), cudaMemcpyDefault,
                        reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return HTEX_ERR_CUDA;
    }
    return HTEX_OK;
}

extern "C" void htex_textures_destroy(htex_textures* t) {
    if (!t) return;
    htex_host_path_destroy(t->host_path);
    void* bufs[4] = {t->d_rec, t->d_hdr, t->d_scale, t->d_pool};
    for (void* b : bufs) {
        if (!b) continue;
        if (t->free_stream) cudaFreeAsync(b, t->free_stream);
        else cudaFree(b);
    }
    delete t;
}
