// The rendering side of Htex (paper Sections 3.1, 4.4, 5.1) as CUDA
// kernels: Alg. 1 (the intrinsic triangle of each halfedge), rendering
// the intrinsic triangulation into a per-pixel query buffer (halfedge,
// perspective-correct barycentrics, footprint), and displacement of a
// tessellated lattice along the input mesh's normals.
//
// Rasterisation: one thread per intrinsic triangle covers the pixel
// centres inside it (barycentrics >= 0, depth z/w in [-1, 1]) and keeps,
// per pixel, the smallest 64-bit key (ordered depth << 32 | halfedge) with
// atomicMin, so ties go to the smaller halfedge id.  A resolve pass turns
// each pixel's key into a query: barycentrics at the pixel centre
// corrected for perspective, and the footprint max(|d(u,v)/dx|,
// |d(u,v)/dy|) from the same triangle's barycentrics one pixel right and
// one pixel down.  Triangles with a vertex behind the camera (w <= 0) are
// not drawn.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <type_traits>

#include <cuda_runtime.h>

#include "htex_internal.h"

struct htex_geometry {
    int32_t H = 0, V = 0, F = 0;
    int32_t* d_next = nullptr;
    int32_t* d_vert = nullptr;
    int32_t* d_face = nullptr;
    float* d_pos = nullptr;      // [V][3]
    float* d_vn = nullptr;       // [V][3] vertex normals
    float* d_fn = nullptr;       // [F][3] face normals
};

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float3 ld3(const float* p, int32_t i) {
    return make_float3(p[3 * i], p[3 * i + 1], p[3 * i + 2]);
}

// Alg. 1: v0 = Vert(Next h), v1 = the mean of the face's vertices walking
// the Next cycle from h, v2 = Vert(h).
__device__ __forceinline__ void alg1(const htex_geometry g, int32_t h, float3& v0, float3& v1, float3& v2) {
    const int32_t nx = g.d_next[h];
    v2 = ld3(g.d_pos, g.d_vert[h]);
    v0 = ld3(g.d_pos, g.d_vert[nx]);
    float3 c = v2;
    int n = 1;
    for (int32_t k = nx; k != h && n <= g.H; k = g.d_next[k]) {
        const float3 p = ld3(g.d_pos, g.d_vert[k]);
        c.x += p.x;
        c.y += p.y;
        c.z += p.z;
        ++n;
    }
    const float inv = 1.0f / float(n);
    v1 = make_float3(c.x * inv, c.y * inv, c.z * inv);
}

__global__ void k_triangles(htex_geometry g, float* out) {
    for (int32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < g.H; h += gridDim.x * blockDim.x) {
        float3 v0, v1, v2;
        alg1(g, h, v0, v1, v2);
        float* o = out + 9 * int64_t(h);
        o[0] = v0.x; o[1] = v0.y; o[2] = v0.z;
        o[3] = v1.x; o[4] = v1.y; o[5] = v1.z;
        o[6] = v2.x; o[7] = v2.y; o[8] = v2.z;
    }
}

struct Camera {
    float m[16];   // row-major view-projection: clip = m * [p, 1]
    int32_t W, Ht;
};

struct Screen {
    float x[3], y[3], z[3], w[3];   // screen position, NDC depth and clip w of v0, v1, v2
    float den;
};

__device__ __forceinline__ bool project(const Camera& cam, const float3 (&v)[3], Screen& s) {
    for (int k = 0; k < 3; ++k) {
        const float* m = cam.m;
        const float cx = m[0] * v[k].x + m[1] * v[k].y + m[2] * v[k].z + m[3];
        const float cy = m[4] * v[k].x + m[5] * v[k].y + m[6] * v[k].z + m[7];
        const float cz = m[8] * v[k].x + m[9] * v[k].y + m[10] * v[k].z + m[11];
        const float cw = m[12] * v[k].x + m[13] * v[k].y + m[14] * v[k].z + m[15];
        if (!(cw > 0.0f)) return false;
        s.w[k] = cw;
        s.x[k] = (cx / cw * 0.5f + 0.5f) * float(cam.W);
        s.y[k] = (0.5f - cy / cw * 0.5f) * float(cam.Ht);
        s.z[k] = cz / cw;
    }
    s.den = (s.y[1] - s.y[2]) * (s.x[0] - s.x[2]) + (s.x[2] - s.x[1]) * (s.y[0] - s.y[2]);
    return s.den != 0.0f;
}

// Screen-space barycentrics of (px, py) with respect to (v0, v1, v2).
__device__ __forceinline__ void screen_bary(const Screen& s, float px, float py, float& l0, float& l1, float& l2) {
    l0 = ((s.y[1] - s.y[2]) * (px - s.x[2]) + (s.x[2] - s.x[1]) * (py - s.y[2])) / s.den;
    l1 = ((s.y[2] - s.y[0]) * (px - s.x[2]) + (s.x[0] - s.x[2]) * (py - s.y[2])) / s.den;
    l2 = 1.0f - l0 - l1;
}

// Perspective-correct (u, v): u weighs v2 = Vert(h), v weighs v0 = Vert(Next h).
__device__ __forceinline__ void uv_at(const Screen& s, float px, float py, float& u, float& v) {
    float l0, l1, l2;
    screen_bary(s, px, py, l0, l1, l2);
    const float a = l0 / s.w[0], b = l1 / s.w[1], c = l2 / s.w[2];
    const float inv = 1.0f / (a + b + c);
    u = c * inv;
    v = a * inv;
}

__device__ __forceinline__ uint32_t ordered(float z) {
    const uint32_t b = __float_as_uint(z);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void k_clear(unsigned long long* vis, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        vis[i] = ~0ull;
}

__global__ void k_raster(htex_geometry g, Camera cam, unsigned long long* vis) {
    for (int32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < g.H; h += gridDim.x * blockDim.x) {
        float3 v[3];
        alg1(g, h, v[0], v[1], v[2]);
        Screen s;
        if (!project(cam, v, s)) continue;
        const float xmin = fminf(s.x[0], fminf(s.x[1], s.x[2])), xmax = fmaxf(s.x[0], fmaxf(s.x[1], s.x[2]));
        const float ymin = fminf(s.y[0], fminf(s.y[1], s.y[2])), ymax = fmaxf(s.y[0], fmaxf(s.y[1], s.y[2]));
        const int x0 = max(0, int(ceilf(xmin - 0.5f))), x1 = min(cam.W - 1, int(floorf(xmax - 0.5f)));
        const int y0 = max(0, int(ceilf(ymin - 0.5f))), y1 = min(cam.Ht - 1, int(floorf(ymax - 0.5f)));
        for (int py = y0; py <= y1; ++py)
            for (int px = x0; px <= x1; ++px) {
                float l0, l1, l2;
                screen_bary(s, px + 0.5f, py + 0.5f, l0, l1, l2);
                if (!(l0 >= 0.0f && l1 >= 0.0f && l2 >= 0.0f)) continue;
                const float z = l0 * s.z[0] + l1 * s.z[1] + l2 * s.z[2];
                if (!(z >= -1.0f && z <= 1.0f)) continue;
                const unsigned long long key = (static_cast<unsigned long long>(ordered(z)) << 32) | uint32_t(h);
                atomicMin(vis + int64_t(py) * cam.W + px, key);
            }
    }
}

// Per pixel: the visible triangle's perspective-correct barycentrics at the
// pixel centre and at the centres one pixel right and one pixel down; Q is
// htex_query (footprint = the longer of the two differences) or
// htex_query_aniso (the two differences as the screen derivatives).
template <class Q>
__global__ void k_resolve(htex_geometry g, Camera cam, const unsigned long long* vis, Q* q, float* depth) {
    const int64_t n = int64_t(cam.W) * cam.Ht;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const unsigned long long key = vis[i];
        int32_t h = -1;
        float u = 0.0f, vv = 0.0f, ux = 0.0f, vx = 0.0f, uy = 0.0f, vy = 0.0f;
        float zd = __int_as_float(0x7fc00000);
        if (key != ~0ull) {
            h = int32_t(uint32_t(key & 0xffffffffull));
            float3 v[3];
            alg1(g, h, v[0], v[1], v[2]);
            Screen s;
            project(cam, v, s);
            const float px = float(i % cam.W) + 0.5f, py = float(i / cam.W) + 0.5f;
            uv_at(s, px, py, u, vv);
            uv_at(s, px + 1.0f, py, ux, vx);
            uv_at(s, px, py + 1.0f, uy, vy);
            float l0, l1, l2;
            screen_bary(s, px, py, l0, l1, l2);
            zd = l0 * s.z[0] + l1 * s.z[1] + l2 * s.z[2];
        }
        if constexpr (std::is_same<Q, htex_query_aniso>::value) {
            q[i] = h < 0 ? htex_query_aniso{-1, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}
                         : htex_query_aniso{h, u, vv, 0.0f, ux - u, vx - vv, uy - u, vy - vv};
        } else {
            q[i] = h < 0 ? htex_query{-1, 0.0f, 0.0f, 0.0f}
                         : htex_query{h, u, vv, fmaxf(hypotf(ux - u, vx - vv), hypotf(uy - u, vy - vv))};
        }
        if (depth) depth[i] = zd;
    }
}

// Displacement: lattice vertex k = (i, j), u = i/T, v = j/T of every
// halfedge triangle; queries first, then positions from the lookups.
__device__ __forceinline__ void lattice(int32_t k, int32_t T, float& u, float& v) {
    // k enumerates i = 0..T, j = 0..T-i in order
    int32_t i = 0, base = 0;
    while (base + (T + 1 - i) <= k) {
        base += T + 1 - i;
        ++i;
    }
    u = float(i) / float(T);
    v = float(k - base) / float(T);
}

__global__ void k_tess_queries(int32_t H, int32_t T, int32_t K, htex_query* q) {
    const int64_t n = int64_t(H) * K;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x) {
        float u, v;
        lattice(int32_t(t % K), T, u, v);
        q[t] = htex_query{int32_t(t / K), u, v, 0.0f};
    }
}

__global__ void k_displace(htex_geometry g, int32_t T, int32_t K, const float* d, int32_t C, int32_t channel,
                           float scale, float* out) {
    const int64_t n = int64_t(g.H) * K;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x) {
        const int32_t h = int32_t(t / K);
        float u, v;
        lattice(int32_t(t % K), T, u, v);
        const float w = 1.0f - u - v;
        float3 v0, v1, v2;
        alg1(g, h, v0, v1, v2);
        const float3 n2 = ld3(g.d_vn, g.d_vert[h]), n0 = ld3(g.d_vn, g.d_vert[g.d_next[h]]), n1 = ld3(g.d_fn, g.d_face[h]);
        float3 N = make_float3(u * n2.x + v * n0.x + w * n1.x, u * n2.y + v * n0.y + w * n1.y, u * n2.z + v * n0.z + w * n1.z);
        const float l = rsqrtf(N.x * N.x + N.y * N.y + N.z * N.z);
        const float s = scale * d[t * C + channel] * l;
        out[3 * t + 0] = u * v2.x + v * v0.x + w * v1.x + s * N.x;
        out[3 * t + 1] = u * v2.y + v * v0.y + w * v1.y + s * N.y;
        out[3 * t + 2] = u * v2.z + v * v0.z + w * v1.z + s * N.z;
    }
}

int grid_for(int64_t n) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return int(std::min<int64_t>((n + kThreads - 1) / kThreads, int64_t(sms) * 8));
}

void free_geometry(htex_geometry* g) {
    if (!g) return;
    cudaFree(g->d_next);
    cudaFree(g->d_vert);
    cudaFree(g->d_face);
    cudaFree(g->d_pos);
    cudaFree(g->d_vn);
    cudaFree(g->d_fn);
    delete g;
}

cudaMemPool_t work_pool(int device) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (device < 0 || device >= 64) return nullptr;
    if (!pools[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        if (cudaMemPoolCreate(&pools[device], &props) != cudaSuccess) return nullptr;
        uint64_t keep = ~uint64_t(0);
        cudaMemPoolSetAttribute(pools[device], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    return pools[device];
}

}  // namespace

extern "C" htex_status htex_geometry_create(const htex_mesh* m, const float* positions, htex_stream stream,
                                            htex_geometry** out) {
    if (!m || !positions || !out) return HTEX_ERR_INVALID_ARG;
    *out = nullptr;
    const int32_t H = m->H, V = m->V, F = m->F;
    std::vector<float> vn(size_t(V) * 3), fn(size_t(F) * 3);
    try {
        // normals of the input mesh: per face, its area vector (Newell's
        // formula); per vertex, the normalised sum of its faces' vectors
        std::vector<double> fa(size_t(F) * 3, 0.0), va(size_t(V) * 3, 0.0);
        for (int32_t h = 0; h < H; ++h) {
            const float* a = positions + 3 * size_t(m->vert[h]);
            const float* b = positions + 3 * size_t(m->vert[m->next[h]]);
            double* f = &fa[3 * size_t(m->face[h])];
            f[0] += 0.5 * (double(a[1]) * b[2] - double(a[2]) * b[1]);
            f[1] += 0.5 * (double(a[2]) * b[0] - double(a[0]) * b[2]);
            f[2] += 0.5 * (double(a[0]) * b[1] - double(a[1]) * b[0]);
        }
        for (int32_t h = 0; h < H; ++h)
            for (int k = 0; k < 3; ++k) va[3 * size_t(m->vert[h]) + k] += fa[3 * size_t(m->face[h]) + k];
        auto unit = [](const double* x, float* y) {
            const double l = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
            for (int k = 0; k < 3; ++k) y[k] = float(l > 0 ? x[k] / l : 0.0);
        };
        for (int32_t i = 0; i < V; ++i) unit(&va[3 * size_t(i)], &vn[3 * size_t(i)]);
        for (int32_t i = 0; i < F; ++i) unit(&fa[3 * size_t(i)], &fn[3 * size_t(i)]);
    } catch (const std::bad_alloc&) {
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    htex_geometry* g = new (std::nothrow) htex_geometry;
    if (!g) return HTEX_ERR_OUT_OF_MEMORY;
    g->H = H;
    g->V = V;
    g->F = F;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t hb = sizeof(int32_t) * size_t(H);
    bool ok = cudaMalloc(&g->d_next, hb) == cudaSuccess && cudaMalloc(&g->d_vert, hb) == cudaSuccess &&
              cudaMalloc(&g->d_face, hb) == cudaSuccess &&
              cudaMalloc(&g->d_pos, sizeof(float) * 3 * size_t(V)) == cudaSuccess &&
              cudaMalloc(&g->d_vn, sizeof(float) * 3 * size_t(V)) == cudaSuccess &&
              cudaMalloc(&g->d_fn, sizeof(float) * 3 * size_t(F)) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(g->d_next, m->next.data(), hb, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(g->d_vert, m->vert.data(), hb, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(g->d_face, m->face.data(), hb, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(g->d_pos, positions, sizeof(float) * 3 * size_t(V), cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(g->d_vn, vn.data(), sizeof(float) * 3 * size_t(V), cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(g->d_fn, fn.data(), sizeof(float) * 3 * size_t(F), cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_geometry(g);
        return HTEX_ERR_CUDA;
    }
    *out = g;
    return HTEX_OK;
}

extern "C" void htex_geometry_destroy(htex_geometry* g) { free_geometry(g); }

extern "C" htex_status htex_triangle_vertices(const htex_geometry* g, float* out, htex_stream stream) {
    if (!g || !out) return HTEX_ERR_INVALID_ARG;
    k_triangles<<<grid_for(g->H), kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(*g, out);
    return cudaGetLastError() == cudaSuccess ? HTEX_OK : HTEX_ERR_CUDA;
}

namespace {

template <class Q>
htex_status rasterize(const htex_geometry* g, const float* view_proj, int32_t width, int32_t height, Q* queries,
                      float* depth, htex_stream stream) {
    if (!g || !view_proj || !queries || width <= 0 || height <= 0) return HTEX_ERR_INVALID_ARG;
    if (int64_t(width) * height >= (int64_t(1) << 31)) return HTEX_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(queries) & 15u) != 0) return HTEX_ERR_INVALID_ARG;
    Camera cam;
    std::memcpy(cam.m, view_proj, sizeof(cam.m));
    cam.W = width;
    cam.Ht = height;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = int64_t(width) * height;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HTEX_ERR_CUDA;
    cudaMemPool_t pool = work_pool(dev);
    if (!pool) return HTEX_ERR_CUDA;
    void* vis = nullptr;
    if (cudaMallocFromPoolAsync(&vis, size_t(n) * 8, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    auto* v = static_cast<unsigned long long*>(vis);
    k_clear<<<grid_for(n), kThreads, 0, s>>>(v, n);
    k_raster<<<grid_for(g->H), kThreads, 0, s>>>(*g, cam, v);
    k_resolve<Q><<<grid_for(n), kThreads, 0, s>>>(*g, cam, v, queries, depth);
    const bool ok = cudaGetLastError() == cudaSuccess;
    cudaFreeAsync(vis, s);
    return ok ? HTEX_OK : HTEX_ERR_CUDA;
}

}  // namespace

extern "C" htex_status htex_rasterize(const htex_geometry* g, const float* view_proj, int32_t width, int32_t height,
                                      htex_query* queries, float* depth, htex_stream stream) {
    return rasterize(g, view_proj, width, height, queries, depth, stream);
}

extern "C" htex_status htex_rasterize_aniso(const htex_geometry* g, const float* view_proj, int32_t width,
                                            int32_t height, htex_query_aniso* queries, float* depth,
                                            htex_stream stream) {
    return rasterize(g, view_proj, width, height, queries, depth, stream);
}

extern "C" htex_status htex_displace(const htex_geometry* g, const htex_textures* t, int32_t tess, float scale,
                                     int32_t channel, float* out, htex_stream stream) {
    if (!g || !t || !out || tess < 1 || tess > 64 || channel < 0 || channel >= t->C || t->H != g->H)
        return HTEX_ERR_INVALID_ARG;
    const int32_t K = (tess + 1) * (tess + 2) / 2;
    const int64_t n = int64_t(g->H) * K;
    if (n >= (int64_t(1) << 31)) return HTEX_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HTEX_ERR_CUDA;
    cudaMemPool_t pool = work_pool(dev);
    if (!pool) return HTEX_ERR_CUDA;
    void* work = nullptr;
    const size_t qb = size_t(n) * sizeof(htex_query), db = size_t(n) * sizeof(float) * size_t(t->C);
    if (cudaMallocFromPoolAsync(&work, qb + db, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    auto* q = static_cast<htex_query*>(work);
    auto* d = reinterpret_cast<float*>(static_cast<uint8_t*>(work) + qb);
    k_tess_queries<<<grid_for(n), kThreads, 0, s>>>(g->H, tess, K, q);
    htex_status st = cudaGetLastError() == cudaSuccess ? HTEX_OK : HTEX_ERR_CUDA;
    if (st == HTEX_OK) st = htex_launch_lookup(t, q, n, d, HTEX_LOOKUP_GLOBAL, stream, nullptr);
    if (st == HTEX_OK) {
        k_displace<<<grid_for(n), kThreads, 0, s>>>(*g, tess, K, d, t->C, channel, scale, out);
        if (cudaGetLastError() != cudaSuccess) st = HTEX_ERR_CUDA;
    }
    cudaFreeAsync(work, s);
    return st;
}
