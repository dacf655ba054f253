// Halfedge mesh construction and validation (paper Section 2, Fig. 2;
// Section 3.2 for edges and boundary halfedges).  Host-only.
#include <cstring>
#include <new>
#include <unordered_map>

#include "htex_internal.h"

namespace {

// Directed edge key (origin, destination) packed into 64 bits.
inline uint64_t dkey(int32_t a, int32_t b) {
    return (uint64_t(uint32_t(a)) << 32) | uint32_t(b);
}

// Edge ids: a new id for the first halfedge of each pair met in id order
// (or for a boundary halfedge), the same id for its twin.
void number_edges(htex_mesh& m) {
    m.edge.assign(m.H, -1);
    int32_t E = 0, B = 0;
    for (int32_t h = 0; h < m.H; ++h) {
        int32_t g = m.twin[h];
        if (g < 0) {
            m.edge[h] = E++;
            ++B;
        } else if (m.edge[g] >= 0) {
            m.edge[h] = m.edge[g];
        } else {
            m.edge[h] = E++;
        }
    }
    m.E = E;
    m.B = B;
}

}  // namespace

extern "C" htex_status htex_mesh_create(const int32_t* face_sizes, int32_t num_faces,
                                        const int32_t* face_verts, int32_t num_verts,
                                        htex_mesh** out) {
    if (!out) return HTEX_ERR_INVALID_ARG;
    *out = nullptr;
    if (!face_sizes || !face_verts || num_faces <= 0 || num_verts <= 0) return HTEX_ERR_INVALID_ARG;
    int64_t H64 = 0;
    for (int32_t f = 0; f < num_faces; ++f) {
        if (face_sizes[f] < 3) return HTEX_ERR_INVALID_ARG;
        H64 += face_sizes[f];
    }
    if (H64 >= (int64_t(1) << 31)) return HTEX_ERR_INVALID_ARG;
    htex_mesh* m = new (std::nothrow) htex_mesh;
    if (!m) return HTEX_ERR_OUT_OF_MEMORY;
    try {
        const int32_t H = int32_t(H64);
        m->H = H;
        m->V = num_verts;
        m->F = num_faces;
        m->twin.resize(H);
        m->next.resize(H);
        m->prev.resize(H);
        m->vert.resize(H);
        m->face.resize(H);
        // A face's halfedges are contiguous: halfedge k of face f runs from
        // its k-th vertex to its (k+1)-th.
        int32_t start = 0;
        for (int32_t f = 0; f < num_faces; ++f) {
            const int32_t n = face_sizes[f];
            for (int32_t k = 0; k < n; ++k) {
                const int32_t v = face_verts[start + k];
                if (v < 0 || v >= num_verts) { delete m; return HTEX_ERR_INVALID_ARG; }
                m->vert[start + k] = v;
                m->face[start + k] = f;
                m->next[start + k] = start + (k + 1 == n ? 0 : k + 1);
                m->prev[start + k] = start + (k == 0 ? n - 1 : k - 1);
            }
            start += n;
        }
        // Twin matching through a hash of directed edges.
        std::unordered_map<uint64_t, int32_t> dir;
        dir.reserve(size_t(H) * 2);
        for (int32_t h = 0; h < H; ++h) {
            const int32_t a = m->vert[h], b = m->vert[m->next[h]];
            if (a == b) { delete m; return HTEX_ERR_INVALID_ARG; }
            if (!dir.emplace(dkey(a, b), h).second) { delete m; return HTEX_ERR_NONMANIFOLD; }
        }
        for (int32_t h = 0; h < H; ++h) {
            auto it = dir.find(dkey(m->vert[m->next[h]], m->vert[h]));
            m->twin[h] = (it == dir.end()) ? -1 : it->second;
        }
        number_edges(*m);
    } catch (const std::bad_alloc&) {
        delete m;
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    *out = m;
    return HTEX_OK;
}

extern "C" htex_status htex_mesh_create_from_halfedges(const int32_t* twin, const int32_t* next,
                                                       const int32_t* prev, const int32_t* vert,
                                                       const int32_t* edge, const int32_t* face,
                                                       int32_t H, int32_t num_verts,
                                                       int32_t num_faces, htex_mesh** out) {
    if (!out) return HTEX_ERR_INVALID_ARG;
    *out = nullptr;
    if (!twin || !next || !prev || !vert || !edge || !face || H <= 0 || num_verts <= 0 ||
        num_faces <= 0)
        return HTEX_ERR_INVALID_ARG;
    // ranges and the Next/Prev inverse pair
    for (int32_t h = 0; h < H; ++h) {
        if (next[h] < 0 || next[h] >= H || prev[h] < 0 || prev[h] >= H) return HTEX_ERR_INVALID_ARG;
        if (vert[h] < 0 || vert[h] >= num_verts || face[h] < 0 || face[h] >= num_faces)
            return HTEX_ERR_INVALID_ARG;
        if (twin[h] < -1 || twin[h] >= H || twin[h] == h) return HTEX_ERR_INVALID_ARG;
        if (edge[h] < 0 || edge[h] >= H) return HTEX_ERR_INVALID_ARG;
    }
    for (int32_t h = 0; h < H; ++h) {
        if (prev[next[h]] != h || next[prev[h]] != h) return HTEX_ERR_INVALID_ARG;
        if (face[next[h]] != face[h]) return HTEX_ERR_INVALID_ARG;
        if (vert[next[h]] == vert[h]) return HTEX_ERR_INVALID_ARG;
        const int32_t g = twin[h];
        if (g >= 0) {
            if (twin[g] != h) return HTEX_ERR_NONMANIFOLD;
            if (vert[g] != vert[next[h]] || vert[next[g]] != vert[h]) return HTEX_ERR_NONMANIFOLD;
            if (edge[g] != edge[h]) return HTEX_ERR_INVALID_ARG;
        }
    }
    // Next cycles of length >= 3
    std::vector<uint8_t> seen(size_t(H), 0);
    for (int32_t h = 0; h < H; ++h) {
        if (seen[h]) continue;
        int32_t len = 0, g = h;
        do {
            seen[g] = 1;
            g = next[g];
            ++len;
        } while (g != h && len <= H);
        if (len < 3) return HTEX_ERR_INVALID_ARG;
    }
    // Edge ids: a bijection of pairs (or lone boundary halfedges) onto [0, E)
    int32_t E = 0;
    for (int32_t h = 0; h < H; ++h) E = edge[h] + 1 > E ? edge[h] + 1 : E;
    std::vector<int32_t> first(size_t(E), -1);
    int32_t B = 0;
    for (int32_t h = 0; h < H; ++h) {
        const int32_t e = edge[h];
        if (twin[h] < 0) ++B;
        if (first[e] < 0) first[e] = h;
        else if (first[e] != twin[h]) return HTEX_ERR_INVALID_ARG;
    }
    for (int32_t e = 0; e < E; ++e)
        if (first[e] < 0) return HTEX_ERR_INVALID_ARG;
    htex_mesh* m = new (std::nothrow) htex_mesh;
    if (!m) return HTEX_ERR_OUT_OF_MEMORY;
    try {
        m->H = H;
        m->E = E;
        m->B = B;
        m->V = num_verts;
        m->F = num_faces;
        m->twin.assign(twin, twin + H);
        m->next.assign(next, next + H);
        m->prev.assign(prev, prev + H);
        m->vert.assign(vert, vert + H);
        m->edge.assign(edge, edge + H);
        m->face.assign(face, face + H);
    } catch (const std::bad_alloc&) {
        delete m;
        return HTEX_ERR_OUT_OF_MEMORY;
    }
    *out = m;
    return HTEX_OK;
}

extern "C" htex_status htex_mesh_info(const htex_mesh* m, int32_t* H, int32_t* E,
                                      int32_t* num_boundary, int32_t* num_verts,
                                      int32_t* num_faces) {
    if (!m) return HTEX_ERR_INVALID_ARG;
    if (H) *H = m->H;
    if (E) *E = m->E;
    if (num_boundary) *num_boundary = m->B;
    if (num_verts) *num_verts = m->V;
    if (num_faces) *num_faces = m->F;
    return HTEX_OK;
}

extern "C" htex_status htex_mesh_get_halfedges(const htex_mesh* m, int32_t* twin, int32_t* next,
                                               int32_t* prev, int32_t* vert, int32_t* edge,
                                               int32_t* face) {
    if (!m) return HTEX_ERR_INVALID_ARG;
    const size_t bytes = sizeof(int32_t) * size_t(m->H);
    if (twin) std::memcpy(twin, m->twin.data(), bytes);
    if (next) std::memcpy(next, m->next.data(), bytes);
    if (prev) std::memcpy(prev, m->prev.data(), bytes);
    if (vert) std::memcpy(vert, m->vert.data(), bytes);
    if (edge) std::memcpy(edge, m->edge.data(), bytes);
    if (face) std::memcpy(face, m->face.data(), bytes);
    return HTEX_OK;
}

extern "C" void htex_mesh_destroy(htex_mesh* m) { delete m; }

extern "C" const char* htex_status_string(htex_status s) {
    switch (s) {
    case HTEX_OK: return "ok";
    case HTEX_ERR_INVALID_ARG: return "invalid argument";
    case HTEX_ERR_NONMANIFOLD: return "non-manifold mesh";
    case HTEX_ERR_BAD_TEXTURE: return "bad texture";
    case HTEX_ERR_OUT_OF_MEMORY: return "out of memory";
    case HTEX_ERR_CUDA: return "CUDA error";
    case HTEX_ERR_QUERY_OUT_OF_RANGE: return "query out of range";
    case HTEX_ERR_TIMEOUT: return "timeout";
    case HTEX_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}
