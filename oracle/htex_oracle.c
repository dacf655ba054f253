/*
 * Htex FP64 CPU oracle — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, deliberately unoptimised restatement of what per-halfedge
 * texturing (Barbier & Dupuy 2022, "Htex: Per-Halfedge Texturing for
 * Arbitrary Mesh Topologies") computes, evaluated in double precision.
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file's library.  It shares no code, header,
 * table or helper with the CUDA library in paper_2207_05618_gb300/.
 *
 * Conventions (each fixed by the passage cited at the function):
 *   - halfedge arrays twin/next/prev/vert/edge/face, int32, Twin = -1 on the
 *     boundary (paper Section 2, Fig. 2 table);
 *   - textures: one square texture per edge, power-of-two size N_e = 2^n_e,
 *     n_e + 1 mip levels N_e, N_e/2, ..., 1 (Section 4.3).  Inside this file
 *     the texel values live in one double array: texture e starts at texel
 *     index toff[e]; its levels follow each other; level l is row-major
 *     [N_l][N_l][C] with texel (i, j) = column i (along quad x), row j
 *     (along quad y) at j * N_l + i.
 *
 * Numbers, not bytes, are what the oracle reasons about; the byte packer at
 * the end writes the documented storage format so stored pools can be
 * compared bit for bit.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* storage formats (numbering is the oracle's own; the Python wrapper maps names) */
enum { ORC_F32 = 0, ORC_U8 = 1, ORC_F16 = 2, ORC_BF16 = 3, ORC_E4M3 = 4 };
enum { ORC_FLAG_BUILD_MIPS = 1, ORC_FLAG_MIRROR = 2, ORC_FLAG_FIX_CORNERS = 4 };

/* ------------------------------------------------------------------------
 * Mesh from polygon faces (Section 2, Fig. 2; Section 3.2).
 * The halfedges of face f are contiguous, in the face's vertex order.  With
 * k the position in the face and n its size: Next = start + (k+1) mod n,
 * Prev = start + (k-1) mod n, Vert(h) = k-th vertex (the origin of h),
 * Face(h) = f.  Twin(h) is the halfedge g running the other way
 * (Vert(g) = Vert(Next h), Vert(Next g) = Vert(h)), or -1 on the boundary.
 * Edge ids: scan h = 0..H-1, a new id whenever Twin(h) < 0 or h < Twin(h);
 * Twin(h) takes the same id (any twin-consistent numbering is valid; this
 * one is the oracle's and the library's documented default).
 * Returns 0, 1 (bad input: face of < 3 vertices, vertex out of range or a
 * zero-length edge), 2 (non-manifold: a directed edge used twice).
 * ---------------------------------------------------------------------- */
typedef struct { int64_t key; int32_t h; } orc_dedge;

static int cmp_dedge(const void* a, const void* b)
{
    const orc_dedge* x = (const orc_dedge*)a;
    const orc_dedge* y = (const orc_dedge*)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->h < y->h) ? -1 : (x->h > y->h);
}

int orc_mesh_from_faces(int32_t F, const int32_t* face_sizes, const int32_t* face_verts,
                        int32_t V, int32_t H, int32_t* twin, int32_t* next, int32_t* prev,
                        int32_t* vert, int32_t* edge, int32_t* face, int32_t* E_out)
{
    int32_t h = 0;
    for (int32_t f = 0; f < F; ++f) {
        int32_t n = face_sizes[f];
        if (n < 3) return 1;
        for (int32_t k = 0; k < n; ++k) {
            int32_t v = face_verts[h + k];
            if (v < 0 || v >= V) return 1;
            next[h + k] = h + (k + 1) % n;
            prev[h + k] = h + (k + n - 1) % n;
            vert[h + k] = v;
            face[h + k] = f;
        }
        h += n;
    }
    if (h != H) return 1;

    /* every directed edge (Vert h -> Vert Next h), sorted by key = a * V + b */
    orc_dedge* d = (orc_dedge*)malloc(sizeof(orc_dedge) * (size_t)(H > 0 ? H : 1));
    for (int32_t g = 0; g < H; ++g) {
        int64_t a = vert[g], b = vert[next[g]];
        if (a == b) { free(d); return 1; }
        d[g].key = a * (int64_t)V + b;
        d[g].h = g;
    }
    qsort(d, (size_t)H, sizeof(orc_dedge), cmp_dedge);
    for (int32_t i = 1; i < H; ++i)
        if (d[i].key == d[i - 1].key) { free(d); return 2; }

    for (int32_t g = 0; g < H; ++g) {
        /* binary search for the reverse directed edge */
        int64_t want = (int64_t)vert[next[g]] * V + vert[g];
        int32_t lo = 0, hi = H - 1, found = -1;
        while (lo <= hi) {
            int32_t mid = lo + (hi - lo) / 2;
            if (d[mid].key == want) { found = d[mid].h; break; }
            if (d[mid].key < want) lo = mid + 1; else hi = mid - 1;
        }
        twin[g] = found;
    }
    free(d);

    int32_t E = 0;
    for (int32_t g = 0; g < H; ++g) {
        if (twin[g] < 0 || g < twin[g]) edge[g] = E++;
        else edge[g] = edge[twin[g]];
    }
    *E_out = E;
    return 0;
}

/* For every edge, the halfedge that owns the lower-left half of its quad:
 * the larger id of the halfedge/twin pair (Alg. 2), or the boundary
 * halfedge itself (Section 3.2, boundary halfedge paired with itself). */
void orc_edge_owner(int32_t H, const int32_t* twin, const int32_t* edge, int32_t* owner)
{
    for (int32_t g = 0; g < H; ++g)
        if (twin[g] < g) owner[edge[g]] = g;   /* twin = -1 also satisfies this */
}

/* ------------------------------------------------------------------------
 * Texture layout inside the oracle: texel-count offsets of each texture.
 * ---------------------------------------------------------------------- */
int64_t orc_texels_in_chain(int32_t n)
{
    int64_t t = 0;
    for (int32_t l = 0; l <= n; ++l) t += ((int64_t)1 << (n - l)) * ((int64_t)1 << (n - l));
    return t;
}

void orc_texture_offsets(int32_t E, const int32_t* log2n, int64_t* toff)
{
    int64_t t = 0;
    for (int32_t e = 0; e < E; ++e) { toff[e] = t; t += orc_texels_in_chain(log2n[e]); }
    toff[E] = t;
}

static int64_t level_base(int64_t toff_e, int32_t n, int32_t l)
{
    int64_t t = toff_e;
    for (int32_t k = 0; k < l; ++k) t += ((int64_t)1 << (n - k)) * ((int64_t)1 << (n - k));
    return t;
}

/* Round a double to the nearest float (the stored precision of float data). */
static double to_f32(double x) { return (double)(float)x; }

/* Mip levels: texel (i, j) of level l+1 is the mean of the 2x2 block
 * (2i..2i+1, 2j..2j+1) of level l.  The paper leaves mip generation to the
 * graphics API; this is the box filter, summed as ((a+b)+c)+d with
 * a=(2i,2j), b=(2i+1,2j), c=(2i,2j+1), d=(2i+1,2j+1), rounded once to the
 * stored precision.  8-bit data uses the integer mean (a+b+c+d+2) >> 2. */
void orc_build_mips(int32_t E, const int32_t* log2n, const int64_t* toff, int32_t C,
                    int32_t fmt_u8, double* tex)
{
    for (int32_t e = 0; e < E; ++e) {
        int32_t n = log2n[e];
        for (int32_t l = 0; l < n; ++l) {
            int64_t src = level_base(toff[e], n, l), dst = level_base(toff[e], n, l + 1);
            int32_t Ns = 1 << (n - l), Nd = Ns >> 1;
            for (int32_t j = 0; j < Nd; ++j)
                for (int32_t i = 0; i < Nd; ++i)
                    for (int32_t c = 0; c < C; ++c) {
                        double a = tex[(src + (int64_t)(2 * j) * Ns + 2 * i) * C + c];
                        double b = tex[(src + (int64_t)(2 * j) * Ns + 2 * i + 1) * C + c];
                        double cc = tex[(src + (int64_t)(2 * j + 1) * Ns + 2 * i) * C + c];
                        double d = tex[(src + (int64_t)(2 * j + 1) * Ns + 2 * i + 1) * C + c];
                        double m;
                        if (fmt_u8) m = (double)(((int64_t)a + (int64_t)b + (int64_t)cc + (int64_t)d + 2) >> 2);
                        else m = to_f32((((a + b) + cc) + d) * 0.25);
                        tex[(dst + (int64_t)j * Nd + i) * C + c] = m;
                    }
        }
    }
}

/* Boundary mirroring (Section 4.3): a boundary edge's quad holds only the
 * real triangle (lower-left half, x + y <= 1); the other half mirrors it
 * across the diagonal x + y = 1, which is where the virtual twin triangle
 * would lie (Section 3.2).  Texel (i, j) with i + j > N - 1 takes the value
 * of (N-1-j, N-1-i).  Applied to every level, or to level 0 alone when
 * 'level0_only' is set (before the mips are built from it). */
void orc_mirror_boundary(int32_t E, const int32_t* log2n, const int64_t* toff, int32_t C,
                         const int32_t* owner, const int32_t* twin, int32_t level0_only, double* tex)
{
    for (int32_t e = 0; e < E; ++e) {
        if (twin[owner[e]] >= 0) continue;
        int32_t n = log2n[e];
        int32_t last = level0_only ? 0 : n;
        for (int32_t l = 0; l <= last; ++l) {
            int64_t base = level_base(toff[e], n, l);
            int32_t N = 1 << (n - l);
            for (int32_t j = 0; j < N; ++j)
                for (int32_t i = 0; i < N; ++i)
                    if (i + j > N - 1)
                        for (int32_t c = 0; c < C; ++c)
                            tex[(base + (int64_t)j * N + i) * C + c] =
                                tex[(base + (int64_t)(N - 1 - i) * N + (N - 1 - j)) * C + c];
        }
    }
}

/* ------------------------------------------------------------------------
 * Corner pre-processing (Section 4.4, "Corner Pre-processing"): the corner
 * texels that meet at one point of the surface are set to one common value,
 * the mean of the group, separately for every resolution R.
 * The points are the mesh vertices and the face centroids.  For the owner
 * h of edge e (the larger id of the pair), texel (R-1, 0) sits at Vert(h),
 * (0, R-1) at Vert(Next h), (0, 0) at the centroid of Face(h) and
 * (R-1, R-1) at the centroid of Face(Twin h); for a boundary edge the last
 * one is the mirror image of (0, 0) and joins the centroid of Face(h) when
 * boundaries are mirrored, else it is left alone.  At R = 1 one texel is
 * all four corners, so groups are the connected components of the
 * texel/point incidence (union-find over points).
 * ---------------------------------------------------------------------- */
static int32_t uf_find(int32_t* p, int32_t x)
{
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
}

void orc_fix_corners(int32_t E, const int32_t* log2n, const int64_t* toff, int32_t C,
                     int32_t fmt_u8, int32_t mirrored, const int32_t* owner,
                     const int32_t* twin, const int32_t* next, const int32_t* vert,
                     const int32_t* face, int32_t V, int32_t F, double* tex)
{
    int32_t nmax = 0;
    for (int32_t e = 0; e < E; ++e) if (log2n[e] > nmax) nmax = log2n[e];
    int32_t P = V + F;
    int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)P);
    double* sum = (double*)malloc(sizeof(double) * (size_t)P * (size_t)C);
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)P);

    for (int32_t r = 0; r <= nmax; ++r) {          /* resolution R = 2^r */
        int32_t R = 1 << r;
        for (int32_t p = 0; p < P; ++p) parent[p] = p;
        /* slots: up to 4 (texel index, point) pairs per texture */
        for (int pass = 0; pass < 3; ++pass) {
            if (pass == 1) {
                for (int32_t p = 0; p < P; ++p) { cnt[p] = 0; for (int32_t c = 0; c < C; ++c) sum[(int64_t)p * C + c] = 0.0; }
            }
            for (int32_t e = 0; e < E; ++e) {
                int32_t n = log2n[e];
                if (n < r) continue;
                int32_t h = owner[e];
                int64_t base = level_base(toff[e], n, n - r);
                int64_t tx[4];
                int32_t pt[4];
                int ns = 0;
                tx[ns] = (int64_t)0 * R + (R - 1); pt[ns++] = vert[h];               /* (R-1, 0) */
                tx[ns] = (int64_t)(R - 1) * R + 0; pt[ns++] = vert[next[h]];         /* (0, R-1) */
                tx[ns] = 0;                        pt[ns++] = V + face[h];           /* (0, 0)   */
                if (twin[h] >= 0) { tx[ns] = (int64_t)(R - 1) * R + (R - 1); pt[ns++] = V + face[twin[h]]; }
                else if (mirrored) { tx[ns] = (int64_t)(R - 1) * R + (R - 1); pt[ns++] = V + face[h]; }
                if (pass == 0) {
                    /* link the points of slots that are the same texel */
                    for (int a = 0; a < ns; ++a)
                        for (int b = a + 1; b < ns; ++b)
                            if (tx[a] == tx[b]) {
                                int32_t x = uf_find(parent, pt[a]), y = uf_find(parent, pt[b]);
                                if (x != y) parent[x] = y;
                            }
                } else {
                    /* each distinct texel counted once, under its group's root */
                    for (int a = 0; a < ns; ++a) {
                        int dup = 0;
                        for (int b = 0; b < a; ++b) if (tx[b] == tx[a]) dup = 1;
                        if (dup) continue;
                        int32_t g = uf_find(parent, pt[a]);
                        double* t = &tex[(base + tx[a]) * C];
                        if (pass == 1) {
                            cnt[g] += 1;
                            for (int32_t c = 0; c < C; ++c) sum[(int64_t)g * C + c] += t[c];
                        } else {
                            for (int32_t c = 0; c < C; ++c) {
                                double s = sum[(int64_t)g * C + c];
                                double m;
                                if (fmt_u8) m = floor((2.0 * s + (double)cnt[g]) / (2.0 * (double)cnt[g]));
                                else m = to_f32(s / (double)cnt[g]);
                                t[c] = m;
                            }
                        }
                    }
                }
            }
        }
    }
    free(parent); free(sum); free(cnt);
}

/* ------------------------------------------------------------------------
 * Reduced-precision storage (not in the paper): round-to-nearest-even of
 * x = T / s into a binary format with p significand bits (implicit bit
 * included), minimum normal exponent emin and largest finite value maxv.
 * E4M3 saturates at 448; FP16/BF16 overflow to infinity (unreachable after
 * scaling).  Written from the IEEE-754 / OCP FP8 definitions.
 * ---------------------------------------------------------------------- */
static double round_to_format(double x, int p, int emin, double maxv, int saturate)
{
    if (x == 0.0 || isnan(x)) return x;
    double ax = fabs(x);
    int e = ilogb(ax);
    if (e < emin) e = emin;                        /* subnormal: fixed quantum */
    double quantum = ldexp(1.0, e - p + 1);
    double r = nearbyint(ax / quantum) * quantum;  /* default rounding mode: to nearest even */
    if (r > maxv) r = saturate ? maxv : INFINITY;
    return copysign(r, x);
}

double orc_round_f16(double x) { return round_to_format(x, 11, -14, 65504.0, 0); }
double orc_round_bf16(double x) { return round_to_format(x, 8, -126, ldexp(255.0, 120), 0); }
double orc_round_e4m3(double x) { return round_to_format(x, 4, -6, 448.0, 1); }

/* bit encoders of already-rounded values */
static uint32_t encode_bits(double r, int p, int emin, int ebits)
{
    uint32_t sign = signbit(r) ? 1u : 0u;
    double ar = fabs(r);
    int mbits = p - 1;
    uint32_t bias = (1u << (ebits - 1)) - 1u;
    uint32_t E, M;
    if (isinf(ar)) { E = (1u << ebits) - 1u; M = 0; }
    else if (ar == 0.0) { E = 0; M = 0; }
    else {
        int e = ilogb(ar);
        if (e < emin) { E = 0; M = (uint32_t)ldexp(ar, -(emin - mbits)); }
        else { E = (uint32_t)(e + (int)bias); M = (uint32_t)(ldexp(ar, -e) * (double)(1u << mbits)) - (1u << mbits); }
    }
    return (sign << (ebits + mbits)) | (E << mbits) | M;
}

static double decode_bits(uint32_t b, int p, int emin, int ebits, int e4m3)
{
    int mbits = p - 1;
    uint32_t sign = (b >> (ebits + mbits)) & 1u;
    uint32_t E = (b >> mbits) & ((1u << ebits) - 1u);
    uint32_t M = b & ((1u << mbits) - 1u);
    double v;
    int bias = (1 << (ebits - 1)) - 1;
    if (e4m3 && E == 15u && M == 7u) v = NAN;
    else if (!e4m3 && E == (1u << ebits) - 1u) v = M ? NAN : INFINITY;
    else if (E == 0) v = ldexp((double)M, emin - mbits);
    else v = ldexp(1.0 + (double)M / (double)(1u << mbits), (int)E - bias);
    return sign ? -v : v;
}

uint32_t orc_encode(int32_t fmt, double rounded)
{
    switch (fmt) {
    case ORC_F16: return encode_bits(rounded, 11, -14, 5);
    case ORC_BF16: return encode_bits(rounded, 8, -126, 8);
    case ORC_E4M3: return encode_bits(rounded, 4, -6, 4);
    }
    return 0;
}

double orc_decode(int32_t fmt, uint32_t bits)
{
    switch (fmt) {
    case ORC_F16: return decode_bits(bits, 11, -14, 5, 0);
    case ORC_BF16: return decode_bits(bits, 8, -126, 8, 0);
    case ORC_E4M3: return decode_bits(bits, 4, -6, 4, 1);
    }
    return NAN;
}

/* Per-texture scale: E4M3 s = max|T| / 448 (so the largest texel maps to the
 * largest finite code), FP16/BF16 s = max|T|; s = 1 for an all-zero
 * texture; rounded to float.  Every stored level counts toward the max.
 * Then each value becomes decode(encode(round(T / s))) * s, exactly in
 * double (a <= 11-bit code times a 24-bit scale). */
void orc_quantize(int32_t E, const int32_t* log2n, const int64_t* toff, int32_t C,
                  int32_t fmt, double* tex, uint32_t* codes, float* scales)
{
    for (int32_t e = 0; e < E; ++e) {
        int64_t a = toff[e] * C, b = toff[e + 1] * C;
        double m = 0.0;
        for (int64_t k = a; k < b; ++k) if (fabs(tex[k]) > m) m = fabs(tex[k]);
        double s;
        if (m == 0.0) s = 1.0;
        else if (fmt == ORC_E4M3) s = to_f32(m / 448.0);
        else s = to_f32(m);
        scales[e] = (float)s;
        for (int64_t k = a; k < b; ++k) {
            double x = tex[k] / s, r;
            if (fmt == ORC_F16) r = orc_round_f16(x);
            else if (fmt == ORC_BF16) r = orc_round_bf16(x);
            else r = orc_round_e4m3(x);
            codes[k] = orc_encode(fmt, r);
            tex[k] = orc_decode(fmt, codes[k]) * s;
        }
    }
    (void)log2n;
}

/* ------------------------------------------------------------------------
 * Filtered lookup (Section 4.4, Alg. 3 with Alg. 2).
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t H;
    const int32_t *twin, *next, *prev, *edge;
    const int32_t* log2n;      /* [E] */
    const int64_t* toff;       /* [E+1] texel offsets */
    const double* tex;         /* values, C per texel */
    int32_t C;
} orc_asset;

/* Alg. 2: the halfedge with the larger id takes the lower-left half of the
 * quad with its barycentrics unchanged; the other is reflected. */
static void triangle_to_quad_uv(const orc_asset* A, int32_t h, double u, double v, double* x, double* y)
{
    if (h > A->twin[h]) { *x = u; *y = v; }
    else { *x = 1.0 - u; *y = 1.0 - v; }
}

/* Bilinear sample of one level with a zero border plus the matching weight
 * of an all-ones normalisation channel (Section 4.4: CLAMP_TO_BORDER with
 * border 0 and a border-normalisation channel).  Texel centres sit at
 * ((i + 1/2) / N, (j + 1/2) / N).  'wl' scales the level's contribution
 * (trilinear blending). */
static void sample_level(const orc_asset* A, int32_t e, int32_t l, double x, double y, double wl,
                         double* acc, double* W, double* gout, double* grad, double invW)
{
    int32_t n = A->log2n[e];
    int32_t N = 1 << (n - l);
    int64_t base = level_base(A->toff[e], n, l);
    double s = x * N - 0.5, t = y * N - 0.5;
    double fi = floor(s), fj = floor(t);
    double a = s - fi, b = t - fj;
    for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
            double i = fi + di, j = fj + dj;
            double w = (di ? a : 1.0 - a) * (dj ? b : 1.0 - b);
            if (i < 0 || j < 0 || i >= N || j >= N) continue;
            int64_t k = (base + (int64_t)j * N + (int64_t)i) * A->C;
            if (grad) {
                for (int32_t c = 0; c < A->C; ++c) grad[k + c] += gout[c] * wl * w * invW;
            } else {
                *W += wl * w;
                for (int32_t c = 0; c < A->C; ++c) acc[c] += wl * w * A->tex[k + c];
            }
        }
}

/* One of the three texture fetches of Alg. 3 with level selection.  The
 * paper leaves level selection to the sampler; the oracle's rule: the
 * footprint f is in quad-uv units, lambda = log2(f * N_e); level 0 when
 * lambda is not > 0 (f <= 0 included), the last level when floor(lambda)
 * reaches it, else levels d = floor(lambda) and d + 1 blended 1 - phi, phi
 * with phi = lambda - d. */
static void fetch(const orc_asset* A, int32_t e, double x, double y, double f,
                  double* acc, double* W, double* gout, double* grad, double invW)
{
    int32_t n = A->log2n[e];
    double lam = (f > 0.0) ? log2(f * (double)(1 << n)) : -1.0;
    if (!(lam > 0.0)) { sample_level(A, e, 0, x, y, 1.0, acc, W, gout, grad, invW); return; }
    double d = floor(lam);
    double phi = lam - d;
    if (d >= (double)n) { sample_level(A, e, n, x, y, 1.0, acc, W, gout, grad, invW); return; }
    sample_level(A, e, (int32_t)d, x, y, 1.0 - phi, acc, W, gout, grad, invW);
    sample_level(A, e, (int32_t)d + 1, x, y, phi, acc, W, gout, grad, invW);
}

/* Query domain (Section 4.2): u weighs Vert(h), v weighs Vert(Next h),
 * 1 - u - v the face centroid.  Outside the closed triangle a finite query
 * is clamped: negatives to 0, then (u, v) scaled back onto u + v = 1.  (A
 * query with an invalid h or a non-finite u or v has no value: NaN.) */
static void clamp_query(double* u, double* v)
{
    double uu = *u, vv = *v;
    if (!(uu > 0.0)) uu = 0.0;
    if (!(vv > 0.0)) vv = 0.0;
    double s = uu + vv;
    if (s > 1.0) { uu /= s; vv /= s; }
    *u = uu; *v = vv;
}

/* Alg. 3: own quad at (u, v), Next's quad at (v, -u), Prev's quad at
 * (-v, u), each through Alg. 2; the data sums are divided by the summed
 * normalisation weight.  An invalid h yields NaN.  With 'grad' set, the
 * same weights scatter gout * w / W into the texel gradient instead
 * (the lookup is linear in the texels). */
static void lookup_one(const orc_asset* A, int32_t h, double u, double v, double f,
                       double* out, double* wout, double* gout, double* grad)
{
    int32_t C = A->C;
    if (h < 0 || h >= A->H || !isfinite(u) || !isfinite(v)) {
        if (out) for (int32_t c = 0; c < C; ++c) out[c] = NAN;
        if (wout) *wout = NAN;
        return;
    }
    clamp_query(&u, &v);
    int32_t hn = A->next[h], hp = A->prev[h];
    double x[3], y[3];
    int32_t e[3];
    triangle_to_quad_uv(A, h, u, v, &x[0], &y[0]);   e[0] = A->edge[h];
    triangle_to_quad_uv(A, hn, v, -u, &x[1], &y[1]); e[1] = A->edge[hn];
    triangle_to_quad_uv(A, hp, -v, u, &x[2], &y[2]); e[2] = A->edge[hp];

    double acc[16], W = 0.0;
    for (int32_t c = 0; c < C; ++c) acc[c] = 0.0;
    for (int k = 0; k < 3; ++k) fetch(A, e[k], x[k], y[k], f, acc, &W, NULL, NULL, 0.0);
    if (grad) {
        double invW = 1.0 / W;
        for (int k = 0; k < 3; ++k) fetch(A, e[k], x[k], y[k], f, NULL, NULL, gout, grad, invW);
    }
    if (out) for (int32_t c = 0; c < C; ++c) out[c] = acc[c] / W;
    if (wout) *wout = W;
}

typedef struct {
    const orc_asset* A;
    const int32_t* h;
    const double *u, *v, *f;
    double* out;
    double* wsum;
    int64_t begin, end;
} orc_job;

static void* lookup_job(void* arg)
{
    orc_job* J = (orc_job*)arg;
    for (int64_t q = J->begin; q < J->end; ++q)
        lookup_one(J->A, J->h[q], J->u[q], J->v[q], J->f[q], J->out + q * J->A->C,
                   J->wsum ? J->wsum + q : NULL, NULL, NULL);
    return NULL;
}

/* Lookups of n queries; 'nthreads' splits the query range (no other change).
 * 'wsum' (nullable) receives each query's summed normalisation weight. */
void orc_lookup(int32_t H, const int32_t* twin, const int32_t* next, const int32_t* prev,
                const int32_t* edge, const int32_t* log2n, const int64_t* toff, const double* tex,
                int32_t C, int64_t n, const int32_t* qh, const double* qu, const double* qv,
                const double* qf, double* out, double* wsum, int32_t nthreads)
{
    orc_asset A = {H, twin, next, prev, edge, log2n, toff, tex, C};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    orc_job jobs[256];
    for (int32_t t = 0; t < nthreads; ++t) {
        jobs[t].A = &A; jobs[t].h = qh; jobs[t].u = qu; jobs[t].v = qv; jobs[t].f = qf; jobs[t].out = out;
        jobs[t].wsum = wsum;
        jobs[t].begin = n * t / nthreads; jobs[t].end = n * (t + 1) / nthreads;
    }
    if (nthreads == 1) { lookup_job(&jobs[0]); return; }
    for (int32_t t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, lookup_job, &jobs[t]);
    for (int32_t t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* Gradient of L = sum_q sum_c gout[q][c] * out[q][c] with respect to every
 * stored texel value (oracle layout); single-threaded, accumulates into grad. */
void orc_lookup_grad(int32_t H, const int32_t* twin, const int32_t* next, const int32_t* prev,
                     const int32_t* edge, const int32_t* log2n, const int64_t* toff,
                     const double* tex, int32_t C, int64_t n, const int32_t* qh, const double* qu,
                     const double* qv, const double* qf, const double* gout, double* grad)
{
    orc_asset A = {H, twin, next, prev, edge, log2n, toff, tex, C};
    for (int64_t q = 0; q < n; ++q)
        lookup_one(&A, qh[q], qu[q], qv[q], qf[q], NULL, NULL, (double*)(gout + q * C), grad);
}

/* ------------------------------------------------------------------------
 * Anisotropic lookup.  Section 5.1 renders Htex with the GPU's anisotropic
 * filter applied to each of Alg. 3's three texture fetches; the paper gives
 * no formula of its own, so this is the reading of it (one sampler applied
 * to each fetch, one shared normalisation):
 *   - the footprint is given by the screen derivatives of the barycentrics,
 *     ax = (du/dx, dv/dx) and ay = (du/dy, dv/dy), in quad-uv units (the
 *     quad coordinates of every fetch are the barycentrics up to a rotation
 *     or reflection, so lengths are the same in all three);
 *   - px2 = |ax|^2, py2 = |ay|^2; the major axis m is ay when py2 > px2,
 *     else ax; the probe count K is 1 when both are zero, else
 *     min(ceil(sqrt(max / min)), kmax) (min = 0 gives kmax).  K is an
 *     integer decided by rounding, so it is computed in FP32 with the same
 *     operations as the kernel (each product, sum, quotient and square root
 *     rounded to float);
 *   - each probe is an isotropic trilinear sample (the level rule of
 *     'fetch') with footprint Pmax / K, Pmax = sqrt(max);
 *   - the K probes sit at c + m * s * ((k + 1/2) / K - 1/2), k = 0..K-1,
 *     around the clamped centre c, with s = min(1, K / Pmax): the probes
 *     span the major axis, but never more than K quad widths;
 *   - every probe samples all three fetches of Alg. 3 at its own (u', v'):
 *     own quad at (u', v'), Next's at (v', -u'), Prev's at (-v', u'), each
 *     through Alg. 2, full 2x2 taps with a zero border; the result is the
 *     summed data over the summed normalisation weight (0 / 0 = NaN when
 *     every tap of every probe falls outside the three quads).
 * An invalid h, a non-finite u, v or derivative, or an overflowing |ax|^2
 * or |ay|^2 gives NaN.
 * ---------------------------------------------------------------------- */
static int32_t aniso_probes(float dudx, float dvdx, float dudy, float dvdy, int32_t kmax, int* major_y,
                            double* pmax)
{
    volatile float px2 = dudx * dudx;
    px2 = px2 + (float)(dvdx * dvdx);
    volatile float py2 = dudy * dudy;
    py2 = py2 + (float)(dvdy * dvdy);
    *major_y = py2 > px2;
    float mx = *major_y ? py2 : px2, mn = *major_y ? px2 : py2;
    *pmax = sqrt((double)mx);
    if (mx == 0.0f) return 1;
    volatile float q = mx / mn;
    float r = sqrtf(q);
    if (!(r < (float)kmax)) return kmax;
    int32_t k = (int32_t)ceilf(r);
    return k < 1 ? 1 : k;
}

static void lookup_aniso_one(const orc_asset* A, int32_t h, double u, double v, const float* d, int32_t kmax,
                             double* out)
{
    int32_t C = A->C;
    int ok = h >= 0 && h < A->H && isfinite(u) && isfinite(v);
    for (int k = 0; k < 4; ++k) ok = ok && isfinite(d[k]);
    if (ok) {
        float px2 = d[0] * d[0], py2 = d[2] * d[2];
        px2 = px2 + (float)(d[1] * d[1]);
        py2 = py2 + (float)(d[3] * d[3]);
        ok = isfinite(px2) && isfinite(py2);
    }
    if (!ok) {
        for (int32_t c = 0; c < C; ++c) out[c] = NAN;
        return;
    }
    clamp_query(&u, &v);
    int major_y;
    double pmax;
    int32_t K = aniso_probes(d[0], d[1], d[2], d[3], kmax, &major_y, &pmax);
    double mu = major_y ? d[2] : d[0], mv = major_y ? d[3] : d[1];
    double s = (pmax > (double)K) ? (double)K / pmax : 1.0;
    double fiso = pmax / (double)K;
    int32_t hn = A->next[h], hp = A->prev[h];
    int32_t e[3] = {A->edge[h], A->edge[hn], A->edge[hp]};
    double acc[16], W = 0.0;
    for (int32_t c = 0; c < C; ++c) acc[c] = 0.0;
    for (int32_t k = 0; k < K; ++k) {
        double t = ((double)k + 0.5) / (double)K - 0.5;
        double pu = u + mu * s * t, pv = v + mv * s * t;
        double x[3], y[3];
        triangle_to_quad_uv(A, h, pu, pv, &x[0], &y[0]);
        triangle_to_quad_uv(A, hn, pv, -pu, &x[1], &y[1]);
        triangle_to_quad_uv(A, hp, -pv, pu, &x[2], &y[2]);
        for (int f = 0; f < 3; ++f) fetch(A, e[f], x[f], y[f], fiso, acc, &W, NULL, NULL, 0.0);
    }
    for (int32_t c = 0; c < C; ++c) out[c] = acc[c] / W;
}

typedef struct {
    const orc_asset* A;
    const int32_t* h;
    const double *u, *v;
    const float* d;
    int32_t kmax;
    double* out;
    int64_t begin, end;
} orc_aniso_job;

static void* aniso_job(void* arg)
{
    orc_aniso_job* J = (orc_aniso_job*)arg;
    for (int64_t q = J->begin; q < J->end; ++q)
        lookup_aniso_one(J->A, J->h[q], J->u[q], J->v[q], J->d + 4 * q, J->kmax, J->out + q * J->A->C);
    return NULL;
}

/* Anisotropic lookups of n queries; d holds du/dx, dv/dx, du/dy, dv/dy per
 * query (float, as stored in the query); kmax >= 1 bounds the probe count. */
void orc_lookup_aniso(int32_t H, const int32_t* twin, const int32_t* next, const int32_t* prev,
                      const int32_t* edge, const int32_t* log2n, const int64_t* toff, const double* tex,
                      int32_t C, int64_t n, const int32_t* qh, const double* qu, const double* qv,
                      const float* qd, int32_t kmax, double* out, int32_t nthreads)
{
    orc_asset A = {H, twin, next, prev, edge, log2n, toff, tex, C};
    if (kmax < 1) kmax = 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    orc_aniso_job jobs[256];
    for (int32_t t = 0; t < nthreads; ++t) {
        jobs[t].A = &A; jobs[t].h = qh; jobs[t].u = qu; jobs[t].v = qv; jobs[t].d = qd; jobs[t].kmax = kmax;
        jobs[t].out = out;
        jobs[t].begin = n * t / nthreads; jobs[t].end = n * (t + 1) / nthreads;
    }
    if (nthreads == 1) { aniso_job(&jobs[0]); return; }
    for (int32_t t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, aniso_job, &jobs[t]);
    for (int32_t t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------
 * Storage-format packer: writes oracle texel values into the documented
 * pool layout so stored pools can be compared byte for byte.  Texture e
 * starts at byte offset poff[e] (each texture padded to a multiple of 16
 * bytes); inside, levels follow each other, each row-major [N][N][C] of
 * the element type.  'codes' holds the reduced-precision codes (FP16/BF16
 * 2 bytes, E4M3 1 byte), else values are written as float or byte.
 * ---------------------------------------------------------------------- */
static int32_t elem_size(int32_t fmt)
{
    switch (fmt) { case ORC_F32: return 4; case ORC_U8: return 1; case ORC_F16: case ORC_BF16: return 2; }
    return 1;
}

int64_t orc_pool_offsets(int32_t E, const int32_t* log2n, int32_t C, int32_t fmt, int64_t* poff)
{
    int64_t off = 0;
    for (int32_t e = 0; e < E; ++e) {
        poff[e] = off;
        int64_t bytes = orc_texels_in_chain(log2n[e]) * C * elem_size(fmt);
        off += (bytes + 15) / 16 * 16;
    }
    poff[E] = off;
    return off;
}

void orc_pack_pool(int32_t E, const int32_t* log2n, const int64_t* toff, const int64_t* poff,
                   int32_t C, int32_t fmt, const double* tex, const uint32_t* codes, uint8_t* pool)
{
    for (int32_t e = 0; e < E; ++e) {
        int64_t cnt = (toff[e + 1] - toff[e]) * C;
        uint8_t* dst = pool + poff[e];
        memset(dst, 0, (size_t)(poff[e + 1] - poff[e]));
        for (int64_t k = 0; k < cnt; ++k) {
            int64_t s = toff[e] * C + k;
            if (fmt == ORC_F32) { float x = (float)tex[s]; memcpy(dst + 4 * k, &x, 4); }
            else if (fmt == ORC_U8) dst[k] = (uint8_t)tex[s];
            else if (fmt == ORC_E4M3) dst[k] = (uint8_t)codes[s];
            else { uint16_t x = (uint16_t)codes[s]; memcpy(dst + 2 * k, &x, 2); }
        }
    }
}

/* ------------------------------------------------------------------------
 * Alg. 1 (Section 3.1): the vertices of the intrinsic triangle of h are
 * v0 = Vert(Next h), v1 = the mean of the face's vertices (walking the
 * Next cycle from h), v2 = Vert(h).  Output [H][3][3] doubles.
 * ---------------------------------------------------------------------- */
void orc_triangle_vertices(int32_t H, const int32_t* next, const int32_t* vert, const double* pos,
                           double* tri)
{
    for (int32_t h = 0; h < H; ++h) {
        int32_t nx = next[h];
        double c[3] = {pos[3 * vert[h] + 0], pos[3 * vert[h] + 1], pos[3 * vert[h] + 2]};
        int32_t n = 1;
        for (int32_t g = nx; g != h; g = next[g]) {
            for (int k = 0; k < 3; ++k) c[k] += pos[3 * vert[g] + k];
            ++n;
        }
        for (int k = 0; k < 3; ++k) {
            tri[9 * (int64_t)h + 0 + k] = pos[3 * vert[nx] + k];
            tri[9 * (int64_t)h + 3 + k] = c[k] / n;
            tri[9 * (int64_t)h + 6 + k] = pos[3 * vert[h] + k];
        }
    }
}

/* Vertex normals for displacement along the input mesh's normals (Section
 * 5.1, displacement): each face contributes its area vector (Newell's
 * formula, half the sum of the cross products of consecutive vertices
 * around the face) to each of its vertices; the vertex normal is the
 * normalised sum.  Face centroid normal: the face's normalised area
 * vector.  Outputs [V][3] and [F][3]. */
void orc_vertex_normals(int32_t H, int32_t V, int32_t F, const int32_t* next, const int32_t* vert,
                        const int32_t* face, const double* pos, double* vn, double* fn)
{
    for (int32_t i = 0; i < 3 * V; ++i) vn[i] = 0.0;
    for (int32_t i = 0; i < 3 * F; ++i) fn[i] = 0.0;
    for (int32_t h = 0; h < H; ++h) {
        const double* a = &pos[3 * vert[h]];
        const double* b = &pos[3 * vert[next[h]]];
        double* f = &fn[3 * face[h]];
        f[0] += 0.5 * (a[1] * b[2] - a[2] * b[1]);
        f[1] += 0.5 * (a[2] * b[0] - a[0] * b[2]);
        f[2] += 0.5 * (a[0] * b[1] - a[1] * b[0]);
    }
    for (int32_t h = 0; h < H; ++h)
        for (int k = 0; k < 3; ++k) vn[3 * vert[h] + k] += fn[3 * face[h] + k];
    for (int32_t i = 0; i < V + F; ++i) {
        double* x = i < V ? &vn[3 * i] : &fn[3 * (i - V)];
        double l = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        if (l > 0) for (int k = 0; k < 3; ++k) x[k] /= l;
    }
}
