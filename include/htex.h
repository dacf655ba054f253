/*
 * htex.h — C ABI of libhtex, batched seamless filtered lookups on
 * per-halfedge textures (Htex: Barbier & Dupuy, "Per-Halfedge Texturing
 * for Arbitrary Mesh Topologies", 2022), for NVIDIA GB300 (sm_103a).
 *
 * The problem, as the paper states it: a polygon mesh given as halfedges
 * (Section 2, Fig. 2: operators Twin, Next, Prev, Vert, Edge, Face) carries
 * one square texture per edge, i.e. per intrinsic quad formed by a halfedge
 * and its twin (Section 3.2, Section 4.3).  A query names a halfedge h and
 * barycentric coordinates (u, v) on the intrinsic triangle of h (Section
 * 4.2); its value blends three border-normalised fetches: the quad of h at
 * (u, v), the quad of Next(h) at (v, -u) and the quad of Prev(h) at (-v, u),
 * each mapped by Alg. 2 (Alg. 3).
 *
 * Conventions for every call:
 *   - Return values are htex_status codes; no call throws or aborts.
 *     Argument errors are reported synchronously, before any device work.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the current device (e.g. torch.Tensor.data_ptr()).
 *   - The library owns the memory behind htex_mesh and htex_textures and
 *     frees it in the matching *_destroy call.  The caller owns every
 *     buffer it passes in.
 *   - Device work is asynchronous on the given stream (NULL = the legacy
 *     default stream) unless the call says it synchronises.
 *   - A htex_stream is a cudaStream_t (the same handle type), spelled
 *     without CUDA headers.
 *   - Per-query problems (h out of range, u or v not finite) do not fail a
 *     call: that query's outputs are NaN and, when a device status word is
 *     given, it is incremented once per such query.
 */
#ifndef HTEX_H
#define HTEX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HTEX_OK = 0,
    HTEX_ERR_INVALID_ARG = 1,        /* null pointer, bad size, bad enum value        */
    HTEX_ERR_NONMANIFOLD = 2,        /* a directed edge used twice, or twins disagree */
    HTEX_ERR_BAD_TEXTURE = 3,        /* resolution not 2^n with 0 <= n <= 13, etc.    */
    HTEX_ERR_OUT_OF_MEMORY = 4,      /* host or device allocation refused             */
    HTEX_ERR_CUDA = 5,               /* a CUDA runtime call failed                    */
    HTEX_ERR_QUERY_OUT_OF_RANGE = 6, /* reserved: per-query errors use the status word */
    HTEX_ERR_TIMEOUT = 7,            /* a bounded host wait ran out                   */
    HTEX_ERR_UNSUPPORTED = 8         /* valid request this build cannot serve         */
} htex_status;

/* Texel storage formats.  Every format is filtered in FP32.
 *   HTEX_F32   IEEE binary32 per channel.
 *   HTEX_U8    8-bit UNORM per channel: byte b stands for b / 255.
 *   HTEX_F16   IEEE binary16 code c stands for c * scale_e.
 *   HTEX_BF16  bfloat16 code c stands for c * scale_e.
 *   HTEX_E4M3  OCP FP8 E4M3 (no infinities, saturating at 448) code c
 *              stands for c * scale_e.
 * scale_e is one FP32 number per texture: max|T| / 448 for E4M3, max|T|
 * for F16/BF16 (over every stored level of texture e; 1 when the texture
 * is all zero).  Codes are T / scale_e rounded to nearest, ties to even. */
typedef enum { HTEX_F32 = 0, HTEX_U8 = 1, HTEX_F16 = 2, HTEX_BF16 = 3, HTEX_E4M3 = 4 } htex_dtype;

/* Texture preparation flags (htex_textures_prepare / _upload). */
#define HTEX_BUILD_MIPS      1u  /* build every coarser level from level 0 by 2x2 box means   */
#define HTEX_MIRROR_BOUNDARY 2u  /* fill the unused half of boundary textures (Section 4.3)  */
#define HTEX_FIX_CORNERS     4u  /* corner pre-processing (Section 4.4)                      */
#define HTEX_LEVELS_GIVEN    8u  /* the caller supplies every level, not only level 0        */

/* Lookup flags (htex_lookup / _backward). */
#define HTEX_LOOKUP_BIN      1u  /* sort queries by halfedge range before filtering (scratch) */
#define HTEX_LOOKUP_GLOBAL   2u  /* never stage textures in shared memory                     */

/* One query: 16 bytes, 16-byte aligned in device memory.
 *   h          halfedge id, 0 <= h < H
 *   u, v       barycentrics on the intrinsic triangle of h (Section 4.2):
 *              u weighs Vert(h), v weighs Vert(Next(h)), 1 - u - v the
 *              face centroid.  Finite values off the closed triangle are
 *              clamped onto it (negatives to 0, then scaled onto u + v = 1).
 *   footprint  isotropic filter width in quad-uv units: level selection
 *              lambda = log2(footprint * N_e) per fetched texture; level 0
 *              when lambda is not > 0 (footprint <= 0 or NaN included), the
 *              1x1 level when floor(lambda) reaches it, else levels
 *              floor(lambda) and floor(lambda) + 1 blended linearly. */
typedef struct {
    int32_t h;
    float u, v, footprint;
} htex_query;

/* One anisotropic query: 32 bytes, 16-byte aligned in device memory.
 *   h, u, v     as in htex_query
 *   pad         ignored
 *   dudx, dvdx  derivatives of (u, v) along screen x (quad-uv units per
 *               pixel), dudy, dvdy along screen y: the footprint whose
 *               longer axis the probes of htex_lookup_aniso follow. */
typedef struct {
    int32_t h;
    float u, v, pad;
    float dudx, dvdx, dudy, dvdy;
} htex_query_aniso;

typedef struct CUstream_st* htex_stream;

typedef struct htex_mesh htex_mesh;          /* host-side halfedge mesh (opaque)        */
typedef struct htex_textures htex_textures;  /* device-resident mesh + textures (opaque) */

/* Human-readable name of a status code (static string). */
const char* htex_status_string(htex_status s);

/* ---------------------------------------------------------------- meshes */

/* Build the halfedge mesh of a polygon mesh (Section 2, Fig. 2; Section 3).
 *   face_sizes  host [num_faces], each >= 3
 *   face_verts  host [sum(face_sizes)], vertex ids in [0, num_verts), each
 *               face's vertices in order (consistent orientation)
 * The halfedges of face f are contiguous in the face's vertex order:
 * Next/Prev cycle within the face, Vert(h) is the origin vertex of h,
 * Face(h) = f.  Twin(h) is the halfedge running the other way, -1 on the
 * boundary.  Edge ids: scanning h = 0..H-1, a new id whenever Twin(h) < 0
 * or h < Twin(h), shared with the twin; so E = (H + boundary halfedges)/2.
 * Host-only (no GPU needed).  Errors: HTEX_ERR_INVALID_ARG (face smaller
 * than 3, vertex id out of range, an edge from a vertex to itself),
 * HTEX_ERR_NONMANIFOLD (a directed edge used by two faces). */
htex_status htex_mesh_create(const int32_t* face_sizes, int32_t num_faces,
                             const int32_t* face_verts, int32_t num_verts, htex_mesh** out);

/* Adopt explicit halfedge arrays (host, each [H]), e.g. the Fig. 2 table.
 * Validated: Next/Prev mutually inverse with cycles of length >= 3, Twin an
 * involution without fixed points running the opposite way
 * (Vert(Twin h) = Vert(Next h)), Face constant along Next cycles, Edge a
 * twin-consistent bijection of halfedge pairs (and boundary halfedges)
 * onto [0, E).  Host-only.  Errors: HTEX_ERR_INVALID_ARG,
 * HTEX_ERR_NONMANIFOLD. */
htex_status htex_mesh_create_from_halfedges(const int32_t* twin, const int32_t* next,
                                            const int32_t* prev, const int32_t* vert,
                                            const int32_t* edge, const int32_t* face, int32_t H,
                                            int32_t num_verts, int32_t num_faces,
                                            htex_mesh** out);

/* Sizes of a mesh; each output pointer is nullable. */
htex_status htex_mesh_info(const htex_mesh* m, int32_t* H, int32_t* E, int32_t* num_boundary,
                           int32_t* num_verts, int32_t* num_faces);

/* Copy the six halfedge operators to host arrays of H int32 (each nullable). */
htex_status htex_mesh_get_halfedges(const htex_mesh* m, int32_t* twin, int32_t* next,
                                    int32_t* prev, int32_t* vert, int32_t* edge, int32_t* face);

void htex_mesh_destroy(htex_mesh* m);

/* -------------------------------------------------------------- textures */

/* Pool layout (Section 4.3: one square texture per edge, each sized
 * independently).  Texture e has resolution N_e = 2^log2_res[e] and
 * log2_res[e] + 1 levels N_e, N_e/2, ..., 1.  In the pool, texture e starts
 * at byte offset texture_offsets[e] (textures in edge order, each padded to
 * a multiple of 16 bytes); its levels follow one another; level l is
 * row-major [N_l][N_l][channels] of the element type, texel (i, j) being
 * column i along quad x and row j along quad y, at element
 * (j * N_l + i) * channels.  Texel centres sit at ((i+1/2)/N_l, (j+1/2)/N_l).
 * Element sizes: F32 4, U8 1, F16/BF16 2, E4M3 1 bytes.
 *   log2_res         host [E], each in [0, 13] (up to 8192 x 8192 texels)
 *   pool_bytes       out: total bytes
 *   texture_offsets  out, nullable: host [E + 1] byte offsets
 * Host-only. */
htex_status htex_textures_layout(const htex_mesh* m, int32_t channels, htex_dtype dtype,
                                 const int32_t* log2_res, int64_t* pool_bytes,
                                 int64_t* texture_offsets);

/* Prepare the stored pool on the host, without a GPU.
 *   texels  host; for HTEX_F32/F16/BF16/E4M3 float32 values, for HTEX_U8
 *           bytes; per edge in edge order, each row-major [N][N][channels];
 *           level 0 only, or every level (HTEX_LEVELS_GIVEN) in pool order.
 *   flags   HTEX_BUILD_MIPS (required unless HTEX_LEVELS_GIVEN),
 *           HTEX_MIRROR_BOUNDARY, HTEX_FIX_CORNERS, HTEX_LEVELS_GIVEN.
 * Steps, in this order: with BUILD_MIPS and MIRROR_BOUNDARY level 0 of every
 * boundary texture is mirrored first; mips: level l+1 texel (i, j) =
 * ((a + b) + c) + d over the 2x2 block (2i, 2j), (2i+1, 2j), (2i, 2j+1),
 * (2i+1, 2j+1), times 1/4, evaluated in double and rounded once to float
 * (U8: (a + b + c + d + 2) >> 2); MIRROR_BOUNDARY: every level of a boundary
 * texture takes, at texel (i, j) with i + j > N - 1, the value of
 * (N-1-j, N-1-i) (reflection across the quad diagonal, where the virtual
 * twin lies, Section 3.2); FIX_CORNERS: for every resolution R, the corner
 * texels meeting at one mesh vertex or face centroid take their group's
 * mean (double, rounded to float; U8: round half up), groups joined where
 * one texel is several corners (R = 1); quantisation to F16/BF16/E4M3 with
 * the per-texture scale (see htex_dtype).
 *   pool_out    host [pool_bytes] (see htex_textures_layout)
 *   scales_out  host [E] float, nullable (1 for F32 and U8)
 * Errors: HTEX_ERR_INVALID_ARG, HTEX_ERR_BAD_TEXTURE, HTEX_ERR_OUT_OF_MEMORY. */
htex_status htex_textures_prepare(const htex_mesh* m, int32_t channels, htex_dtype dtype,
                                  const int32_t* log2_res, const void* texels, uint32_t flags,
                                  void* pool_out, float* scales_out);

/* Prepare (as htex_textures_prepare) and make the mesh and its textures
 * resident on the current device.  Allocates device memory owned by the
 * returned object; copies on 'stream' and synchronises it before
 * returning.  Refuses with HTEX_ERR_OUT_OF_MEMORY, before allocating,
 * when the device does not have room. */
htex_status htex_textures_upload(const htex_mesh* m, int32_t channels, htex_dtype dtype,
                                 const int32_t* log2_res, const void* texels, uint32_t flags,
                                 htex_stream stream, htex_textures** out);

/* Same as htex_textures_upload with HTEX_LEVELS_GIVEN: 'texels' holds every
 * level of every texture (pool order, no padding). */
htex_status htex_textures_upload_levels(const htex_mesh* m, int32_t channels, htex_dtype dtype,
                                        const int32_t* log2_res, const void* texels,
                                        uint32_t flags, htex_stream stream, htex_textures** out);

/* Make an already prepared pool resident (bytes as htex_textures_prepare
 * writes them; scales [E] nullable for F32/U8).  Synchronises 'stream'. */
htex_status htex_textures_upload_pool(const htex_mesh* m, int32_t channels, htex_dtype dtype,
                                      const int32_t* log2_res, const void* pool,
                                      const float* scales, htex_stream stream,
                                      htex_textures** out);

/* Sizes of resident textures; each output pointer is nullable.
 * device_bytes counts every device allocation the object holds. */
htex_status htex_textures_info(const htex_textures* t, int32_t* channels, htex_dtype* dtype,
                               int32_t* H, int32_t* E, int64_t* pool_bytes,
                               int64_t* device_bytes);

/* Copy the resident pool (and scales, nullable) back to the host;
 * synchronises 'stream'. */
htex_status htex_textures_download_pool(const htex_textures* t, void* pool, float* scales,
                                        htex_stream stream);

/* Overwrite 'bytes' bytes of the resident pool at byte 'offset' with 'src'
 * (host or device memory), asynchronously on 'stream': in-place texel
 * edits, e.g. the updates of a texture fit.  The bytes are stored values in
 * the pool layout (for scaled formats, codes; the scales are unchanged).
 * HTEX_ERR_INVALID_ARG if the range leaves the pool.  'src' must stay valid
 * until 'stream' reaches the copy. */
htex_status htex_textures_write_pool(const htex_textures* t, int64_t offset, int64_t bytes,
                                     const void* src, htex_stream stream);

void htex_textures_destroy(htex_textures* t);

/* ---------------------------------------------------------------- lookups */

/* Filtered lookups (Section 4.4, Alg. 3 with Alg. 2), n queries.
 *   q         device [n] htex_query (16-byte aligned)
 *   out       device [n][channels] float (16-byte aligned when channels = 4)
 *   flags     HTEX_LOOKUP_BIN: when the pool exceeds 64 MiB, counting-sort
 *             the queries into ranges of consecutive halfedges first, in
 *             chunks of 2^24 queries, filter them in that order and gather
 *             the results back into query order (same results, bit for bit;
 *             scratch of 20 + 4 * channels bytes per chunk query,
 *             allocated stream-ordered on 'stream' from a library-owned
 *             pool and released there; HTEX_ERR_OUT_OF_MEMORY when it cannot
 *             be had); HTEX_LOOKUP_GLOBAL: never stage the pool in shared
 *             memory (by default a pool of at most 96 KiB is staged)
 *   d_status  device int32, nullable: incremented once per invalid query
 * For each query: own = quad of Edge(h) at Alg. 2 (h, (u, v)), then the
 * quads of Next(h) at (v, -u) and of Prev(h) at (-v, u); each fetch is a
 * bilinear (or trilinear, see htex_query) sample with zero border whose
 * in-bounds weights form the normalisation sum (the border-normalisation
 * channel of Section 4.4, computed instead of stored); the result is the
 * data sum over the three fetches divided by the weight sum.  Accumulates
 * in FP32.  n = 0 is valid and launches nothing.  Asynchronous. */
htex_status htex_lookup(const htex_textures* t, const htex_query* q, int64_t n, float* out,
                        uint32_t flags, htex_stream stream, int32_t* d_status);

/* Anisotropic filtered lookups, n queries.  Section 5.1 renders Htex with
 * the GPU's anisotropic filter applied to each of Alg. 3's three fetches;
 * the paper states no formula, so this is one reading of it:
 *   px2 = |(dudx, dvdx)|^2, py2 = |(dudy, dvdy)|^2 (float); the major axis
 *   m is the y derivative when py2 > px2, else the x derivative; the probe
 *   count K = 1 when both are zero, else min(ceil(sqrt(max / min)),
 *   max_aniso); each probe is a trilinear sample with footprint Pmax / K
 *   (Pmax = sqrt(max), the level rule of htex_query); probe k sits at
 *   (u, v) + m s ((k + 1/2) / K - 1/2) with s = min(1, K / Pmax), and
 *   samples all three fetches there (own quad at (u', v'), Next's at
 *   (v', -u'), Prev's at (-v', u'), through Alg. 2, zero border); the result
 *   is the summed data over the summed normalisation weight.  (u, v) is
 *   clamped onto the triangle as in htex_lookup before the probes are
 *   placed.
 *   q          device [n] htex_query_aniso (16-byte aligned)
 *   max_aniso  1..16
 *   flags      HTEX_LOOKUP_BIN: sort the queries by halfedge range first,
 *              as htex_lookup does (same results, bit for bit: each
 *              query's probes are summed in probe order whatever queries
 *              share its warp; scratch of 36 + 4 * channels bytes per
 *              chunk query)
 *   out        device [n][channels] float (alignment as htex_lookup)
 *   d_status   device int32, nullable: incremented once per invalid query
 *              (h out of range, non-finite u, v or derivative, or an
 *              overflowing squared length); such a query gives NaN.
 * FP32 accumulation over at most 24 * max_aniso taps.  Asynchronous. */
htex_status htex_lookup_aniso(const htex_textures* t, const htex_query_aniso* q, int64_t n, int32_t max_aniso,
                              uint32_t flags, float* out, htex_stream stream, int32_t* d_status);

/* The two halves of HTEX_LOOKUP_BIN as calls of their own, for callers
 * that filter one sorted batch more than once (several texture sets on
 * one mesh) or time the filter on its own.  The paper has no counterpart:
 * query order does not change any result (each query is filtered on its
 * own, Section 4.4, Alg. 3), only which texels share L2 at a time.
 *
 * htex_queries_sort: counting-sorts the queries, within consecutive chunks
 * of 2^24, into ranges of consecutive halfedges (at most 128 ranges of
 * 2^s halfedges, the ranges in ascending order, invalid queries last in
 * their chunk; the order inside a range is unspecified and may differ
 * from call to call).
 *   q        device [n] htex_query, 16-byte aligned, n <= 2^31 - 1
 *   sorted   device [n] htex_query, 16-byte aligned, must not overlap q:
 *            the queries in sorted order, each unchanged
 *   pos      device [n] int32: pos[i] = index in 'sorted' of query i
 * Only t's halfedge count is used.  Needs a few KiB of scratch, allocated
 * stream-ordered from a library-owned pool (HTEX_ERR_OUT_OF_MEMORY when it
 * cannot be had).  Asynchronous on 'stream'. */
htex_status htex_queries_sort(const htex_textures* t, const htex_query* q, int64_t n, htex_query* sorted,
                              int32_t* pos, htex_stream stream);

/* htex_results_gather: out[i][c] = sorted_out[pos[i]][c] for i < n,
 * c < channels: the results of htex_lookup on htex_queries_sort's sorted
 * copy, back in query order.  A pos[i] outside [0, n) gives NaN in every
 * channel of out[i] and reads nothing.
 *   sorted_out, out  device float [n][channels], channels 1..4, aligned
 *                    to 16 bytes (channels 4), 8 (2) or 4 (1, 3); must not
 *                    overlap
 *   pos              device int32 [n]
 * Runs on the current device.  Asynchronous on 'stream'. */
htex_status htex_results_gather(const float* sorted_out, const int32_t* pos, int64_t n, int32_t channels,
                                float* out, htex_stream stream);

/* htex_lookup on host buffers (the end-to-end path for callers whose
 * queries and results live in host memory).
 *   q    host [n] htex_query;  out  host [n][channels] float
 * When both buffers are page-locked and mapped into the device's address
 * space (cudaHostAlloc, torch pin_memory, cudaHostRegister with mapping)
 * and aligned as htex_lookup requires, the lookup kernels read the queries
 * and write the results across the link in place, in one pass
 * (HTEX_LOOKUP_BIN is then ignored: its sort would read the queries across
 * the link twice more).  Otherwise the queries go to the device and the
 * results come back in chunks of 2,097,152, each chunk on one of three
 * library-owned streams, so that the copy in of one chunk, the lookup of
 * another and the copy out of a third overlap; pageable buffers give the
 * same results, without overlap.  The first call on a textures object creates its streams and
 * about 200 MB of device staging (freed by htex_textures_destroy; returns
 * HTEX_ERR_OUT_OF_MEMORY if that fails).  Ordered after earlier work on
 * 'stream' and asynchronous: 'out' is complete once 'stream' is; 'q' and
 * 'out' must stay valid until then.  Calls on one textures object are
 * serialised on its internal streams.  Flags and d_status as htex_lookup. */
htex_status htex_lookup_host(const htex_textures* t, const htex_query* q, int64_t n, float* out,
                             uint32_t flags, htex_stream stream, int32_t* d_status);

/* Gradient of L = sum_q sum_c grad_out[q][c] * lookup(q)[c] with respect to
 * every stored texel value (the decoded value T = code * scale for scaled
 * formats).  The lookup is linear in the texels, so each in-bounds tap k
 * of query q receives grad_out[q][c] * w_k / W_q with the forward weights.
 *   grad_out     device [n][channels] float
 *   grad_texels  device float, one per pool element (pool_bytes / element
 *                size), same element order as the pool; accumulated into
 *                (the caller zeroes it); padding elements keep their values
 *   flags        HTEX_LOOKUP_BIN: when the pool exceeds 64 MiB, sort the
 *                queries as htex_lookup does (chunks of 2^24, ranges of
 *                consecutive halfedges; grad_out rows move with their
 *                queries) so that the threads resident together add into
 *                a narrow range of textures; lanes of a warp whose taps
 *                coincide (the same texture, level and 2x2 block or edge
 *                texel pair) sum their contributions across the warp and
 *                one lane issues the atomics.  Scratch of 16 + 4 * channels
 *                bytes per chunk query from the library pool.
 *                HTEX_LOOKUP_GLOBAL ignored.
 *   d_status     as for htex_lookup
 * Uses float atomics; per three-channel texel, when grad_texels is 16-byte
 * aligned, one four-float atomic if its three values share a 16-byte block
 * (adding +0.0 to the block's fourth element, which keeps its value; -0.0
 * there becomes +0.0), else a float2 and a scalar one (also when only
 * 8-byte aligned), else three scalar ones.  The summation order, hence the
 * last bits, may vary from run to run.  Asynchronous. */
htex_status htex_lookup_backward(const htex_textures* t, const htex_query* q, int64_t n,
                                 const float* grad_out, float* grad_texels, uint32_t flags,
                                 htex_stream stream, int32_t* d_status);

/* One Adam step on the texels of an FP32 asset, for fitting textures from
 * the gradients of htex_lookup_backward (no counterpart in the paper).  Per
 * element, with t = step:
 *   m = beta1 m + (1 - beta1) g;  v = beta2 v + (1 - beta2) g^2;
 *   master -= (lr / (1 - beta1^t)) m / (sqrt(v) / sqrt(1 - beta2^t) + eps)
 * then the new value is written into the resident pool (the next lookup
 * sees it) and g is set to 0 (ready for the next accumulation).
 *   master, grad, m, v  device float [n], 16-byte aligned, n = pool_bytes
 *                       / 4 (pool element order, as htex_lookup_backward);
 *                       master nullable: NULL optimises the pool's own
 *                       values in place (an FP32 pool holds them exactly;
 *                       one read and one write of n floats fewer)
 *   step                >= 1; beta1, beta2 in [0, 1); eps > 0
 * HTEX_ERR_INVALID_ARG for other formats or sizes.  Asynchronous. */
htex_status htex_textures_adam_step(htex_textures* t, float* master, float* grad, float* m, float* v, int64_t n,
                                    float lr, float beta1, float beta2, float eps, int32_t step,
                                    htex_stream stream);

/* -------------------------------------------------------------- rendering */

/* The step before the lookup in the paper's pipeline (Section 4.4,
 * "Rendering": one triangle per halfedge is drawn and each fragment samples
 * the Htex at its (halfedge, barycentrics)), as CUDA kernels. */
typedef struct htex_geometry htex_geometry;

/* Device geometry of a mesh: its Next/Vert/Face operators, vertex
 * positions (host [V][3] float, copied) and the normals of the input mesh
 * (per face its area vector by Newell's formula, per vertex the normalised
 * sum of its faces' vectors), computed on the host.  Synchronises stream. */
htex_status htex_geometry_create(const htex_mesh* m, const float* positions, htex_stream stream,
                                 htex_geometry** out);
void htex_geometry_destroy(htex_geometry* g);

/* Alg. 1 (Section 3.1) for every halfedge h: out (device [H][3][3] float)
 * receives v0 = Vert(Next h), v1 = the mean of the vertices of Face(h),
 * v2 = Vert(h).  Asynchronous. */
htex_status htex_triangle_vertices(const htex_geometry* g, float* out, htex_stream stream);

/* Render the intrinsic triangulation (every halfedge's Alg. 1 triangle)
 * into a query per pixel.
 *   view_proj  host float[16], row-major: clip = view_proj * (x, y, z, 1);
 *              NDC x right, y up, depth z/w visible in [-1, 1]; pixel
 *              (x, y), y down, has its centre at (x + 1/2, y + 1/2)
 *   queries    device [height][width] htex_query (16-byte aligned): the
 *              nearest triangle whose closed interior contains the pixel
 *              centre (ties to the smaller halfedge), its perspective-
 *              correct barycentrics (u weighs Vert(h), v Vert(Next h),
 *              Section 4.2) and footprint max(|d(u,v)/dx|, |d(u,v)/dy|)
 *              per pixel; h = -1 (an invalid query) where nothing is seen
 *   depth      device [height][width] float, nullable: NDC depth (NaN if empty)
 * Triangles with a vertex at or behind the camera plane (w <= 0) are not
 * drawn.  Scratch (8 bytes per pixel) comes stream-ordered from a
 * library-owned pool.  Asynchronous. */
htex_status htex_rasterize(const htex_geometry* g, const float* view_proj, int32_t width, int32_t height,
                           htex_query* queries, float* depth, htex_stream stream);

/* htex_rasterize for anisotropic filtering: the same pixels, triangles and
 * barycentrics, written as htex_query_aniso (32 bytes, 16-byte aligned)
 * whose derivatives are the differences of the barycentrics at the centres
 * one pixel right (du/dx, dv/dx) and one pixel down (du/dy, dv/dy) in the
 * same triangle; h = -1 and zero derivatives where nothing is seen.  For
 * htex_lookup_aniso. */
htex_status htex_rasterize_aniso(const htex_geometry* g, const float* view_proj, int32_t width, int32_t height,
                                 htex_query_aniso* queries, float* depth, htex_stream stream);

/* Displacement (Section 5.1): for every halfedge triangle the lattice
 * (u, v) = (i/T, j/T), i + j <= T (k = 0.. in order of i, then j), is
 * moved along the interpolated normal of the input mesh (vertex normals at
 * Vert(h) and Vert(Next h), the face normal at the centroid) by scale times
 * channel 'channel' of the level-0 lookup at (h, u, v).
 *   t     textures of the same mesh;  tess  T in [1, 64]
 *   out   device [H][(T+1)(T+2)/2][3] float
 * Asynchronous; scratch as htex_rasterize. */
htex_status htex_displace(const htex_geometry* g, const htex_textures* t, int32_t tess, float scale,
                          int32_t channel, float* out, htex_stream stream);

/* ---------------------------------------------------------------- serving */

/* A lookup server: many assets kept resident under a device-memory budget
 * and requests of uneven sizes from different assets served by continuous
 * batching.  The paper renders one asset per frame; this serves the same
 * per-query computation (Alg. 3) to a stream of requests.  A scheduler
 * thread owned by the server
 *   - admits a request when its asset is resident, and a small request
 *     (at most 65,536 queries) at once: while its asset is not resident
 *     (or still uploading) its batches read the asset's page-locked host
 *     copy across the CPU-GPU link (same kernel, same bytes, so the same
 *     results); larger requests wait for the upload;
 *   - uploads the assets that unfinished requests need, most requested
 *     first, as far as the budget allows after evicting the least recently
 *     used assets that no unfinished request needs;
 *   - fills each free batch slot from the admitted requests, shortest
 *     remaining work first with ageing (the remaining query count is
 *     divided by 1 + wait / 1 ms, so small requests overtake large ones
 *     and a waiting request keeps moving forward), at most request_chunk
 *     queries of one request per batch, so a request that arrives while
 *     others run joins the next batch;
 *   - launches a batch as an instantiated CUDA graph (descriptor table
 *     copy, then one persistent kernel per texel format pulling 4096-query
 *     tiles of any request), with the query and result copies around it.
 * Results are those htex_lookup gives for the same queries (each query is
 * computed by the same code, whatever shares its batch).
 * Buffers: queries and results live in host memory (page-locked for copy
 * speed) and must stay valid until the request completes. */
typedef struct htex_server htex_server;

typedef struct {
    int64_t budget_bytes;   /* device bytes for resident assets                    */
    int64_t batch_queries;  /* queries per batch (staging per slot: 32 B x this)   */
    int32_t batch_slots;    /* batches in flight, 1..8                             */
    int32_t max_items;      /* request chunks per batch, 1..256                    */
    int64_t request_chunk;  /* most queries of one request in one batch            */
} htex_server_config;

typedef struct {
    int64_t completed;       /* requests completed                  */
    int64_t queries;         /* queries launched                    */
    int64_t batches;         /* batches launched                    */
    int64_t uploads;         /* asset uploads (admissions)          */
    int64_t evictions;       /* assets evicted to make room         */
    int64_t resident_bytes;  /* device bytes of resident assets now */
    int64_t host_queries;    /* queries served from an asset's host copy */
} htex_server_stats;

/* Create a server on the current device (allocates its staging, streams
 * and graphs' buffers, starts its thread). */
htex_status htex_server_create(const htex_server_config* cfg, htex_server** out);

/* Register an asset from a prepared pool (htex_textures_prepare layout;
 * scales required for scaled formats).  The pool is copied into page-locked
 * host memory owned by the server; the asset becomes resident on demand.
 * HTEX_ERR_OUT_OF_MEMORY if it alone exceeds the budget.  The host copy
 * (records, headers, scales and pool) is page-locked and mapped, so
 * requests can be served from it before the asset is resident. */
htex_status htex_server_add_asset(htex_server* s, const htex_mesh* m, int32_t channels, htex_dtype dtype,
                                  const int32_t* log2_res, const void* pool, const float* scales,
                                  int32_t* asset_id);

/* Queue n queries (host) against an asset; results go to out (host,
 * [n][channels] float).  Returns at once with the request's id.  When q
 * and out are page-locked, mapped into the device's address space and
 * 16-byte aligned, the batches read and write them in place; otherwise
 * they are copied through the server's device staging.  Either way the
 * buffers must stay valid until the request completes. */
htex_status htex_server_submit(htex_server* s, int32_t asset_id, const htex_query* q, int64_t n,
                               float* out, int64_t* request_id);

/* Take up to 'capacity' completed requests: their ids and latencies in
 * seconds (submission to observed completion).  Returns the server's
 * sticky error, if any. */
htex_status htex_server_poll(htex_server* s, int64_t* ids, double* latency_s, int32_t capacity,
                             int32_t* count);

/* Wait until every submitted request has completed, at most timeout_s
 * seconds (HTEX_ERR_TIMEOUT when the wait runs out). */
htex_status htex_server_drain(htex_server* s, double timeout_s);

htex_status htex_server_get_stats(htex_server* s, htex_server_stats* st);

/* Stop the thread, wait for the device work and free everything. */
void htex_server_destroy(htex_server* s);

/* ------------------------------------------------- allocation-free lookup */

/* The paper has no counterpart to this call: it serves callers that must
 * not allocate device memory.  Such callers include host applications or
 * engines that own every device allocation and forbid the libraries they
 * load to make their own, and frame loops that cannot absorb the
 * device-wide synchronisation that cudaMalloc and cudaFree may cause.
 *
 * htex_lookup_noalloc returns what htex_lookup with HTEX_LOOKUP_BIN
 * returns for the same arguments, bit for bit (the same per-query filter
 * code; only the order in which the queries are filtered differs), without
 * any allocation: its scratch (the reordered queries, their original
 * indices and the bucket counters) is one fixed device array inside the
 * library, about 20 MiB, which every device that loads the library holds
 * until the process exits.
 *   n         at most htex_lookup_noalloc_max_queries() (1,048,576);
 *             larger n returns HTEX_ERR_UNSUPPORTED before any device work
 * The first call made with a given device current looks up the array's
 * device address (cudaGetSymbolAddress) and keeps it for the rest of the
 * process; make that first call before any stream capture, and do not use
 * this entry point again after cudaDeviceReset (the module, and with it
 * the array, may then live at another address).  Every call on every stream shares the one array and the
 * array keeps the previous call's contents (the call clears its counters
 * itself), so calls whose device work overlaps (different streams without
 * ordering between them) race and must not be issued.  The textures must
 * live on the current device (HTEX_ERR_INVALID_ARG otherwise).
 * Asynchronous on 'stream'. */
htex_status htex_lookup_noalloc(const htex_textures* t, const htex_query* q, int64_t n, float* out,
                                htex_stream stream, int32_t* d_status);

/* Largest query count htex_lookup_noalloc accepts. */
int64_t htex_lookup_noalloc_max_queries(void);

#ifdef __cplusplus
}
#endif

#endif /* HTEX_H */
