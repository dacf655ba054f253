"""Oracle pins: filtered lookup (paper Section 4.4, Alg. 3 with Alg. 2).

The paper prints no lookup values, so the pins are values derived by hand
from the algorithms, an independent brute-force evaluation (tent weights
summed over every texel), a library bilinear interpolator, and properties
the paper states: three fetches blend seamlessly across shared edges, and
with corner pre-processing around every vertex and face centroid.
"""
import math

import numpy as np
import pytest
from scipy import ndimage

import htex_synth as syn
import oracle

F32 = oracle.BUILD_MIPS


def _tex_1x1(mesh, values):
    vals = np.asarray(values, np.float32).reshape(-1)
    return oracle.prepare_textures(mesh, np.zeros(mesh.num_edges, np.int32), vals, 1, "f32", F32)


def _q(h, u, v, f=0.0):
    return (np.array([h], np.int32), np.array([u]), np.array([v]), np.array([f]))


# ---------------------------------------------------------------- hand values

def test_hand_value_single_quad():
    """One quad, 4 boundary halfedges, 1x1 textures T_e = 1, 10, 100, 1000.

    At (u, v) = (1/4, 1/4) the 1-D in-bounds weight of a 1x1 texture is
    1/2 + x on [0, 1/2] and 3/2 - x on [1/2, 1]; own (1/4, 1/4): 0.5625,
    Next at (1/4, -1/4): 0.1875, Prev at (-1/4, 1/4): 0.1875, so the blend is
    0.6 T_own + 0.2 T_next + 0.2 T_prev."""
    m = oracle.mesh_from_faces(*syn.single_quad())
    assert list(m.edge) == [0, 1, 2, 3]
    t = _tex_1x1(m, [1, 10, 100, 1000])
    out, w = oracle.lookup(m, t, _q(0, 0.25, 0.25), return_weight=True)
    assert out[0, 0] == pytest.approx(202.6, abs=1e-12)
    assert w[0] == pytest.approx(0.9375, abs=1e-15)
    out = oracle.lookup(m, t, _q(1, 0.25, 0.25))
    assert out[0, 0] == pytest.approx(0.6 * 10 + 0.2 * 100 + 0.2 * 1, abs=1e-12)


def test_hand_values_fig2(fig2_table):
    """Fig. 2 mesh with the paper's own edge ids, 1x1 textures T_e = 2^e.

    h7 (no flips): 0.6 T_e4 + 0.2 T_e5 + 0.2 T_e8.  h1 is the smaller id of
    its pair, so its own fetch flips to (3/4, 3/4); Prev(h1) = h0 also flips,
    to (5/4, 3/4): 0.6 T_e4 + 0.2 T_e0 + 0.2 T_e3.  At (1/2, 1/2) both sides
    of the diagonal give T_e4."""
    t = fig2_table
    m = oracle.mesh_from_halfedges(t["Twin"], t["Next"], t["Prev"], t["Vert"], t["Edge"],
                                   t["Face"], 7, 3)
    T = [2.0 ** e for e in range(9)]
    tex = _tex_1x1(m, T)
    o = oracle.lookup(m, tex, _q(7, 0.25, 0.25))[0, 0]
    assert o == pytest.approx(0.6 * T[4] + 0.2 * T[5] + 0.2 * T[8], abs=1e-12)
    o = oracle.lookup(m, tex, _q(1, 0.25, 0.25))[0, 0]
    assert o == pytest.approx(0.6 * T[4] + 0.2 * T[0] + 0.2 * T[3], abs=1e-12)
    for h in (7, 1):
        assert oracle.lookup(m, tex, _q(h, 0.5, 0.5))[0, 0] == pytest.approx(T[4], abs=1e-12)


def test_hand_value_face_centroid_without_corner_fix():
    """Centroid of the single quad: h0 gives (T0 + T1 + T3) / 3, h1 gives
    (T1 + T2 + T0) / 3, so without corner pre-processing the centroid is a
    discontinuity (Section 4.4, corner pre-processing)."""
    m = oracle.mesh_from_faces(*syn.single_quad())
    T = [1.0, 10.0, 100.0, 1000.0]
    t = _tex_1x1(m, T)
    assert oracle.lookup(m, t, _q(0, 0.0, 0.0))[0, 0] == pytest.approx((T[0] + T[1] + T[3]) / 3)
    assert oracle.lookup(m, t, _q(1, 0.0, 0.0))[0, 0] == pytest.approx((T[1] + T[2] + T[0]) / 3)


def test_hand_value_lod_last_level():
    """2x2 textures, footprint 1: lambda = log2(1 * 2) = 1 reaches the last
    level, the 1x1 mip (the mean of the four texels), so the blend is the
    1x1 hand value with the means."""
    m = oracle.mesh_from_faces(*syn.single_quad())
    rng = np.random.default_rng(5)
    lvl0 = rng.random((4, 2, 2, 1)).astype(np.float32)
    t = oracle.prepare_textures(m, np.ones(4, np.int32), lvl0.reshape(-1), 1, "f32", F32)
    mean = lvl0.astype(np.float64).mean(axis=(1, 2, 3))
    o = oracle.lookup(m, t, _q(0, 0.25, 0.25, 1.0))[0, 0]
    assert o == pytest.approx(0.6 * mean[0] + 0.2 * mean[1] + 0.2 * mean[3], abs=1e-7)
    # footprint 1/2: lambda = 0, level 0 only; (1/4, 1/4) is texel (0, 0)'s
    # centre and the neighbours' taps carry zero weight
    o = oracle.lookup(m, t, _q(0, 0.25, 0.25, 0.5))[0, 0]
    assert o == pytest.approx(float(lvl0[0, 0, 0, 0]), abs=1e-12)


def test_hand_value_trilinear_blend():
    """2x2 textures, lambda between 0 and 1: level 0 (own texel (0, 0) with
    weight 1 at (1/4, 1/4)) and level 1 (the 1x1 hand weights) blend with
    1 - phi and phi, in both the data and the normalisation sums."""
    m = oracle.mesh_from_faces(*syn.single_quad())
    rng = np.random.default_rng(6)
    lvl0 = rng.random((4, 2, 2, 1)).astype(np.float32)
    t = oracle.prepare_textures(m, np.ones(4, np.int32), lvl0.reshape(-1), 1, "f32", F32)
    mean = t.values.reshape(4, 5)[:, 4]                 # stored 1x1 mips
    f = np.float32(0.7)
    phi = math.log2(float(f) * 2.0)
    data = (1 - phi) * float(lvl0[0, 0, 0, 0]) + phi * (0.5625 * mean[0] + 0.1875 * mean[1] + 0.1875 * mean[3])
    W = (1 - phi) * 1.0 + phi * 0.9375
    o = oracle.lookup(m, t, _q(0, 0.25, 0.25, float(f)))[0, 0]
    assert o == pytest.approx(data / W, abs=1e-12)


# ------------------------------------------------------ brute force (tent sums)

def _brute_fetch(levels, x, y, f):
    """Independent evaluation: every texel of the selected level(s) weighted
    by the tensor product of tent functions max(0, 1 - |x N - 1/2 - i|)."""
    n = len(levels) - 1
    N0 = levels[0].shape[0]
    lam = math.log2(f * N0) if f > 0 else -1.0
    if not lam > 0:
        sel = [(0, 1.0)]
    elif math.floor(lam) >= n:
        sel = [(n, 1.0)]
    else:
        d = math.floor(lam)
        sel = [(d, 1.0 - (lam - d)), (d + 1, lam - d)]
    acc = np.zeros(levels[0].shape[2])
    W = 0.0
    for l, wl in sel:
        T = levels[l]
        N = T.shape[0]
        for j in range(N):
            for i in range(N):
                w = max(0.0, 1 - abs(x * N - 0.5 - i)) * max(0.0, 1 - abs(y * N - 0.5 - j))
                acc += wl * w * T[j, i]
                W += wl * w
    return acc, W


def _brute_lookup(m, tex, h, u, v, f):
    u, v = max(u, 0.0), max(v, 0.0)
    if u + v > 1:
        u, v = u / (u + v), v / (u + v)

    def quad(g, a, b):
        return (a, b) if g > m.twin[g] else (1 - a, 1 - b)

    acc = 0.0
    W = 0.0
    for g, (a, b) in ((h, (u, v)), (m.next[h], (v, -u)), (m.prev[h], (-v, u))):
        e = int(m.edge[g])
        levels = [tex.level(e, l) for l in range(int(tex.log2n[e]) + 1)]
        x, y = quad(g, a, b)
        da, dw = _brute_fetch(levels, x, y, f)
        acc = acc + da
        W += dw
    return acc / W


@pytest.mark.parametrize("n", [0, 1, 2])
def test_brute_force_tiny(n):
    m = oracle.mesh_from_faces(*syn.fig2_faces())
    log2n = np.full(m.num_edges, n, np.int32)
    lvl0 = syn.texels_f32(log2n, 2, seed=11 + n)
    t = oracle.prepare_textures(m, log2n, lvl0, 2, "f32", F32)
    h, u, v, _ = syn.queries(m.H, 300, seed=n)
    f = np.where(np.arange(300) % 3 == 0, 0.0, np.exp2(np.random.default_rng(n).uniform(-4, 1, 300)))
    got = oracle.lookup(m, t, (h, u, v, f))
    for q in range(300):
        ref = _brute_lookup(m, t, int(h[q]), float(u[q]), float(v[q]), float(f[q]))
        np.testing.assert_allclose(got[q], ref, rtol=0, atol=1e-12)


def test_brute_force_mixed_resolutions():
    m = oracle.mesh_from_faces(*syn.fig2_faces())
    log2n = (np.arange(m.num_edges) % 3).astype(np.int32)
    t = oracle.prepare_textures(m, log2n, syn.texels_f32(log2n, 1, seed=2), 1, "f32", F32)
    h, u, v, _ = syn.queries(m.H, 200, seed=9)
    f = np.exp2(np.random.default_rng(1).uniform(-5, 1, 200))
    got = oracle.lookup(m, t, (h, u, v, f))
    for q in range(200):
        ref = _brute_lookup(m, t, int(h[q]), float(u[q]), float(v[q]), float(f[q]))
        np.testing.assert_allclose(got[q], ref, atol=1e-12)


# -------------------------------------------------------------- special cases

def test_interior_query_is_library_bilinear():
    """More than half a texel from every quad side, only the own fetch has
    in-bounds taps, and the lookup is plain bilinear interpolation of the own
    texture (scipy's map_coordinates, order 1, at array coordinates
    (y N - 1/2, x N - 1/2))."""
    fs, fv, V, _ = syn.cube()
    m = oracle.mesh_from_faces(fs, fv, V)
    N = 8
    log2n = np.full(m.num_edges, 3, np.int32)
    t = oracle.prepare_textures(m, log2n, syn.texels_f32(log2n, 3, seed=4), 3, "f32", F32)
    rng = np.random.default_rng(0)
    for _ in range(200):
        h = int(rng.integers(0, m.H))
        u = rng.uniform(0.5 / N + 1e-9, 1)
        v = rng.uniform(0.5 / N + 1e-9, 1)
        if u + v > 1 - 1e-9:
            continue
        x, y = (u, v) if h > m.twin[h] else (1 - u, 1 - v)
        T = t.level(int(m.edge[h]), 0)
        ref = [ndimage.map_coordinates(T[:, :, c], [[y * N - 0.5], [x * N - 0.5]], order=1)[0]
               for c in range(3)]
        got = oracle.lookup(m, t, _q(h, u, v))[0]
        np.testing.assert_allclose(got, ref, atol=1e-12)


def test_texel_centres_return_texel():
    fs, fv, V, _ = syn.cube()
    m = oracle.mesh_from_faces(fs, fv, V)
    N = 4
    log2n = np.full(m.num_edges, 2, np.int32)
    t = oracle.prepare_textures(m, log2n, syn.texels_f32(log2n, 1, seed=8), 1, "f32", F32)
    for h in range(m.H):
        T = t.level(int(m.edge[h]), 0)
        for j in range(N):
            for i in range(N):
                u, v = (i + 0.5) / N, (j + 0.5) / N
                if u + v > 1:
                    continue
                x, y = (u, v) if h > m.twin[h] else (1 - u, 1 - v)
                ii, jj = int(round(x * N - 0.5)), int(round(y * N - 0.5))
                assert oracle.lookup(m, t, _q(h, u, v))[0, 0] == pytest.approx(T[jj, ii, 0], abs=1e-12)


def test_constant_texture_reproduced():
    fs, fv, V, _ = syn.cylinder(around=12, rows=6, seed=1)
    m = oracle.mesh_from_faces(fs, fv, V)
    log2n = (np.arange(m.num_edges) % 4).astype(np.int32)
    cnt = int(sum(4 ** int(n) for n in log2n))
    t = oracle.prepare_textures(m, log2n, np.full(cnt * 2, 0.375, np.float32), 2, "f32",
                                F32 | oracle.MIRROR_BOUNDARY)
    qs = syn.queries(m.H, 2000, seed=3, footprint="loguniform", lo=-6, hi=1)
    np.testing.assert_allclose(oracle.lookup(m, t, qs), 0.375, atol=1e-14)
    qs = syn.edge_queries(m.H, 2, footprints=(0.0, 0.3))
    np.testing.assert_allclose(oracle.lookup(m, t, qs), 0.375, atol=1e-14)


def test_partition_of_unity_via_gradient():
    """The blend weights w / W over all texels sum to one for every query."""
    m = oracle.mesh_from_faces(*syn.fig2_faces())
    log2n = np.full(m.num_edges, 2, np.int32)
    t = oracle.prepare_textures(m, log2n, syn.texels_f32(log2n, 1, 3), 1, "f32", F32)
    h, u, v, f = syn.queries(m.H, 50, seed=4, footprint="loguniform", lo=-5, hi=1)
    for q in range(50):
        g = oracle.lookup_grad(m, t, (h[q:q + 1], u[q:q + 1], v[q:q + 1], f[q:q + 1]), np.ones(1))
        assert g.sum() == pytest.approx(1.0, abs=1e-13)
        assert g.min() >= 0


def test_unit_weight_away_from_corners():
    """Uniform resolution N: the three fetches' normalisation weights sum to
    exactly one once u, v >= 1/(2N) (no quad corner within half a texel)."""
    fs, fv, V, _ = syn.cylinder(around=10, rows=5, seed=2)
    m = oracle.mesh_from_faces(fs, fv, V)
    N = 8
    log2n = np.full(m.num_edges, 3, np.int32)
    t = oracle.prepare_textures(m, log2n, syn.texels_f32(log2n, 1, 1), 1, "f32", F32)
    h, u, v, f = syn.queries(m.H, 5000, seed=7)
    keep = (u >= 0.5 / N) & (v >= 0.5 / N)
    _, w = oracle.lookup(m, t, (h[keep], u[keep], v[keep], f[keep]), return_weight=True)
    np.testing.assert_allclose(w, 1.0, atol=1e-14)
    # near the face centroid the weight is 3/4 + a/2 + b/2 - ab < 1 (a = uN, b = vN)
    _, w = oracle.lookup(m, t, _q(5, 0.01, 0.02), return_weight=True)
    a, b = 0.01 * N, 0.02 * N
    assert w[0] == pytest.approx(0.75 + a / 2 + b / 2 - a * b, abs=1e-14)


def test_clamp_and_invalid_queries():
    m = oracle.mesh_from_faces(*syn.single_quad())
    t = _tex_1x1(m, [1, 10, 100, 1000])
    h, u, v, f = syn.invalid_queries(m.H)
    out = oracle.lookup(m, t, (h, u, v, f))
    assert np.all(np.isnan(out[:3]))           # h out of range
    assert np.all(np.isnan(out[6:]))           # u or v not finite
    # (-0.5, 0.3) -> (0, 0.3); (0.9, 0.9) -> (0.5, 0.5); (2, -1) -> (1, 0)
    ref = oracle.lookup(m, t, (np.array([0, 0, 0], np.int32), np.array([0.0, 0.5, 1.0]),
                               np.array([0.3, 0.5, 0.0]), np.zeros(3)))
    np.testing.assert_allclose(out[3:6], ref, atol=1e-15)


# ------------------------------------------------------------------- seams

def _seam_points(m, rng, count):
    return rng.integers(0, m.H, count), rng.random(count)


def test_seams_across_next_and_twin_edges():
    """Both sides of every shared edge agree (Section 4.3, seamless
    filtering), except within half a texel of the edge's ends when corners
    are not pre-processed."""
    fs, fv, V, _ = syn.cylinder(around=12, rows=6, seed=4)
    m = oracle.mesh_from_faces(fs, fv, V)
    N = 4
    log2n = np.full(m.num_edges, 2, np.int32)
    t = oracle.prepare_textures(m, log2n, syn.texels_f32(log2n, 2, 5), 2, "f32", F32)
    rng = np.random.default_rng(0)
    hs, ts = _seam_points(m, rng, 3000)
    ts = 0.5 / N + ts * (1 - 1.0 / N)                  # stay half a texel from both ends
    zero = np.zeros_like(ts)
    # Next edge: (h, (0, t)) == (Next h, (t, 0))
    a = oracle.lookup(m, t, (hs.astype(np.int32), zero, ts, zero))
    b = oracle.lookup(m, t, (m.next[hs], ts, zero, zero))
    np.testing.assert_allclose(a, b, atol=1e-13)
    # twin diagonal: (h, (u, 1 - u)) == (Twin h, (1 - u, u))
    inner = m.twin[hs] >= 0
    h2 = hs[inner]
    u2 = ts[inner]
    a = oracle.lookup(m, t, (h2.astype(np.int32), u2, 1 - u2, np.zeros_like(u2)))
    b = oracle.lookup(m, t, (m.twin[h2], 1 - u2, u2, np.zeros_like(u2)))
    np.testing.assert_allclose(a, b, atol=1e-13)


def _corner_fixed(mesh, n, C, seed, flags=0):
    log2n = np.full(mesh.num_edges, n, np.int32)
    return oracle.prepare_textures(mesh, log2n, syn.texels_f32(log2n, C, seed), C, "f32",
                                   F32 | oracle.FIX_CORNERS | flags)


@pytest.mark.parametrize("gen", ["sphere", "cylinder"])
def test_corner_preprocessing_makes_vertices_and_centroids_continuous(gen):
    """With corner pre-processing and equal resolutions the lookup is
    continuous everywhere (Section 4.4): every triangle around a vertex of
    any valence returns one value there, every triangle of a face one value
    at its centroid, and shared edges agree up to their ends."""
    if gen == "sphere":
        fs, fv, V, _ = syn.uv_sphere(slices=9, rings=7, seed=1)
        flags = 0
    else:
        fs, fv, V, _ = syn.cylinder(around=9, rows=4, seed=1)
        flags = oracle.MIRROR_BOUNDARY
    m = oracle.mesh_from_faces(fs, fv, V)
    for fp in (0.0, 0.3, 1.0):
        t = _corner_fixed(m, 3, 2, seed=3, flags=flags)
        hs = np.arange(m.H, dtype=np.int32)
        f = np.full(m.H, fp)
        at_v = oracle.lookup(m, t, (hs, np.ones(m.H), np.zeros(m.H), f))       # Vert(h)
        at_n = oracle.lookup(m, t, (hs, np.zeros(m.H), np.ones(m.H), f))       # Vert(Next h)
        at_c = oracle.lookup(m, t, (hs, np.zeros(m.H), np.zeros(m.H), f))      # centroid
        for vtx in range(V):
            vals = np.concatenate([at_v[m.vert == vtx], at_n[m.vert[m.next] == vtx]])
            if len(vals):
                np.testing.assert_allclose(vals, np.broadcast_to(vals[0], vals.shape), atol=1e-13)
        for fc in range(m.num_faces):
            vals = at_c[m.face == fc]
            np.testing.assert_allclose(vals, np.broadcast_to(vals[0], vals.shape), atol=1e-13)
        # edges right up to their ends
        rng = np.random.default_rng(1)
        h = rng.integers(0, m.H, 2000)
        s = rng.random(2000)
        s[:50] = 0.0
        s[50:100] = 1e-3
        z = np.zeros_like(s)
        a = oracle.lookup(m, t, (h.astype(np.int32), z, s, z + fp))
        b = oracle.lookup(m, t, (m.next[h], s, z, z + fp))
        np.testing.assert_allclose(a, b, atol=1e-13)


def test_without_corner_fix_vertices_differ():
    fs, fv, V, _ = syn.uv_sphere(slices=9, rings=7, seed=1)
    m = oracle.mesh_from_faces(fs, fv, V)
    log2n = np.full(m.num_edges, 3, np.int32)
    t = oracle.prepare_textures(m, log2n, syn.texels_f32(log2n, 1, 3), 1, "f32", F32)
    hs = np.arange(m.H, dtype=np.int32)
    at_c = oracle.lookup(m, t, (hs, np.zeros(m.H), np.zeros(m.H), np.zeros(m.H)))
    spread = [np.ptp(at_c[m.face == fc]) for fc in range(m.num_faces)]
    assert max(spread) > 1e-3


# ------------------------------------------------------------ metamorphic

def test_renumbering_invariance():
    """Renumbering faces and rotating each face's vertex list gives new
    halfedge ids; with each texture carried to its edge's new id, and turned
    180 degrees wherever the larger id of its pair changed sides (Alg. 2),
    every lookup is unchanged."""
    fs, fv, V, _ = syn.uv_sphere(slices=8, rings=6, seed=2)
    m = oracle.mesh_from_faces(fs, fv, V)
    n = 2
    log2n = np.full(m.num_edges, n, np.int32)
    t = oracle.prepare_textures(m, log2n, syn.texels_f32(log2n, 1, 6), 1, "f32", F32)
    rng = np.random.default_rng(3)
    starts = np.concatenate([[0], np.cumsum(fs)[:-1]])
    faces = [list(fv[s:s + k]) for s, k in zip(starts, fs)]
    perm = rng.permutation(len(faces))
    nf = []
    for p in perm:
        r = int(rng.integers(0, len(faces[p])))
        nf.append(faces[p][r:] + faces[p][:r])
    m2 = oracle.mesh_from_faces([len(f) for f in nf], sum(nf, []), V)
    key = {(int(m2.vert[g]), int(m2.vert[m2.next[g]])): g for g in range(m2.H)}
    hmap = np.array([key[(int(m.vert[g]), int(m.vert[m.next[g]]))] for g in range(m.H)])
    own1, own2 = m.owner(), m2.owner()
    levels = []
    for e2 in range(m2.num_edges):
        g2 = own2[e2]
        g1 = int(np.nonzero(hmap == g2)[0][0])
        e1 = int(m.edge[g1])
        rotate = hmap[own1[e1]] != g2
        for l in range(n + 1):
            L = t.level(e1, l)
            levels.append((L[::-1, ::-1] if rotate else L).reshape(-1))
    t2 = oracle.prepare_textures(m2, log2n, np.concatenate(levels).astype(np.float32), 1, "f32",
                                 0, levels_given=True)
    h, u, v, f = syn.queries(m.H, 3000, seed=8, footprint="loguniform", lo=-4, hi=0.5)
    a = oracle.lookup(m, t, (h, u, v, f))
    b = oracle.lookup(m2, t2, (hmap[h].astype(np.int32), u, v, f))
    np.testing.assert_allclose(a, b, atol=1e-13)


# --------------------------------------------------------------- gradient

def test_gradient_matches_central_differences():
    """The lookup is linear in the texels, so central differences are exact
    up to rounding."""
    fs, fv, V, _ = syn.cylinder(around=6, rows=3, seed=5)
    m = oracle.mesh_from_faces(fs, fv, V)
    log2n = np.full(m.num_edges, 2, np.int32)
    t = oracle.prepare_textures(m, log2n, syn.texels_f32(log2n, 3, 2), 3, "f32", F32)
    qs = syn.queries(m.H, 400, seed=1, footprint="loguniform", lo=-4, hi=0)
    g = np.random.default_rng(0).standard_normal((400, 3))
    grad = oracle.lookup_grad(m, t, qs, g)
    rng = np.random.default_rng(1)
    nz = np.nonzero(grad)[0]
    pick = np.concatenate([rng.choice(nz, 40, replace=False),
                           rng.choice(grad.shape[0], 20, replace=False)])
    eps = 1e-3
    base = t.values.copy()
    for k in pick:
        t.values[:] = base
        t.values[k] += eps
        lp = float((oracle.lookup(m, t, qs) * g).sum())
        t.values[k] -= 2 * eps
        lm = float((oracle.lookup(m, t, qs) * g).sum())
        assert (lp - lm) / (2 * eps) == pytest.approx(grad[k], abs=1e-9)
    t.values[:] = base
