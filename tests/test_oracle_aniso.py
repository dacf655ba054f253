"""Pins of the oracle's anisotropic lookup (the reading of Section 5.1's
anisotropic filtering: K probes along the footprint's major axis, each
sampling Alg. 3's three fetches trilinearly, one shared normalisation).

Checked against what the definitions fix: reduction to the pinned isotropic
lookup, a constant texture, probe positions landing on texel centres
(hand-computed means of mip texels), the spread cap in closed form at the
1x1 level, agreement of the two halfedges of a shared edge, and NaN for
invalid queries."""
import numpy as np
import pytest

import htex_synth as syn
import oracle


def _cube_case(n=4, C=4, seed=1, flags=oracle.BUILD_MIPS):
    fs, fv, V, _ = syn.cube()
    m = oracle.mesh_from_faces(fs, fv, V)
    log2n = np.full(m.num_edges, n, np.int32)
    t = oracle.prepare_textures(m, log2n, syn.texels_f32(log2n, C, seed), C, "f32", flags)
    return m, t


def _q12(x):
    """Values with at most 12 significant bits: their float squares are exact."""
    m, e = np.frexp(np.asarray(x, np.float64))
    return np.ldexp(np.round(m * 4096.0) / 4096.0, e).astype(np.float32)


def _texel(t, e, l, i, j):
    n = int(t.log2n[e])
    N = 1 << (n - l)
    base = int(t.toff[e]) + sum((1 << (n - k)) ** 2 for k in range(l))
    return t.values[(base + j * N + i) * t.channels:(base + j * N + i + 1) * t.channels]


def test_zero_footprint_equals_level0_lookup():
    m, t = _cube_case()
    h, u, v, _ = syn.queries(m.H, 3000, seed=3)
    z = np.zeros(3000, np.float32)
    a = oracle.lookup_aniso(m, t, (h, u, v, z, z, z, z), 16)
    b = oracle.lookup(m, t, (h, u, v, z))
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("swap", [False, True])
def test_isotropic_derivatives_reduce_to_trilinear(swap):
    """|ax| = |ay| = f: one probe at the centre with footprint f, i.e. the
    isotropic lookup of footprint f (trilinear), exactly."""
    m, t = _cube_case(n=5)
    h, u, v, f = syn.queries(m.H, 3000, seed=4, footprint="loguniform", lo=-8, hi=1)
    f = _q12(f)
    z = np.zeros_like(f)
    d = (z, f, f, z) if swap else (f, z, z, f)
    a = oracle.lookup_aniso(m, t, (h, u, v) + d, 16)
    b = oracle.lookup(m, t, (h, u, v, f))
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)


def test_constant_texture_any_footprint():
    """Normalisation: a constant texture gives the constant for every
    anisotropy, direction, probe bound and footprint size (spread cap
    included)."""
    fs, fv, V, _ = syn.uv_sphere(slices=10, rings=7, seed=1)
    m = oracle.mesh_from_faces(fs, fv, V)
    log2n = (np.arange(m.num_edges) % 4 + 1).astype(np.int32)
    tot = int(sum(4 ** int(k) for k in log2n))
    t = oracle.prepare_textures(m, log2n, np.full(tot * 3, 0.625, np.float32), 3, "f32", oracle.BUILD_MIPS)
    rng = np.random.default_rng(5)
    n = 4000
    h, u, v, _ = syn.queries(m.H, n, seed=6)
    mag = np.exp(rng.uniform(np.log(1e-4), np.log(50.0), (n, 2))).astype(np.float32)
    th = rng.uniform(0, 2 * np.pi, n)
    d = (mag[:, 0] * np.cos(th), mag[:, 0] * np.sin(th), -mag[:, 1] * np.sin(th), mag[:, 1] * np.cos(th))
    for kmax in (1, 2, 7, 16):
        out = oracle.lookup_aniso(m, t, (h, u, v) + tuple(np.float32(x) for x in d), kmax)
        np.testing.assert_allclose(out, 0.625, rtol=0, atol=1e-12)


def _own_quad_halfedge(m):
    """A halfedge whose quad coordinates are its barycentrics (Alg. 2: the
    larger id of its pair)."""
    for h in range(m.H):
        if h > m.twin[h] >= 0:
            return h
    raise AssertionError


@pytest.mark.parametrize("K,r", [(3, 3.0), (4, 4.0), (4, 3.5)])
def test_probes_land_on_texel_centres(K, r):
    """Hand-computed: 16x16 textures.  K = 4: |ax| = 1/2, |ay| = 1/8, so
    K = ceil(sqrt(16)) = 4 and the per-probe footprint 1/8 selects level 1
    (8x8) alone; the probes sit 1.5 and 0.5 texels either side of u = 1/2,
    on the centres of texels 2..5 of row 1; |ay| = 1/7 (ratio 3.5) rounds the
    probe count up to the same 4.  K = 3: |ax| = 3/4, |ay| = 1/4, footprint
    1/4 selects level 2 (4x4); probes at texels 0, 1, 2 of row 0.  The Next
    and Prev fetches have no tap in bounds; the result is the plain mean of
    those mip texels."""
    m, t = _cube_case(n=4, C=4, seed=7)
    h = _own_quad_halfedge(m)
    e = int(m.edge[h])
    if K == 4:
        s, u, v, lvl, cols, row = 0.5, 0.5, 1.5 / 8, 1, range(2, 6), 1
    else:
        s, u, v, lvl, cols, row = 0.75, 1.5 / 4, 0.5 / 4, 2, range(0, 3), 0
    q = (np.array([h], np.int32), np.array([u], np.float32), np.array([v], np.float32),
         np.array([s], np.float32), np.array([0], np.float32), np.array([0], np.float32),
         np.array([s / r], np.float32))
    got = oracle.lookup_aniso(m, t, q, 16)[0]
    want = np.mean([_texel(t, e, lvl, i, row) for i in cols], axis=0)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)
    # a probe bound below K changes the result (fewer, wider-spaced probes)
    assert not np.allclose(oracle.lookup_aniso(m, t, q, K - 1)[0], want, atol=1e-6)


def _tent(z):
    return np.maximum(0.0, 1.0 - np.abs(z - 0.5))


def test_spread_cap_closed_form_at_the_1x1_level():
    """|ax| = 8, ay = 0, at most 2 probes: K = 2, per-probe footprint 4 puts
    every fetch on its 1x1 level, and the spread is capped at K = 2 quad
    widths, so the probes sit at u +- 1/2.  At the 1x1 level a fetch at quad
    coordinates (x, y) is T * tent(x) * tent(y) with weight tent(x) tent(y),
    tent(z) = max(0, 1 - |z - 1/2|) (symmetric about 1/2, so Alg. 2's
    reflection does not change it)."""
    m, t = _cube_case(n=4, C=3, seed=8)
    n = 200
    h, u, v, _ = syn.queries(m.H, n, seed=10)
    z = np.zeros(n, np.float32)
    got = oracle.lookup_aniso(m, t, (h, u, v, np.full(n, 8, np.float32), z, z, z), 2)
    for k in range(n):
        hk = int(h[k])
        T = [_texel(t, int(m.edge[g]), 4, 0, 0) for g in (hk, m.next[hk], m.prev[hk])]
        num, den = np.zeros(3), 0.0
        for off in (-0.5, 0.5):
            up, vp = float(u[k]) + off, float(v[k])
            ws = (_tent(up) * _tent(vp), _tent(vp) * _tent(-up), _tent(-vp) * _tent(up))
            for w, tv in zip(ws, T):
                num += w * tv
                den += w
        np.testing.assert_allclose(got[k], num / den, rtol=0, atol=1e-13)


def test_shared_edge_agrees_from_both_sides():
    """A point on a mesh edge seen from h at (u, 1 - u) and from Twin(h) at
    (1 - u, u).  Over the shared quad the twin's barycentrics are 1 - x and
    1 - y where h's are x and y (Alg. 2), so the same quad-space footprint
    has the negated derivatives.  Both then take the same samples of the
    shared quad; away from the face centroids the Next and Prev fetches have
    no tap in bounds, so the two results agree."""
    m, t = _cube_case(n=5, C=4, seed=11)
    rng = np.random.default_rng(12)
    hs = np.array([h for h in range(m.H) if m.twin[h] >= 0], np.int32)
    n = 2000
    h = rng.choice(hs, n)
    u = (rng.integers(int(0.35 * 65536), int(0.65 * 65536), n) / 65536.0).astype(np.float32)
    v = (1.0 - u).astype(np.float32)   # exact: u + v = 1 on the edge
    a = (rng.uniform(-1, 1, (n, 4)) * np.exp(rng.uniform(np.log(1e-3), np.log(2e-2), (n, 1)))).astype(np.float32)
    own = oracle.lookup_aniso(m, t, (h, u, v, a[:, 0], a[:, 1], a[:, 2], a[:, 3]), 16)
    tw = m.twin[h].astype(np.int32)
    other = oracle.lookup_aniso(m, t, (tw, v, u, -a[:, 0], -a[:, 1], -a[:, 2], -a[:, 3]), 16)
    np.testing.assert_allclose(own, other, rtol=0, atol=1e-12)


def test_invalid_queries_are_nan():
    m, t = _cube_case()
    big = np.float32(2e19)
    qs = [(-1, 0.2, 0.2, 0, 0, 0, 0), (m.H, 0.2, 0.2, 0, 0, 0, 0), (0, np.nan, 0.2, 0, 0, 0, 0),
          (0, 0.2, 0.2, np.inf, 0, 0, 0), (0, 0.2, 0.2, 0, 0, np.nan, 0), (0, 0.2, 0.2, big, 0, 0, 0)]
    cols = list(zip(*qs))
    q = (np.array(cols[0], np.int32),) + tuple(np.array(c, np.float32) for c in cols[1:])
    assert np.isnan(oracle.lookup_aniso(m, t, q, 8)).all()
