"""GPU parity: libhtex's CUDA lookup against the FP64 oracle, element by
element, on the same seeded inputs.  Tolerance: 1e-5 absolute for every
texel format when both sides filter the same stored values (FP32
accumulation of at most 24 weighted texels, weights in [0, 1], divided by a
normalisation sum >= 1/4); reduced-precision formats are also held to the
format bound u_fmt * max|T| + 1e-5 against the oracle on the original FP32
texels."""
import numpy as np
import pytest

import htex_synth as syn
import oracle
import paper_2207_05618_gb300 as hx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2207_05618_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _case(gen, log2n_fn, C, fmt, flags, seed=0, signed=False):
    fs, fv, V = gen()[:3]
    mo = oracle.mesh_from_faces(fs, fv, V)
    ml = hx.Mesh(fs, fv, V)
    log2n = log2n_fn(mo.num_edges)
    tex = (syn.texels_u8 if fmt == "u8" else syn.texels_f32)(log2n, C, seed)
    if signed:
        tex = tex * 3.0 - 1.0
    to = oracle.prepare_textures(mo, log2n, tex, C, fmt, flags)
    tl = hx.Textures.upload(ml, log2n, tex, C, fmt, flags)
    return mo, to, tl, log2n, tex


def _gpu(tl, qs, flags=0, status=None):
    q = torch.from_numpy(hx.pack_queries(*qs)).cuda()
    out = hx.lookup(tl, q, flags=flags, status=status)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _cmp(got, ref, tol=TOL):
    assert got.shape == ref.shape
    nan_g, nan_r = np.isnan(got), np.isnan(ref)
    np.testing.assert_array_equal(nan_g, nan_r)
    err = np.abs(got - ref)[~nan_r]
    assert err.size == 0 or err.max() <= tol, f"max err {err.max():.3g} at {np.argmax(err)}"
    return float(err.max()) if err.size else 0.0


def _cube():
    return syn.cube()


def _u(n):
    return lambda E: np.full(E, n, np.int32)


def _mixed(E):
    return (np.arange(E) * 7 % 5).astype(np.int32)


def test_cube_plain_fp32_single_batch():
    """Plain method on the closed cube: 16x16 RGBA FP32 textures with mips,
    65,536 queries with uniform h and barycentrics, level 0 bilinear."""
    mo, to, tl, *_ = _case(_cube, _u(4), 4, "f32", hx.BUILD_MIPS, seed=1)
    qs = syn.queries(mo.H, 65536, seed=2)
    _cmp(_gpu(tl, qs), oracle.lookup(mo, to, qs, nthreads=8))


def test_cube_staged_and_global_paths_agree():
    """Above a million queries the pool is staged in shared memory; both
    memory paths run the same arithmetic and must agree bit for bit, and
    with the oracle.  Ragged count (not a multiple of the block)."""
    mo, to, tl, *_ = _case(_cube, _u(4), 4, "f32", hx.BUILD_MIPS, seed=3)
    n = (1 << 20) + 13
    qs = syn.queries(mo.H, n, seed=4)
    a = _gpu(tl, qs)
    b = _gpu(tl, qs, flags=hx.LOOKUP_GLOBAL)
    np.testing.assert_array_equal(a, b)
    sel = np.random.default_rng(0).choice(n, 50000, replace=False)
    sel[:13] = np.arange(n - 13, n)
    ref = oracle.lookup(mo, to, tuple(x[sel] for x in qs), nthreads=8)
    _cmp(a[sel], ref)


@pytest.mark.parametrize("fmt", ["f32", "u8", "f16", "bf16", "e4m3"])
@pytest.mark.parametrize("C", [1, 2, 3, 4])
def test_formats_and_channels_cylinder(fmt, C):
    """Open cylinder (boundary halfedges, triangles and merged polygons),
    mixed resolutions 1..16, mirrored boundaries, trilinear footprints."""
    gen = lambda: syn.cylinder(around=20, rows=8, seed=5)
    mo, to, tl, *_ = _case(gen, _mixed, C, fmt, hx.BUILD_MIPS | hx.MIRROR_BOUNDARY, seed=C,
                           signed=fmt in ("f16", "bf16", "e4m3"))
    qs = syn.queries(mo.H, 20011, seed=6, footprint="loguniform", lo=-6, hi=1)
    _cmp(_gpu(tl, qs), oracle.lookup(mo, to, qs, nthreads=8))


@pytest.mark.parametrize("flags", [hx.BUILD_MIPS | hx.FIX_CORNERS,
                                   hx.BUILD_MIPS | hx.FIX_CORNERS | hx.MIRROR_BOUNDARY])
def test_adversarial_lattice_queries(flags):
    """Texel centres and borders, triangle sides and corners, at several
    footprints including level boundaries, on every halfedge."""
    gen = lambda: syn.cylinder(around=6, rows=3, seed=7)
    mo, to, tl, *_ = _case(gen, _u(2), 3, "f32", flags, seed=8)
    qs = syn.edge_queries(mo.H, 4, footprints=(0.0, 0.25, 0.5, 0.3, 1.0, 4.0))
    _cmp(_gpu(tl, qs), oracle.lookup(mo, to, qs))
    qs = syn.edge_queries(mo.H, 4, footprints=(0.125,))
    _cmp(_gpu(tl, qs, flags=hx.LOOKUP_GLOBAL), oracle.lookup(mo, to, qs))


def test_seamless_on_gpu_with_corner_fix():
    """Seamlessness checked on the GPU values themselves: with corner
    pre-processing every triangle around a vertex returns one value."""
    gen = lambda: syn.uv_sphere(slices=10, rings=8, seed=2)
    mo, to, tl, *_ = _case(gen, _u(3), 2, "f32", hx.BUILD_MIPS | hx.FIX_CORNERS, seed=9)
    H = mo.H
    hs = np.arange(H, dtype=np.int32)
    at_v = _gpu(tl, (hs, np.ones(H), np.zeros(H), np.zeros(H)))
    for vtx in range(mo.num_verts):
        vals = at_v[mo.vert == vtx]
        np.testing.assert_allclose(vals, np.broadcast_to(vals[0], vals.shape), atol=2e-6)


@pytest.mark.parametrize("fmt,u", [("f16", 2.0 ** -11), ("bf16", 2.0 ** -8), ("e4m3", 2.0 ** -4)])
def test_reduced_precision_against_fp32_oracle(fmt, u):
    """The config-1 cube and queries with FP16/BF16/E4M3 texels: within 1e-5
    of the oracle on the same stored values, and within u_fmt * max|T| +
    1e-5 of the oracle on the original FP32 texels."""
    mo, to, tl, log2n, tex = _case(_cube, _u(4), 4, fmt, hx.BUILD_MIPS, seed=1)
    ref32 = oracle.prepare_textures(mo, log2n, tex, 4, "f32", hx.BUILD_MIPS)
    qs = syn.queries(mo.H, 65536, seed=2)
    got = _gpu(tl, qs)
    _cmp(got, oracle.lookup(mo, to, qs, nthreads=8))
    err = np.abs(got - oracle.lookup(mo, ref32, qs, nthreads=8)).max()
    assert err <= u * np.abs(ref32.values).max() + TOL


def test_invalid_queries_give_nan_and_count():
    mo, to, tl, *_ = _case(_cube, _u(2), 4, "f32", hx.BUILD_MIPS)
    qs = syn.invalid_queries(mo.H)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = _gpu(tl, qs, status=status)
    _cmp(got, oracle.lookup(mo, to, qs))
    assert int(status.item()) == 5           # 3 bad ids, a NaN u, an infinite v


def test_empty_and_single_query():
    mo, to, tl, *_ = _case(_cube, _u(1), 2, "u8", hx.BUILD_MIPS)
    q = torch.empty((0, 4), dtype=torch.int32, device="cuda")
    assert hx.lookup(tl, q).shape == (0, 2)
    qs = syn.queries(mo.H, 1, seed=1)
    _cmp(_gpu(tl, qs), oracle.lookup(mo, to, qs))


@pytest.mark.parametrize("top,C,fmt", [(13, 1, "u8"), (12, 4, "f32")])
def test_maximum_resolution_texture(top, C, fmt):
    """One texture at the top resolution (8192^2 is the cap), the others
    small, footprints spanning every level of it (2^-15 .. 2): 32-bit
    texel offsets reach the top of the chain, and the result matches the
    oracle; also the sorted step and the anisotropic lookup."""
    fs, fv, V, _ = syn.cube()
    mo = oracle.mesh_from_faces(fs, fv, V)
    ml = hx.Mesh(fs, fv, V)
    log2n = (np.arange(mo.num_edges) % 4).astype(np.int32)
    log2n[5] = top
    tex = (syn.texels_u8 if fmt == "u8" else syn.texels_f32)(log2n, C, seed=31)
    to = oracle.prepare_textures(mo, log2n, tex, C, fmt, hx.BUILD_MIPS)
    tl = hx.Textures.upload(ml, log2n, tex, C, fmt, hx.BUILD_MIPS)
    hs = np.array([h for h in range(mo.H) if mo.edge[h] == 5 or mo.edge[mo.next[h]] == 5
                   or mo.edge[mo.prev[h]] == 5], np.int32)
    n = 200003
    _, u, v, f = syn.queries(mo.H, n, seed=32, footprint="loguniform", lo=-15, hi=1)
    h = np.random.default_rng(33).choice(hs, n).astype(np.int32)
    qs = (h, u, v, f)
    ref = oracle.lookup(mo, to, qs, nthreads=8)
    got = _gpu(tl, qs)
    _cmp(got, ref)
    q = torch.from_numpy(hx.pack_queries(*qs)).cuda()
    sq, pos = hx.sort_queries(tl, q)
    np.testing.assert_array_equal(hx.gather_results(hx.lookup(tl, sq), pos).cpu().numpy().astype(np.float64), got)
    rng = np.random.default_rng(34)
    d = [np.float32(x) for x in rng.uniform(-1e-3, 1e-3, (4, 20000))]
    qa = (h[:20000], u[:20000], v[:20000], *d)
    a = hx.lookup_aniso(tl, torch.from_numpy(hx.pack_queries_aniso(*qa)).cuda(), 16).cpu().numpy()
    # probe positions are rounded to float (<= 2^-24 in quad units), which moves
    # bilinear weights by up to N 2^-24 per axis: at N = 2^top that term dominates
    tol = 2 * 24 * 16 * 2.0 ** -24 + 4 * (1 << top) * 2.0 ** -24
    _cmp(a.astype(np.float64), oracle.lookup_aniso(mo, to, qa, 16, nthreads=8), tol)


def test_pool_round_trip_matches_host_preparation():
    fs, fv, V, _ = syn.cylinder(around=12, rows=5, seed=1)
    ml = hx.Mesh(fs, fv, V)
    log2n = _mixed(ml.E)
    tex = syn.texels_f32(log2n, 2, 3) * 2 - 1
    flags = hx.BUILD_MIPS | hx.MIRROR_BOUNDARY | hx.FIX_CORNERS
    for fmt in ("f32", "e4m3"):
        pool, scales = hx.Textures.prepare(ml, log2n, tex, 2, fmt, flags)
        tl = hx.Textures.upload(ml, log2n, tex, 2, fmt, flags)
        p2, s2 = tl.download_pool()
        np.testing.assert_array_equal(p2, pool)
        np.testing.assert_array_equal(s2, scales)
        t3 = hx.Textures.upload_pool(ml, log2n, pool, scales, 2, fmt)
        qs = syn.queries(ml.H, 5000, seed=2, footprint="loguniform")
        np.testing.assert_array_equal(_gpu(tl, qs), _gpu(t3, qs))


# ------------------------------------------------------------------ asset scale

def _subset_textures(mo, log2n, tex_u8, edges, C):
    """Oracle textures holding the real data only for 'edges' (1x1 zeros
    elsewhere).  Exact for queries whose faces use only those edges, since
    plain storage (mips only) treats every texture independently."""
    keep = np.zeros(mo.num_edges, bool)
    keep[edges] = True
    ln = np.where(keep, log2n, 0).astype(np.int32)
    starts = np.concatenate([[0], np.cumsum((1 << (2 * log2n.astype(np.int64))) * C)])
    parts = []
    for e in range(mo.num_edges):
        parts.append(tex_u8[starts[e]:starts[e + 1]] if keep[e] else np.zeros(C, np.uint8))
    return oracle.prepare_textures(mo, ln, np.concatenate(parts), C, "u8", hx.BUILD_MIPS)


def test_asset_scale_small():
    """Config-2 shape at a size the oracle covers whole: open cylinder with
    splits and merges, 64x64 RGBA8 textures with mips, log-uniform
    footprints over 2^-8..1, ragged query count."""
    gen = lambda: syn.cylinder(around=32, rows=16, seed=11)
    mo, to, tl, *_ = _case(gen, _u(6), 4, "u8", hx.BUILD_MIPS, seed=12)
    qs = syn.queries(mo.H, 300007, seed=13, footprint="loguniform")
    _cmp(_gpu(tl, qs), oracle.lookup(mo, to, qs, nthreads=8))


def test_binned_lookup_mid_asset():
    """Binning reorders queries by halfedge range once the pool exceeds a
    couple of L2-sized buckets (here about 97 MB of 32x32 RGBA8 texels):
    results equal the unbinned kernel's bit for bit and the oracle's within
    1e-5, including invalid queries (their own bucket) and a ragged count."""
    gen = lambda: syn.cylinder(around=128, rows=60, seed=14)
    mo, to, tl, *_ = _case(gen, _u(5), 4, "u8", hx.BUILD_MIPS | hx.MIRROR_BOUNDARY, seed=15)
    assert tl.pool_bytes > (64 << 20)
    h, u, v, f = syn.queries(mo.H, 300001, seed=16, footprint="loguniform")
    hb, ub, vb, fb = syn.invalid_queries(mo.H)
    qs = tuple(np.concatenate([a, b]) for a, b in zip((h, u, v, f), (hb, ub, vb, fb)))
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    a = _gpu(tl, qs, flags=hx.LOOKUP_BIN, status=status)
    b = _gpu(tl, qs)
    np.testing.assert_array_equal(a, b)
    assert int(status.item()) == 5
    _cmp(a, oracle.lookup(mo, to, qs, nthreads=8))


@pytest.mark.parametrize("fmt,C,n", [("u8", 4, 32), ("f32", 3, 16), ("f16", 1, 64), ("bf16", 2, 32)])
def test_sorted_lookup_multi_chunk(fmt, C, n):
    """The sorted path works on chunks of 2^24 queries: a full chunk plus a
    ragged one, every channel count (results go back to their queries'
    places), equal bit for bit to the unsorted kernel and to the oracle
    within 1e-5 on a sample (invalid queries included)."""
    gen = lambda: syn.cylinder(around=128, rows=60, seed=14)
    log2n_fn = _u(int(np.log2(n)))
    mo, to, tl, *_ = _case(gen, log2n_fn, C, fmt, hx.BUILD_MIPS | hx.MIRROR_BOUNDARY, seed=17)
    assert tl.pool_bytes > (64 << 20)
    h, u, v, f = syn.queries(mo.H, (3 << 23) + 4321, seed=18, footprint="loguniform")
    hb, ub, vb, fb = syn.invalid_queries(mo.H)
    k = len(h) // 2
    qs = tuple(np.concatenate([a[:k], b, a[k:]]) for a, b in zip((h, u, v, f), (hb, ub, vb, fb)))
    a = _gpu(tl, qs, flags=hx.LOOKUP_BIN)
    b = _gpu(tl, qs)
    np.testing.assert_array_equal(np.isnan(a), np.isnan(b))
    np.testing.assert_array_equal(np.nan_to_num(a, nan=0.0), np.nan_to_num(b, nan=0.0))
    sel = np.concatenate([np.random.default_rng(3).choice(len(qs[0]), 60000, replace=False),
                          np.arange(k, k + len(hb)), [0, len(qs[0]) - 1]])
    _cmp(a[sel], oracle.lookup(mo, to, tuple(x[sel] for x in qs), nthreads=8))


def _range_shift(H, ranges=128):
    s = 0
    while (H >> s) + 1 > ranges:
        s += 1
    return s


def test_sort_queries_and_gather_results():
    """htex_queries_sort permutes the queries (each one unchanged, pos its
    new place) into ascending halfedge ranges within each 2^24-query chunk,
    invalid queries last; filtering the sorted copy and gathering the
    results back equals the unsorted lookup bit for bit; a gather position
    outside [0, n) gives NaN."""
    gen = lambda: syn.cylinder(around=128, rows=60, seed=14)
    mo, to, tl, *_ = _case(gen, _u(5), 4, "u8", hx.BUILD_MIPS | hx.MIRROR_BOUNDARY, seed=15)
    n = (1 << 24) + 77777
    h, u, v, f = syn.queries(mo.H, n, seed=19, footprint="loguniform")
    h[::1001] = -3
    h[5::2003] = mo.H
    q = torch.from_numpy(hx.pack_queries(h, u, v, f)).cuda()
    sq, pos = hx.sort_queries(tl, q)
    p = pos.cpu().numpy().astype(np.int64)
    assert np.array_equal(np.sort(p), np.arange(n))
    sq_np, q_np = sq.cpu().numpy(), q.cpu().numpy()
    assert np.array_equal(sq_np[p], q_np)
    s = _range_shift(mo.H)
    hs = sq_np[:, 0].astype(np.int64)
    key = np.where((hs >= 0) & (hs < mo.H), hs >> s, 1 << 40)
    for c0 in range(0, n, 1 << 24):
        k = key[c0:c0 + (1 << 24)]
        assert np.all(np.diff(k) >= 0)
        assert np.all((p[c0:c0 + (1 << 24)] >= c0) & (p[c0:c0 + (1 << 24)] < c0 + len(k)))
    sout = hx.lookup(tl, sq)
    got = hx.gather_results(sout, pos)
    ref = hx.lookup(tl, q)
    assert torch.equal(torch.isnan(got), torch.isnan(ref))
    assert torch.equal(torch.nan_to_num(got, nan=0.0), torch.nan_to_num(ref, nan=0.0))
    assert torch.equal(hx.lookup(tl, q, flags=hx.LOOKUP_BIN).nan_to_num(nan=0.0), ref.nan_to_num(nan=0.0))
    bad = pos.clone()
    bad[:3] = torch.tensor([-1, n, 2**31 - 1], dtype=torch.int32)
    g2 = hx.gather_results(sout, bad).cpu()
    assert torch.isnan(g2[:3]).all() and torch.equal(g2[3:].nan_to_num(nan=0.0), got[3:].cpu().nan_to_num(nan=0.0))
    sel = np.random.default_rng(4).choice(n, 30000, replace=False)
    _cmp(got.cpu().numpy().astype(np.float64)[sel],
         oracle.lookup(mo, to, tuple(x[sel] for x in (h, u, v, f)), nthreads=8))


@pytest.mark.slow
@pytest.mark.parametrize("flags", [0, hx.LOOKUP_BIN])
def test_asset_scale_full_sampled(flags):
    """The full asset-scale workload as the benchmark runs it (about 520k
    halfedges, 4.3 GB of level-0 RGBA8 texels, 16M queries in one launch);
    a sample of 100k outputs plus the first and last checked against the
    oracle restricted to the sampled queries' faces."""
    fs, fv, V, _ = syn.cylinder()
    ml = hx.Mesh(fs, fv, V)
    mo = oracle.mesh_from_faces(fs, fv, V)
    log2n = np.full(ml.E, 6, np.int32)
    tex = syn.texels_u8(log2n, 4, seed=21)
    tl = hx.Textures.upload(ml, log2n, tex, 4, "u8", hx.BUILD_MIPS)
    n = 1 << 24
    qs = syn.queries(ml.H, n, seed=22, footprint="loguniform")
    got = _gpu(tl, qs, flags=flags)
    sel = np.random.default_rng(1).choice(n, 100000, replace=False)
    sel[:2] = (0, n - 1)
    hs = qs[0][sel]
    edges = np.unique(np.concatenate([mo.edge[hs], mo.edge[mo.next[hs]], mo.edge[mo.prev[hs]]]))
    to = _subset_textures(mo, log2n, tex, edges, 4)
    ref = oracle.lookup(mo, to, tuple(x[sel] for x in qs), nthreads=16)
    _cmp(got[sel], ref)
    tl.close()


# --------------------------------------------------------------------- backward

@pytest.mark.parametrize("fmt,C", [("f32", 3), ("f32", 4), ("u8", 4), ("f16", 2), ("e4m3", 1)])
def test_backward_matches_oracle_gradient(fmt, C):
    gen = lambda: syn.uv_sphere(slices=12, rings=9, seed=3)
    mo, to, tl, *_ = _case(gen, _mixed, C, fmt, hx.BUILD_MIPS, seed=4)
    n = 40000
    qs = syn.queries(mo.H, n, seed=5, footprint="loguniform", lo=-5, hi=0.5)
    g = np.random.default_rng(6).standard_normal((n, C)).astype(np.float32)
    q = torch.from_numpy(hx.pack_queries(*qs)).cuda()
    grad = hx.lookup_backward(tl, q, torch.from_numpy(g).cuda())
    torch.cuda.synchronize()
    ref = oracle.grad_to_pool_layout(to, oracle.lookup_grad(mo, to, qs, g.astype(np.float64)),
                                     {"f32": 4, "u8": 1, "f16": 2, "bf16": 2, "e4m3": 1}[fmt])
    got = grad.cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-5 * max(scale, 1.0)


# ------------------------------------------------------------------- host path

@pytest.mark.parametrize("mode", ["pinned", "pageable", "mixed", "misaligned"])
def test_lookup_host_matches_device_lookup(mode):
    """htex_lookup_host gives the device lookup's results bit for bit, in
    place on pinned memory and through chunks of 2^21 over three internal
    streams otherwise (pageable buffers, a pinned/pageable mix, a pinned
    result buffer misaligned for 16-byte stores), across chunk boundaries
    and a ragged tail."""
    gen = lambda: syn.cylinder(around=32, rows=16, seed=11)
    mo, to, tl, *_ = _case(gen, _u(6), 4, "u8", hx.BUILD_MIPS, seed=12)
    n = 2 * (1 << 21) + 13
    qs = syn.queries(mo.H, n, seed=13, footprint="loguniform")
    qh = torch.from_numpy(hx.pack_queries(*qs))
    if mode != "pageable":
        qh = qh.pin_memory()
    if mode == "misaligned":
        out = torch.empty(n * 4 + 1, dtype=torch.float32).pin_memory()[1:].view(n, 4)
    else:
        out = torch.empty((n, 4), dtype=torch.float32)
        out = out.pin_memory() if mode == "pinned" else out
    hx.lookup_host(tl, qh, out=out, flags=hx.LOOKUP_BIN if mode == "pinned" else 0)
    torch.cuda.synchronize()
    ref = hx.lookup(tl, qh.cuda()).cpu()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    sel = np.random.default_rng(2).choice(n, 20000, replace=False)
    _cmp(out.numpy()[sel].astype(np.float64), oracle.lookup(mo, to, tuple(x[sel] for x in qs), nthreads=8))
