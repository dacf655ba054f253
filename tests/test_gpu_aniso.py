"""GPU parity of htex_lookup_aniso against the FP64 oracle's anisotropic
lookup, element by element on the same seeded inputs.

Tolerance: the result is a convex combination of at most m = 24 * max_aniso
taps accumulated in FP32 (numerator and weight sum), so |err| <= 2 m u
max|T| with u = 2^-24; each probe position is rounded to float (<= u in
quad units), which moves a bilinear weight by up to N u per axis, adding
4 N u max|T| for textures of N texels a side.  The tests use
max(1e-5, 2 m u max|T| + 4 N u max|T|) against the oracle on the same
stored values."""
import numpy as np
import pytest

import htex_synth as syn
import oracle
import paper_2207_05618_gb300 as hx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2207_05618_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _tol(kmax, tmax=1.0, nmax=16):
    return max(1e-5, (2 * 24 * kmax + 4 * nmax) * 2.0 ** -24 * tmax)


def _aniso_queries(H, n, seed, lo=-9.0, hi=1.0, max_ratio=24.0):
    """Log-uniform major axis length 2^lo..2^hi, log-uniform anisotropy
    1..max_ratio, uniform direction; barycentrics uniform on the triangle."""
    h, u, v, _ = syn.queries(H, n, seed=seed)
    rng = np.random.default_rng(seed + 1)
    major = np.exp2(rng.uniform(lo, hi, n))
    minor = major / np.exp(rng.uniform(0.0, np.log(max_ratio), n))
    th = rng.uniform(0, 2 * np.pi, n)
    c, s = np.cos(th), np.sin(th)
    d = (major * c, major * s, -minor * s, minor * c)
    swap = rng.random(n) < 0.5            # the major axis on x or on y
    d = tuple(np.where(swap, d[(k + 2) % 4], d[k]).astype(np.float32) for k in range(4))
    return (h, u, v) + d


def _case(gen, log2n_fn, C, fmt, flags, seed):
    fs, fv, V = gen()[:3]
    mo = oracle.mesh_from_faces(fs, fv, V)
    ml = hx.Mesh(fs, fv, V)
    log2n = log2n_fn(mo.num_edges)
    tex = (syn.texels_u8 if fmt == "u8" else syn.texels_f32)(log2n, C, seed)
    to = oracle.prepare_textures(mo, log2n, tex, C, fmt, flags)
    tl = hx.Textures.upload(ml, log2n, tex, C, fmt, flags)
    return mo, to, tl


def _gpu(tl, qs, kmax, status=None):
    q = torch.from_numpy(hx.pack_queries_aniso(*qs)).cuda()
    out = hx.lookup_aniso(tl, q, kmax, status=status)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _cmp(got, ref, tol):
    assert got.shape == ref.shape
    np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    err = np.abs(got - ref)[ok]
    assert err.size == 0 or err.max() <= tol, f"max err {err.max():.3g} (tol {tol:.3g})"


@pytest.mark.parametrize("fmt,C,kmax", [("f32", 4, 16), ("f32", 3, 4), ("u8", 4, 8), ("f16", 2, 16),
                                        ("e4m3", 1, 2), ("bf16", 4, 1)])
def test_aniso_matches_oracle_mixed_resolutions(fmt, C, kmax):
    """Sphere with mixed texture resolutions (1x1 .. 16x16) and mips,
    footprints from a fraction of a texel to a few quads, anisotropy up to
    24 (so K reaches the bound), ragged query count."""
    gen = lambda: syn.uv_sphere(slices=12, rings=9, seed=3)
    mo, to, tl = _case(gen, lambda E: (np.arange(E) * 7 % 5).astype(np.int32), C, fmt,
                       hx.BUILD_MIPS | hx.MIRROR_BOUNDARY, seed=4)
    qs = _aniso_queries(mo.H, 30011, seed=5, lo=-9, hi=2)
    _cmp(_gpu(tl, qs, kmax), oracle.lookup_aniso(mo, to, qs, kmax, nthreads=8), _tol(kmax))


def test_aniso_asset_shape_spans_many_tiles():
    """Open cylinder with splits and merges, 32x32 RGBA8 with mips, 200k
    queries (many blocks, ragged tail), max_aniso 16."""
    gen = lambda: syn.cylinder(around=40, rows=20, seed=11)
    mo, to, tl = _case(gen, lambda E: np.full(E, 5, np.int32), 4, "u8", hx.BUILD_MIPS, seed=12)
    qs = _aniso_queries(mo.H, 200003, seed=13)
    _cmp(_gpu(tl, qs, 16), oracle.lookup_aniso(mo, to, qs, 16, nthreads=8), _tol(16, nmax=32))


def test_aniso_isotropic_footprint_equals_trilinear_lookup():
    """Equal axis lengths whose squares are exact in float: one probe with
    footprint f, the isotropic lookup's arithmetic on the GPU up to
    accumulation order (both within 1e-5 of each other)."""
    gen = lambda: syn.cube()
    mo, to, tl = _case(gen, lambda E: np.full(E, 4, np.int32), 4, "f32", hx.BUILD_MIPS, seed=1)
    h, u, v, f = syn.queries(mo.H, 65536, seed=2, footprint="loguniform")
    m, e = np.frexp(f.astype(np.float64))
    f = np.ldexp(np.round(m * 4096) / 4096, e).astype(np.float32)
    z = np.zeros_like(f)
    a = _gpu(tl, (h, u, v, f, z, z, f), 16)
    qi = torch.from_numpy(hx.pack_queries(h, u, v, f)).cuda()
    b = hx.lookup(tl, qi).cpu().numpy().astype(np.float64)
    _cmp(a, b, 1e-5)


def test_aniso_invalid_queries_and_arguments():
    gen = lambda: syn.cube()
    mo, to, tl = _case(gen, lambda E: np.full(E, 3, np.int32), 2, "f32", hx.BUILD_MIPS, seed=6)
    qs = _aniso_queries(mo.H, 1000, seed=7)
    qs = tuple(np.array(x) for x in qs)
    qs[0][:3] = (-1, mo.H, 5)
    qs[1][3] = np.nan
    qs[3][4] = np.inf
    qs[6][5] = np.nan
    qs[3][6] = np.float32(3e19)        # squared length overflows float
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = _gpu(tl, qs, 8, status=status)
    assert int(status.item()) == 6
    assert np.isnan(got[[0, 1, 3, 4, 5, 6]]).all() and not np.isnan(got[2]).any()
    _cmp(got, oracle.lookup_aniso(mo, to, qs, 8), _tol(8))
    q = torch.from_numpy(hx.pack_queries_aniso(*qs)).cuda()
    for bad in (0, 17):
        with pytest.raises(hx.HtexError):
            hx.lookup_aniso(tl, q, bad)
    assert hx.lookup_aniso(tl, q[:0], 4).shape == (0, 2)


def test_sorted_aniso_equals_unsorted_multi_chunk():
    """HTEX_LOOKUP_BIN on the anisotropic lookup: 32-byte queries sorted by
    halfedge range in chunks of 2^24 (a full chunk and a ragged one, invalid
    queries inside) on a pool above the 64 MiB threshold give the unsorted
    results bit for bit, and the oracle's on a sample."""
    gen = lambda: syn.cylinder(around=128, rows=60, seed=14)
    mo, to, tl = _case(gen, lambda E: np.full(E, 5, np.int32), 4, "u8", hx.BUILD_MIPS, seed=15)
    assert tl.pool_bytes > (64 << 20)
    n = (1 << 24) + 1237
    qs = tuple(np.array(x) for x in _aniso_queries(mo.H, n, seed=16, lo=-8, hi=0))
    qs[0][::70001] = -2
    q = torch.from_numpy(hx.pack_queries_aniso(*qs)).cuda()
    s0 = torch.zeros(1, dtype=torch.int32, device="cuda")
    s1 = torch.zeros(1, dtype=torch.int32, device="cuda")
    a = hx.lookup_aniso(tl, q, 16, status=s0)
    b = hx.lookup_aniso(tl, q, 16, status=s1, flags=hx.LOOKUP_BIN)
    assert int(s0.item()) == int(s1.item()) == int((qs[0] < 0).sum())
    assert torch.equal(torch.isnan(a), torch.isnan(b))
    assert torch.equal(a.nan_to_num(nan=0.0), b.nan_to_num(nan=0.0))
    sel = np.random.default_rng(17).choice(n, 20000, replace=False)
    _cmp(b.cpu().numpy().astype(np.float64)[sel],
         oracle.lookup_aniso(mo, to, tuple(x[sel] for x in qs), 16, nthreads=8), _tol(16, nmax=32))
