"""Oracle pins: texture storage (paper Sections 4.3 and 4.4) and the
reduced-precision formats, checked against library conversions and
closed-form bounds."""
import numpy as np
import pytest
import torch

import htex_synth as syn
import oracle


def _mesh(gen="cyl"):
    if gen == "cyl":
        fs, fv, V, _ = syn.cylinder(around=7, rows=3, seed=9)
    else:
        fs, fv, V, _ = syn.uv_sphere(slices=7, rings=5, seed=9)
    return oracle.mesh_from_faces(fs, fv, V)


def test_mips_are_box_means():
    m = _mesh()
    log2n = (np.arange(m.num_edges) % 4).astype(np.int32)
    lvl0 = syn.texels_f32(log2n, 3, seed=1)
    t = oracle.prepare_textures(m, log2n, lvl0, 3, "f32", oracle.BUILD_MIPS)
    for e in range(m.num_edges):
        for l in range(int(log2n[e])):
            a = t.level(e, l)
            N = a.shape[0]
            ref = a.reshape(N // 2, 2, N // 2, 2, 3).mean(axis=(1, 3)).astype(np.float32)
            np.testing.assert_array_equal(t.level(e, l + 1), ref.astype(np.float64))


def test_u8_mips_integer_means():
    m = _mesh()
    log2n = np.full(m.num_edges, 3, np.int32)
    lvl0 = syn.texels_u8(log2n, 4, seed=2)
    t = oracle.prepare_textures(m, log2n, lvl0, 4, "u8", oracle.BUILD_MIPS)
    raw = t.extra["raw"]
    for e in range(m.num_edges):
        for l in range(3):
            a = np.round(t.level(e, l) * 255.0).astype(np.int64)
            N = a.shape[0]
            ref = (a.reshape(N // 2, 2, N // 2, 2, 4).sum(axis=(1, 3)) + 2) // 4
            np.testing.assert_array_equal(np.round(t.level(e, l + 1) * 255), ref)
    assert np.all(raw == np.round(raw))


def test_boundary_mirroring():
    """Boundary textures mirror across the diagonal x + y = 1 at every level;
    interior textures are untouched."""
    m = _mesh()
    log2n = np.full(m.num_edges, 3, np.int32)
    lvl0 = syn.texels_f32(log2n, 2, seed=3)
    plain = oracle.prepare_textures(m, log2n, lvl0, 2, "f32", oracle.BUILD_MIPS)
    t = oracle.prepare_textures(m, log2n, lvl0, 2, "f32", oracle.BUILD_MIPS | oracle.MIRROR_BOUNDARY)
    owner = m.owner()
    nb = 0
    for e in range(m.num_edges):
        boundary = m.twin[owner[e]] < 0
        nb += boundary
        for l in range(4):
            L = t.level(e, l)
            if boundary:
                # reflection (i, j) -> (N-1-j, N-1-i) is a transpose of the flipped image
                np.testing.assert_array_equal(L, L[::-1, ::-1].transpose(1, 0, 2))
                if l == 0:
                    N = L.shape[0]
                    keep = np.add.outer(np.arange(N), np.arange(N)) <= N - 1
                    np.testing.assert_array_equal(L[keep], plain.level(e, 0)[keep])
            else:
                np.testing.assert_array_equal(L, plain.level(e, l))
    assert nb == 14


def _corners(t, m, e, l):
    L = t.level(e, l)
    N = L.shape[0]
    return [L[0, N - 1], L[N - 1, 0], L[0, 0], L[N - 1, N - 1]]


@pytest.mark.parametrize("fmt", ["f32", "u8"])
def test_corner_fix_touches_corners_only_and_keeps_means(fmt):
    m = _mesh("sph")
    log2n = np.full(m.num_edges, 2, np.int32)
    gen = syn.texels_u8 if fmt == "u8" else syn.texels_f32
    lvl0 = gen(log2n, 1, seed=4)
    a = oracle.prepare_textures(m, log2n, lvl0, 1, fmt, oracle.BUILD_MIPS)
    b = oracle.prepare_textures(m, log2n, lvl0, 1, fmt, oracle.BUILD_MIPS | oracle.FIX_CORNERS)
    for l in (0, 1):      # 4x4 and 2x2: corners are distinct texels
        sa = sb = 0.0
        for e in range(m.num_edges):
            La, Lb = a.level(e, l), b.level(e, l)
            N = La.shape[0]
            mask = np.ones((N, N), bool)
            mask[[0, 0, N - 1, N - 1], [0, N - 1, 0, N - 1]] = False
            np.testing.assert_array_equal(La[mask], Lb[mask])
            sa += sum(float(x[0]) for x in _corners(a, m, e, l))
            sb += sum(float(x[0]) for x in _corners(b, m, e, l))
        # group means preserve the sum of corner values (exactly for floats
        # up to rounding; within half a code per group for bytes)
        assert sb == pytest.approx(sa, abs=(1e-5 if fmt == "f32" else 0.5 * (m.num_verts + m.num_faces) / 255))
    # 1x1: a closed connected mesh becomes one group, a constant
    vals = np.array([b.level(e, 2)[0, 0, 0] for e in range(m.num_edges)])
    assert np.ptp(vals) == 0.0


# ----------------------------------------------------------- number formats

def _rand_f32(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n).astype(np.float32) * np.exp2(rng.integers(-20, 5, n)).astype(np.float32)
    return x


def test_f16_rounding_matches_numpy():
    for x in _rand_f32(20000, 1).astype(np.float64):
        assert oracle.round_format("f16", x) == float(np.float16(x))
    # values between float32 grid points still round once, to nearest even
    rng = np.random.default_rng(2)
    for x in rng.uniform(-1, 1, 20000):
        assert oracle.round_format("f16", x) == float(np.float16(x))


def test_bf16_rounding_matches_torch():
    x = _rand_f32(20000, 3)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.round_format("bf16", float(v)) for v in x])
    np.testing.assert_array_equal(got, ref)
    # exact halfway cases in double: ties go to the even code
    assert oracle.round_format("bf16", 1 + 2.0 ** -8) == 1.0
    assert oracle.round_format("bf16", 1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6


def test_e4m3_rounding_matches_torch_and_saturates():
    rng = np.random.default_rng(4)
    x = (rng.uniform(-448, 448, 20000) * np.exp2(rng.integers(-12, 1, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = np.array([oracle.round_format("e4m3", float(v)) for v in x])
    np.testing.assert_array_equal(got, ref)
    assert oracle.round_format("e4m3", 448.0) == 448.0
    assert oracle.round_format("e4m3", 10000.0) == 448.0
    assert oracle.round_format("e4m3", -470.0) == -448.0
    assert oracle.round_format("e4m3", 2.0 ** -9) == 2.0 ** -9          # smallest subnormal
    assert oracle.round_format("e4m3", 2.0 ** -11) == 0.0               # ties to even (zero)


@pytest.mark.parametrize("fmt,nbits,tdt", [("f16", 16, torch.float16), ("bf16", 16, torch.bfloat16),
                                            ("e4m3", 8, torch.float8_e4m3fn)])
def test_decode_every_code(fmt, nbits, tdt):
    codes = np.arange(1 << nbits, dtype=np.uint32)
    store = codes.astype(np.uint16 if nbits == 16 else np.uint8)
    itype = torch.int16 if nbits == 16 else torch.uint8
    ref = torch.from_numpy(store.view(np.int16) if nbits == 16 else store).view(itype)
    ref = ref.view(tdt).to(torch.float64).numpy()
    got = np.array([oracle.decode(fmt, int(c)) for c in codes])
    same = (got == ref) | (np.isnan(got) & np.isnan(ref))
    assert same.all()
    # encode is the inverse on every finite code
    for c in codes[np.isfinite(got)]:
        if got[c] == 0 and c != 0:
            continue          # negative zero
        assert oracle.encode(fmt, got[c]) == c


@pytest.mark.parametrize("fmt,u", [("f16", 2.0 ** -11), ("bf16", 2.0 ** -8), ("e4m3", 2.0 ** -4)])
def test_quantised_error_within_format_bound(fmt, u):
    """|stored - original| <= u_fmt * max|T| per texture (round to nearest
    with unit roundoff u_fmt, after scaling by the texture maximum), plus the
    subnormal floor, which is far smaller here."""
    m = _mesh()
    log2n = (np.arange(m.num_edges) % 3 + 1).astype(np.int32)
    lvl0 = syn.texels_f32(log2n, 4, seed=5) * 3.0 - 1.0
    ref = oracle.prepare_textures(m, log2n, lvl0, 4, "f32", oracle.BUILD_MIPS)
    q = oracle.prepare_textures(m, log2n, lvl0, 4, fmt, oracle.BUILD_MIPS)
    for e in range(m.num_edges):
        a, b = int(ref.toff[e]) * 4, int(ref.toff[e + 1]) * 4
        mx = np.abs(ref.values[a:b]).max()
        assert np.abs(q.values[a:b] - ref.values[a:b]).max() <= u * mx * (1 + 1e-6)
        if fmt == "e4m3":
            assert q.scales[e] == np.float32(mx / 448.0)
        else:
            assert q.scales[e] == np.float32(mx)


def test_pool_layout_f32_and_u8():
    m = _mesh()
    log2n = (np.arange(m.num_edges) % 3).astype(np.int32)
    for fmt, C, size in (("f32", 3, 4), ("u8", 3, 1)):
        gen = syn.texels_u8 if fmt == "u8" else syn.texels_f32
        t = oracle.prepare_textures(m, log2n, gen(log2n, C, 6), C, fmt, oracle.BUILD_MIPS)
        pool, poff = t.pool_bytes()
        off = 0
        for e in range(m.num_edges):
            assert poff[e] == off and off % 16 == 0
            n = int(log2n[e])
            cnt = sum(4 ** (n - l) for l in range(n + 1)) * C
            dt = np.float32 if fmt == "f32" else np.uint8
            stored = pool[off:off + cnt * size].view(dt).astype(np.float64)
            exp = t.values[int(t.toff[e]) * C:int(t.toff[e + 1]) * C]
            np.testing.assert_array_equal(stored, exp if fmt == "f32" else np.round(exp * 255))
            off += -(-cnt * size // 16) * 16
        assert poff[-1] == off == pool.shape[0]
