"""GPU parity of the rendering side (htex_triangle_vertices,
htex_rasterize, htex_displace) against the FP64 oracle."""
import numpy as np
import pytest

import htex_synth as syn
import oracle
import paper_2207_05618_gb300 as hx
from paper_2207_05618_gb300 import render

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2207_05618_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _sphere():
    fs, fv, V, pos = syn.uv_sphere(slices=14, rings=10, seed=5)
    return fs, fv, V, pos


def test_triangle_vertices_match_alg1():
    for fs, fv, V, pos in (_sphere(), syn.cylinder(around=20, rows=6, seed=2)):
        mo = oracle.mesh_from_faces(fs, fv, V)
        g = render.Geometry(hx.Mesh(fs, fv, V), pos)
        got = g.triangle_vertices().cpu().numpy()
        ref = oracle.triangle_vertices(mo, pos.astype(np.float32).astype(np.float64))
        np.testing.assert_allclose(got, ref, atol=2e-6)


@pytest.mark.parametrize("W,H", [(96, 64), (61, 37)])
def test_rasterizer_matches_reference(W, H):
    """Pixels whose nearest triangle is clear (barycentric margin and depth
    gap above float rounding) carry the oracle's halfedge, barycentrics and
    footprint; every other covered pixel names a triangle that covers it
    at the nearest depth up to rounding; empty pixels agree."""
    fs, fv, V, pos = _sphere()
    mo = oracle.mesh_from_faces(fs, fv, V)
    M = syn.perspective(40.0, W / H, 0.3, 10.0) @ syn.look_at([2.3, -1.1, 0.9], [0, 0, 0], [0, 0, 1])
    g = render.Geometry(hx.Mesh(fs, fv, V), pos)
    depth = torch.empty(W * H, dtype=torch.float32, device="cuda")
    q = g.rasterize(M, W, H, depth=depth).cpu().numpy()
    pos32 = pos.astype(np.float32).astype(np.float64)
    hh, u, v, f, dref, margin, gap = oracle.rasterize(mo, pos32, M.astype(np.float32).astype(np.float64), W, H)
    gh = q[:, 0].reshape(H, W)
    gu = q[:, 1].copy().view(np.float32).reshape(H, W)
    gv = q[:, 2].copy().view(np.float32).reshape(H, W)
    gf = q[:, 3].copy().view(np.float32).reshape(H, W)
    clear = (hh >= 0) & (margin > 1e-4) & (gap > 1e-4)
    assert clear.sum() > 0.5 * (hh >= 0).sum() > 0
    np.testing.assert_array_equal(gh[clear], hh[clear])
    np.testing.assert_allclose(gu[clear], u[clear], atol=2e-4)
    np.testing.assert_allclose(gv[clear], v[clear], atol=2e-4)
    np.testing.assert_allclose(gf[clear], f[clear], rtol=2e-3, atol=1e-6)
    np.testing.assert_allclose(depth.cpu().numpy().reshape(H, W)[clear], dref[clear], atol=1e-5)
    # empty pixels: far from every triangle in the reference
    empty = gh < 0
    assert np.all((hh[empty] < 0) | (margin[empty] < 1e-4))
    # the rest: the GPU's triangle covers the pixel (up to rounding)
    tri = oracle.triangle_vertices(mo, pos32)
    for y, x in np.argwhere((gh >= 0) & ~clear):
        k = gh[y, x]
        P = gu[y, x] * tri[k, 2] + gv[y, x] * tri[k, 0] + (1 - gu[y, x] - gv[y, x]) * tri[k, 1]
        c = M @ np.append(P, 1.0)
        assert abs((c[0] / c[3] * 0.5 + 0.5) * W - (x + 0.5)) < 1e-2
        assert abs((0.5 - c[1] / c[3] * 0.5) * H - (y + 0.5)) < 1e-2
        if hh[y, x] >= 0:
            assert c[2] / c[3] <= dref[y, x] + 1e-4


@pytest.mark.parametrize("W,H", [(96, 64), (61, 37)])
def test_anisotropic_rasterizer_matches_reference(W, H):
    """htex_rasterize_aniso: the same halfedges and barycentrics as
    htex_rasterize (bit for bit), and on clear pixels the oracle's screen
    derivatives of the barycentrics; empty pixels carry h = -1."""
    fs, fv, V, pos = _sphere()
    mo = oracle.mesh_from_faces(fs, fv, V)
    M = syn.perspective(40.0, W / H, 0.3, 10.0) @ syn.look_at([2.3, -1.1, 0.9], [0, 0, 0], [0, 0, 1])
    g = render.Geometry(hx.Mesh(fs, fv, V), pos)
    qi = g.rasterize(M, W, H).cpu().numpy()
    qa = g.rasterize_aniso(M, W, H).cpu().numpy()
    np.testing.assert_array_equal(qa[:, :3], qi[:, :3])
    pos32 = pos.astype(np.float32).astype(np.float64)
    r = oracle.rasterize(mo, pos32, M.astype(np.float32).astype(np.float64), W, H, derivatives=True)
    hh, margin, gap = r[0], r[5], r[6]
    clear = (hh >= 0) & (margin > 1e-4) & (gap > 1e-4)
    assert clear.sum() > 0
    for col, ref in zip(range(4, 8), r[7:11]):
        got = qa[:, col].copy().view(np.float32).reshape(H, W)
        np.testing.assert_allclose(got[clear], ref[clear], rtol=2e-3, atol=2e-6)
    empty = qa[:, 0] < 0
    assert np.all(qa[empty][:, 4:] == 0)


def test_frame_pipeline_full_hd():
    """1920x1080 frame of the closed sphere filling the view: every pixel
    inside the silhouette gets a valid query, the lookup returns finite
    values there and NaN outside."""
    fs, fv, V, pos = _sphere()
    mesh = hx.Mesh(fs, fv, V)
    log2n = np.full(mesh.E, 5, np.int32)
    tex = hx.Textures.upload(mesh, log2n, syn.texels_u8(log2n, 4, seed=1), 4, "u8", hx.BUILD_MIPS)
    g = render.Geometry(mesh, pos)
    M = syn.perspective(45.0, 1920 / 1080, 0.3, 10.0) @ syn.look_at([2.2, 0, 0], [0, 0, 0], [0, 0, 1])
    q = g.rasterize(M, 1920, 1080)
    out = hx.lookup(tex, q).cpu().numpy()
    valid = q[:, 0].cpu().numpy() >= 0
    assert 0.2 < valid.mean() < 0.9
    assert np.all(np.isfinite(out[valid])) and np.all(np.isnan(out[~valid]))


def test_displacement_matches_oracle_and_is_crack_free():
    fs, fv, V, pos = syn.uv_sphere(slices=9, rings=7, seed=2)
    mo = oracle.mesh_from_faces(fs, fv, V)
    mesh = hx.Mesh(fs, fv, V)
    log2n = np.full(mesh.E, 3, np.int32)
    flags = hx.BUILD_MIPS | hx.FIX_CORNERS
    tex_np = syn.texels_f32(log2n, 2, 3)
    tl = hx.Textures.upload(mesh, log2n, tex_np, 2, "f32", flags)
    to = oracle.prepare_textures(mo, log2n, tex_np, 2, "f32", flags)
    g = render.Geometry(mesh, pos)
    T = 4
    got = g.displace(tl, T, 0.3, channel=1).cpu().numpy()
    pos32 = pos.astype(np.float32).astype(np.float64)
    ref = oracle.displace(mo, to, pos32, T, 0.3, channel=1)
    np.testing.assert_allclose(got, ref, atol=2e-5)
    P0 = oracle.displace(mo, to, pos32, T, 0.0).reshape(-1, 3)
    key = np.round(P0 * 1e6).astype(np.int64)
    _, inv = np.unique(key, axis=0, return_inverse=True)
    flat = got.reshape(-1, 3)
    for grp in np.unique(inv):
        pts = flat[inv == grp]
        assert np.abs(pts - pts[0]).max() < 2e-5
