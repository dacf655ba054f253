"""Oracle pins for the rendering side: Alg. 1 (Section 3.1), normals of the
input mesh, the reference rasteriser and displacement (Section 5.1)."""
import numpy as np
import pytest

import htex_synth as syn
import oracle


def test_alg1_fig2_example():
    """Section 3.1: the vertices of t7 are Vert(h8), the mean of the five
    vertices of the pentagon h7..h11, and Vert(h7)."""
    fs, fv, V = syn.fig2_faces()
    m = oracle.mesh_from_faces(fs, fv, V)
    pos = np.random.default_rng(0).normal(size=(V, 3))
    tri = oracle.triangle_vertices(m, pos)
    np.testing.assert_allclose(tri[7, 0], pos[m.vert[8]], atol=1e-15)
    np.testing.assert_allclose(tri[7, 1], pos[[m.vert[k] for k in range(7, 12)]].mean(0), atol=1e-15)
    np.testing.assert_allclose(tri[7, 2], pos[m.vert[7]], atol=1e-15)


def test_alg1_triangles_tile_a_planar_polygon():
    """The intrinsic triangles of a planar polygon cover it: their areas sum
    to the shoelace area."""
    k = 7
    th = np.sort(np.random.default_rng(1).uniform(0, 2 * np.pi, k))
    pos = np.stack([np.cos(th) * 2, np.sin(th), np.zeros(k)], 1)
    m = oracle.mesh_from_faces([k], list(range(k)), k)
    tri = oracle.triangle_vertices(m, pos)
    area = sum(0.5 * abs(np.cross(t[0] - t[1], t[2] - t[1])[2]) for t in tri)
    x, y = pos[:, 0], pos[:, 1]
    shoelace = 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))
    assert area == pytest.approx(shoelace, abs=1e-12)


def test_cube_normals():
    fs, fv, V, pos = syn.cube()
    m = oracle.mesh_from_faces(fs, fv, V)
    vn, fn = oracle.vertex_normals(m, pos)
    centre = np.array([0.5, 0.5, 0.5])
    for k in range(8):
        d = pos[k] - centre
        np.testing.assert_allclose(vn[k], d / np.linalg.norm(d), atol=1e-15)
    assert np.allclose(np.abs(fn).sum(1), 1.0) and np.allclose(np.abs(fn).max(1), 1.0)


def _camera(W, H):
    return syn.perspective(32.0, W / H, 0.5, 10.0) @ syn.look_at([2.2, -1.7, 1.6], [0.5, 0.5, 0.5], [0, 0, 1])


def test_rasterizer_round_trip_and_nearest_hit():
    """Every covered pixel's (h, u, v) names a surface point that projects
    back onto the pixel centre at the recorded depth (perspective-correct
    barycentrics), and the closed cube seen from outside only shows faces
    turned towards the camera."""
    fs, fv, V, pos = syn.cube()
    m = oracle.mesh_from_faces(fs, fv, V)
    W, H = 40, 30
    M = _camera(W, H)
    hh, u, v, f, depth, margin, gap = oracle.rasterize(m, pos, M, W, H)
    tri = oracle.triangle_vertices(m, pos)
    eye = np.array([2.2, -1.7, 1.6])
    covered = np.argwhere(hh >= 0)
    assert 0.2 * W * H < len(covered) < W * H
    for y, x in covered:
        k = hh[y, x]
        P = u[y, x] * tri[k, 2] + v[y, x] * tri[k, 0] + (1 - u[y, x] - v[y, x]) * tri[k, 1]
        c = M @ np.append(P, 1.0)
        sx = (c[0] / c[3] * 0.5 + 0.5) * W
        sy = (0.5 - c[1] / c[3] * 0.5) * H
        assert abs(sx - (x + 0.5)) < 1e-9 and abs(sy - (y + 0.5)) < 1e-9
        assert abs(c[2] / c[3] - depth[y, x]) < 1e-9
        n = np.cross(tri[k, 0] - tri[k, 1], tri[k, 2] - tri[k, 1])
        assert np.dot(n, eye - P) != 0
        assert f[y, x] > 0


def test_constant_displacement_moves_along_unit_normals():
    fs, fv, V, pos = syn.uv_sphere(slices=10, rings=7, seed=1)
    m = oracle.mesh_from_faces(fs, fv, V)
    log2n = np.full(m.num_edges, 2, np.int32)
    t = oracle.prepare_textures(m, log2n, np.full(m.num_edges * 16, 0.25, np.float32), 1, "f32",
                                oracle.BUILD_MIPS)
    P0 = oracle.displace(m, t, pos, 3, 0.0)
    P1 = oracle.displace(m, t, pos, 3, 2.0)
    np.testing.assert_allclose(np.linalg.norm(P1 - P0, axis=-1), 0.5, atol=1e-12)


def test_displacement_is_crack_free_with_corner_preprocessing():
    """Section 5.1 / 4.4: with corner pre-processing, lattice vertices that
    coincide before displacement coincide after it (no cracks), on edges
    between triangles, around vertices and at face centroids."""
    fs, fv, V, pos = syn.uv_sphere(slices=9, rings=7, seed=2)
    m = oracle.mesh_from_faces(fs, fv, V)
    log2n = np.full(m.num_edges, 3, np.int32)
    t = oracle.prepare_textures(m, log2n, syn.texels_f32(log2n, 1, 3), 1, "f32",
                                oracle.BUILD_MIPS | oracle.FIX_CORNERS)
    T = 4
    P0 = oracle.displace(m, t, pos, T, 0.0).reshape(-1, 3)
    P1 = oracle.displace(m, t, pos, T, 0.3).reshape(-1, 3)
    key = np.round(P0 * 1e9).astype(np.int64)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    shared = cnt[inv] > 1
    assert shared.sum() > 0.3 * len(P0)
    for g in np.unique(inv[shared]):
        pts = P1[inv == g]
        assert np.abs(pts - pts[0]).max() < 1e-12
    # without corner pre-processing the vertices crack
    t2 = oracle.prepare_textures(m, log2n, syn.texels_f32(log2n, 1, 3), 1, "f32", oracle.BUILD_MIPS)
    P2 = oracle.displace(m, t2, pos, T, 0.3).reshape(-1, 3)
    spread = max(np.abs(P2[inv == g] - P2[inv == g][0]).max() for g in np.unique(inv[shared]))
    assert spread > 1e-3


def test_rasterizer_derivatives_project_to_neighbour_pixels():
    """The derivatives are differences of the same triangle's barycentrics
    at the centres one pixel right and one pixel down: the surface points at
    (u + du/dx, v + dv/dx) and (u + du/dy, v + dv/dy) project onto those
    centres, and the isotropic footprint is the longer of the two."""
    fs, fv, V, pos = syn.cube()
    m = oracle.mesh_from_faces(fs, fv, V)
    W, H = 32, 24
    M = _camera(W, H)
    hh, u, v, f, depth, margin, gap, dudx, dvdx, dudy, dvdy = oracle.rasterize(m, pos, M, W, H, derivatives=True)
    tri = oracle.triangle_vertices(m, pos)
    covered = np.argwhere(hh >= 0)
    assert len(covered) > 0.2 * W * H
    for y, x in covered:
        k = hh[y, x]
        for du, dv, ex, ey in ((dudx[y, x], dvdx[y, x], x + 1.5, y + 0.5), (dudy[y, x], dvdy[y, x], x + 0.5, y + 1.5)):
            uu, vv = u[y, x] + du, v[y, x] + dv
            P = uu * tri[k, 2] + vv * tri[k, 0] + (1 - uu - vv) * tri[k, 1]
            c = M @ np.append(P, 1.0)
            assert abs((c[0] / c[3] * 0.5 + 0.5) * W - ex) < 1e-9
            assert abs((0.5 - c[1] / c[3] * 0.5) * H - ey) < 1e-9
        assert f[y, x] == max(np.hypot(dudx[y, x], dvdx[y, x]), np.hypot(dudy[y, x], dvdy[y, x]))
