"""CPU tests of libhtex's host logic: ABI exports, halfedge construction and
texture preparation, compared bit for bit with the oracle (integer, index
and byte work) on the same seeded inputs."""
import numpy as np
import pytest

import htex_synth as syn
import oracle
import paper_2207_05618_gb300 as hx
from paper_2207_05618_gb300 import _lib


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2207_05618_gb300 import build
    build.build()


def test_library_exports_every_declared_function():
    lib = _lib.load()
    names = _lib.header_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib._SIGNATURES), "binding and header disagree"
    assert lib.htex_status_string(0) == b"ok"
    assert lib.htex_status_string(2) == b"non-manifold mesh"


MESHES = {
    "fig2": lambda: syn.fig2_faces(),
    "quad": lambda: syn.single_quad(),
    "cube": lambda: syn.cube()[:3],
    "cylinder": lambda: syn.cylinder(around=24, rows=9, seed=3)[:3],
    "sphere": lambda: syn.uv_sphere(slices=16, rings=12, seed=4)[:3],
}


@pytest.mark.parametrize("name", list(MESHES))
def test_mesh_matches_oracle(name):
    fs, fv, V = MESHES[name]()
    mo = oracle.mesh_from_faces(fs, fv, V)
    ml = hx.Mesh(fs, fv, V)
    he = ml.halfedges()
    for k in ("twin", "next", "prev", "vert", "edge", "face"):
        np.testing.assert_array_equal(he[k], getattr(mo, k), err_msg=k)
    assert (ml.H, ml.E, ml.num_boundary) == (mo.H, mo.num_edges, mo.num_boundary)


def test_fig2_table_adopted(fig2_table):
    t = fig2_table
    m = hx.Mesh.from_halfedges(t["Twin"], t["Next"], t["Prev"], t["Vert"], t["Edge"], t["Face"], 7, 3)
    assert (m.H, m.E, m.num_boundary) == (12, 9, 6)
    he = m.halfedges()
    assert list(he["edge"]) == t["Edge"]


def test_mesh_rejections(fig2_table):
    with pytest.raises(hx.HtexError) as e:
        hx.Mesh([3, 3], [0, 1, 2, 0, 1, 3], 4)
    assert e.value.code == 2
    for fs, fv, V in (([2], [0, 1], 2), ([3], [0, 1, 5], 3), ([3], [0, 0, 1], 2)):
        with pytest.raises(hx.HtexError) as e:
            hx.Mesh(fs, fv, V)
        assert e.value.code == 1
    t = {k: list(v) for k, v in fig2_table.items()}
    bad = dict(t)
    bad["Twin"] = list(t["Twin"])
    bad["Twin"][0] = 5              # not an involution
    with pytest.raises(hx.HtexError):
        hx.Mesh.from_halfedges(bad["Twin"], t["Next"], t["Prev"], t["Vert"], t["Edge"], t["Face"], 7, 3)
    bad = list(t["Edge"])
    bad[6] = 2                      # twins with different edges
    with pytest.raises(hx.HtexError):
        hx.Mesh.from_halfedges(t["Twin"], t["Next"], t["Prev"], t["Vert"], bad, t["Face"], 7, 3)


def _both(name, log2n_fn, fmt, C, flags, seed=0, levels_given=False):
    fs, fv, V = MESHES[name]()
    mo = oracle.mesh_from_faces(fs, fv, V)
    ml = hx.Mesh(fs, fv, V)
    log2n = log2n_fn(mo.num_edges)
    if levels_given:
        cnt = sum(((4 ** (int(n) + 1)) - 1) // 3 for n in log2n)
        rng = np.random.default_rng(seed)
        tex = (rng.integers(0, 256, cnt * C).astype(np.uint8) if fmt == "u8"
               else rng.random(cnt * C, dtype=np.float32))
    else:
        tex = (syn.texels_u8 if fmt == "u8" else syn.texels_f32)(log2n, C, seed)
        if fmt not in ("u8", "f32"):
            tex = tex * 4.0 - 1.5            # signed data for the scaled formats
    to = oracle.prepare_textures(mo, log2n, tex, C, fmt, flags & 7, levels_given=levels_given)
    pool_o, poff = to.pool_bytes()
    lflags = flags | (hx.LEVELS_GIVEN if levels_given else 0)
    pool_l, scales_l = hx.Textures.prepare(ml, log2n, tex, C, fmt, lflags)
    total, offs = hx.Textures.layout(ml, log2n, C, fmt)
    return pool_o, poff, pool_l, scales_l, to, total, offs


UNIFORM = {0: lambda E: np.zeros(E, np.int32), 3: lambda E: np.full(E, 3, np.int32)}


def _mixed(E):
    return (np.arange(E) * 7 % 5).astype(np.int32)


@pytest.mark.parametrize("fmt", ["f32", "u8", "f16", "bf16", "e4m3"])
@pytest.mark.parametrize("flags", [hx.BUILD_MIPS, hx.BUILD_MIPS | hx.MIRROR_BOUNDARY,
                                   hx.BUILD_MIPS | hx.MIRROR_BOUNDARY | hx.FIX_CORNERS,
                                   hx.BUILD_MIPS | hx.FIX_CORNERS])
@pytest.mark.parametrize("mesh", ["cylinder", "sphere"])
def test_prepared_pool_bitexact(fmt, flags, mesh):
    C = 4 if fmt != "f32" else 3
    pool_o, poff, pool_l, scales_l, to, total, offs = _both(mesh, _mixed, fmt, C, flags, seed=7)
    np.testing.assert_array_equal(offs, poff)
    assert total == pool_o.shape[0]
    np.testing.assert_array_equal(scales_l, to.scales)
    if not np.array_equal(pool_l, pool_o):
        bad = np.nonzero(pool_l != pool_o)[0]
        pytest.fail(f"{bad.size} bytes differ, first at {bad[:8]}")


@pytest.mark.parametrize("fmt", ["f32", "u8", "e4m3"])
def test_prepared_pool_levels_given(fmt):
    pool_o, poff, pool_l, *_ = _both("cylinder", _mixed, fmt, 2, hx.MIRROR_BOUNDARY, seed=3,
                                     levels_given=True)
    np.testing.assert_array_equal(pool_l, pool_o)


def test_prepare_rejects_bad_arguments():
    fs, fv, V = MESHES["cube"]()
    m = hx.Mesh(fs, fv, V)
    with pytest.raises(hx.HtexError) as e:
        hx.Textures.prepare(m, np.full(m.E, 16, np.int32), np.zeros(10, np.float32), 4)
    assert e.value.code == 3
    with pytest.raises(hx.HtexError):
        hx.Textures.prepare(m, np.zeros(m.E, np.int32), np.zeros(m.E * 5, np.float32), 5)
    with pytest.raises(hx.HtexError):   # level 0 only needs BUILD_MIPS
        hx.Textures.prepare(m, np.zeros(m.E, np.int32), np.zeros(m.E, np.float32), 1, "f32", 0)
