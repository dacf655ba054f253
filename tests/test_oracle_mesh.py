"""Oracle pins: halfedge construction (paper Section 2, Fig. 2; Section 3)."""
import numpy as np
import pytest

import htex_synth as syn
import oracle


def test_fig2_columns_reproduced(fig2_table):
    fs, fv, V = syn.fig2_faces()
    m = oracle.mesh_from_faces(fs, fv, V)
    t = fig2_table
    assert m.H == 12
    for name, arr in (("Twin", m.twin), ("Next", m.next), ("Prev", m.prev),
                      ("Vert", m.vert), ("Face", m.face)):
        assert list(arr) == t[name], name
    # Edge column: equal up to a twin-consistent relabelling (a bijection)
    pairs = set(zip(m.edge.tolist(), t["Edge"]))
    assert len(pairs) == 9 == m.num_edges
    assert len({a for a, _ in pairs}) == 9 and len({b for _, b in pairs}) == 9
    assert m.num_boundary == 6          # H = 12, B = 6, E = (H + B) / 2 = 9


def test_fig2_text_facts():
    """Facts stated in Sections 3.1 and 3.2 about halfedges h7, h4, h1."""
    fs, fv, V = syn.fig2_faces()
    m = oracle.mesh_from_faces(fs, fv, V)
    assert m.next[7] == 8 and m.prev[7] == 11 and m.twin[7] == 1
    assert m.prev[4] == 6 and m.next[4] == 5 and m.twin[4] == -1
    assert m.edge[7] == m.edge[1]
    # boundary triangles have exactly two neighbours: Prev and Next
    assert m.twin[4] < 0 and m.prev[4] >= 0 and m.next[4] >= 0


def test_cube_closed():
    fs, fv, V, _ = syn.cube()
    m = oracle.mesh_from_faces(fs, fv, V)
    assert m.H == 24 and m.num_edges == 12 and m.num_boundary == 0
    h = np.arange(24)
    assert np.all(m.twin[m.twin] == h)
    assert np.all(m.vert[m.next[m.twin]] == m.vert)       # twin runs the other way
    assert np.all(m.edge[m.twin] == m.edge)


@pytest.mark.parametrize("gen", ["cylinder", "sphere"])
def test_generated_meshes_consistent(gen):
    if gen == "cylinder":
        fs, fv, V, _ = syn.cylinder(around=16, rows=12, seed=3)
    else:
        fs, fv, V, _ = syn.uv_sphere(slices=12, rings=10, seed=3)
    m = oracle.mesh_from_faces(fs, fv, V)
    h = np.arange(m.H)
    inner = m.twin >= 0
    assert np.all(m.twin[m.twin[inner]] == h[inner])
    assert np.all(m.next[m.prev] == h) and np.all(m.prev[m.next] == h)
    assert m.num_edges == (m.H + m.num_boundary) // 2
    assert set(np.bincount(m.edge).tolist()) <= {1, 2}
    if gen == "sphere":
        assert m.num_boundary == 0
    else:
        assert m.num_boundary == 2 * 16
    assert fs.max() >= 5 and fs.min() == 3      # merged polygons and split triangles exist


def test_reject_nonmanifold_and_bad_faces():
    # two faces using the directed edge 0 -> 1
    with pytest.raises(oracle.OracleError):
        oracle.mesh_from_faces([3, 3], [0, 1, 2, 0, 1, 3], 4)
    with pytest.raises(oracle.OracleError):
        oracle.mesh_from_faces([2], [0, 1], 2)
    with pytest.raises(oracle.OracleError):
        oracle.mesh_from_faces([3], [0, 1, 5], 3)
    with pytest.raises(oracle.OracleError):
        oracle.mesh_from_faces([3], [0, 0, 1], 2)


def test_asset_scale_cylinder_size():
    """The asset-scale workload: about 520k halfedges, 260k edges."""
    fs, fv, V, _ = syn.cylinder()
    H = int(fs.sum())
    assert abs(H - 520_000) / 520_000 < 0.01
    frac_tri = float((fs == 3).mean())
    frac_big = float((fs >= 5).mean())
    assert 0.3 < frac_tri < 0.5 and 0.01 < frac_big < 0.1
