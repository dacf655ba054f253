"""Host-side helpers of bench.py (CPU): the algorithmic byte counts its
roofline entries divide by, and the tap counter behind them, checked on
queries whose taps follow from the bilinear rule by hand (texel centres
pick one tap per axis, interior points of a texel two; a query far from
every side of its triangle reads only its own quad)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import htex_synth as syn  # noqa: E402
import oracle  # noqa: E402


def _cube_halfedges():
    fs, fv, V, _ = syn.cube()
    m = oracle.mesh_from_faces(fs, fv, V)
    return {"twin": m.twin, "next": m.next, "prev": m.prev}, m.H


def test_algorithmic_bytes_definitions():
    ab = bench.algorithmic_bytes(6.5, 4)
    assert ab["hot_path"] == 16 + 16 + 48 + 26.0       # query, output, three 16-byte records, taps
    assert ab["packed"] == 16 + 16 + 16 + 26.0       # one pre-evaluated record
    assert ab["taps"] == 6.5


def test_mean_taps_interior_queries():
    """(u, v) = (1/3, 1/3) on 16x16 textures: the own quad's coordinates
    are (1/3, 1/3) or (2/3, 2/3), inside a texel and 5.3 texels from the
    quad's sides, so the Next and Prev fetches (half a texel wide across
    the shared side) read nothing: 4 taps at level 0, 8 with two levels."""
    he, H = _cube_halfedges()
    n = 64
    h = np.arange(n, dtype=np.int32) % H
    u = np.full(n, 1 / 3, np.float32)
    v = np.full(n, 1 / 3, np.float32)
    assert bench.mean_taps(he, 4, (h, u, v, np.zeros(n, np.float32))) == 4.0
    # footprint 2^-2.5 quad widths: lambda = 1.5, levels 1 and 2 (8x8, 4x4), weights 1/2 each
    f = np.full(n, 2.0 ** -2.5, np.float32)
    assert bench.mean_taps(he, 4, (h, u, v, f)) == 8.0


def test_mean_taps_texel_centre_and_edge():
    """A query at a texel centre of its own quad has a = b = 0: one tap of
    nonzero weight.  A query on the triangle's side toward Next(h) (u = 0)
    also reads the Next quad's row: half a texel across, so weight 1/2 on
    the row's taps."""
    he, H = _cube_halfedges()
    N = 16
    # own coordinate (x, y) = (u, v) when h > Twin(h), else (1 - u, 1 - v):
    # both are texel centres when u, v are centres
    big = [g for g in range(H) if g > he["twin"][g]]
    h = np.array(big, np.int32)
    u = np.full(len(h), 3.5 / N, np.float32)
    v = np.full(len(h), 5.5 / N, np.float32)
    assert bench.mean_taps(he, 4, (h, u, v, np.zeros(len(h), np.float32))) == 1.0
    # u = 0, v = 5.25/N: the own x = 0 gives s = -1/2, columns -1 and 0 of
    # which only column 0 is in bounds, and y between rows 4 and 5: 2 own
    # taps; the Next fetch at (v, -u) = (5.25/N, 0) reads row 0 at columns 4
    # and 5: 2 taps; the Prev fetch at (-v, u) lies 5.25 texels outside: none
    u0 = np.zeros(len(h), np.float32)
    v0 = np.full(len(h), 5.25 / N, np.float32)
    assert bench.mean_taps(he, 4, (h, u0, v0, np.zeros(len(h), np.float32))) == 4.0
