"""Seeded synthetic inputs for Htex lookups: meshes, texels, queries.

This module produces inputs only (face lists, texel arrays, query arrays)
and holds none of the method's arithmetic: no halfedge construction, no
parameterisation, no filtering.  Both the FP64 oracle and the CUDA library
consume what it returns.

Recipes (workload shapes follow the paper's production assets, which are
mostly quads with a few triangles, some larger polygons and boundary edges,
paper Section 5.1):
  fig2_faces       the 3-face mesh of the paper's Fig. 2 table
  single_quad      one quad, four boundary halfedges
  cube             closed unit cube, 6 quads (24 halfedges, 12 edges)
  cylinder         open cylinder grid: `around` x `rows` quads, a fraction
                   split into 2 triangles along a random diagonal, and runs
                   of adjacent quads merged into 5- to 8-gons
  uv_sphere        closed sphere: rings of quads with triangle fans at the
                   poles, with the same splits and merges
  texels_*         level-0 texel data per edge, in edge order
  queries          halfedge ids uniform, barycentrics uniform on the
                   triangle (folding), footprint 0 or log-uniform
"""
from __future__ import annotations

import numpy as np


def fig2_faces():
    """Faces read off the Vert/Face columns of the paper's Fig. 2 table."""
    face_sizes = np.array([4, 3, 5], np.int32)
    face_verts = np.array([3, 2, 1, 0, 3, 4, 2, 1, 2, 4, 5, 6], np.int32)
    return face_sizes, face_verts, 7


def single_quad():
    return np.array([4], np.int32), np.array([0, 1, 2, 3], np.int32), 4


def cube():
    """Unit cube, vertex k at (k&1, (k>>1)&1, (k>>2)&1), outward CCW quads."""
    faces = [[0, 2, 3, 1], [4, 5, 7, 6], [0, 1, 5, 4], [2, 6, 7, 3], [0, 4, 6, 2], [1, 3, 7, 5]]
    pos = np.array([[k & 1, (k >> 1) & 1, (k >> 2) & 1] for k in range(8)], np.float64)
    return (np.array([4] * 6, np.int32), np.array(sum(faces, []), np.int32), 8, pos)


def _band(bottom, top, rng, split_frac, merge_frac, wrap=True):
    """Faces of one band of quads between two vertex rings of equal length.

    Cell c spans bottom[c], bottom[c+1], top[c+1], top[c].  Returns a list of
    vertex lists (consistent orientation)."""
    A = len(bottom)
    ncell = A if wrap else A - 1

    def b(c):
        return bottom[c % A]

    def t(c):
        return top[c % A]

    split = rng.random(ncell) < split_frac
    diag = rng.integers(0, 2, ncell)
    used = np.zeros(ncell, bool)
    faces = []
    c = 0
    while c < ncell:
        if not used[c] and not split[c] and rng.random() < merge_frac:
            # choose a run shape among those that fit without wrapping
            options = []
            for k, tri in ((1, True), (2, False), (2, True), (3, False)):
                last = c + k - 1 + (1 if tri else 0)
                if last >= ncell:
                    continue
                if any(split[c:c + k]) or any(used[c:c + k]):
                    continue
                if tri and not (split[c + k] and diag[c + k] == 0 and not used[c + k]):
                    continue
                options.append((k, tri))
            if options:
                k, tri = options[int(rng.integers(0, len(options)))]
                poly = [b(c + i) for i in range(k + 1)]
                if tri:
                    poly.append(t(c + k + 1))
                poly += [t(c + k - i) for i in range(k + 1)]
                faces.append(poly)
                used[c:c + k] = True
                if tri:
                    # the split cell keeps its other triangle
                    cc = c + k
                    faces.append([b(cc), b(cc + 1), t(cc + 1)])
                    used[cc] = True
                c += k + (1 if tri else 0)
                continue
        if not used[c]:
            bl, br, tr, tl = b(c), b(c + 1), t(c + 1), t(c)
            if split[c]:
                if diag[c] == 0:
                    faces += [[bl, br, tr], [bl, tr, tl]]
                else:
                    faces += [[bl, br, tl], [br, tr, tl]]
            else:
                faces.append([bl, br, tr, tl])
            used[c] = True
        c += 1
    return faces


def _pack(faces):
    sizes = np.array([len(f) for f in faces], np.int32)
    verts = np.array([v for f in faces for v in f], np.int32)
    return sizes, verts


def cylinder(around=256, rows=460, split_frac=0.3, merge_frac=0.11, seed=0):
    """Open cylinder: (rows + 1) rings of `around` vertices; boundary rings at both ends."""
    rng = np.random.default_rng(seed)
    faces = []
    for r in range(rows):
        bottom = [r * around + c for c in range(around)]
        top = [(r + 1) * around + c for c in range(around)]
        faces += _band(bottom, top, rng, split_frac, merge_frac, wrap=True)
    sizes, verts = _pack(faces)
    V = (rows + 1) * around
    th = 2 * np.pi * (np.arange(V) % around) / around
    pos = np.stack([np.cos(th), np.sin(th), (np.arange(V) // around) / around], 1)
    return sizes, verts, V, pos


def uv_sphere(slices=160, rings=160, split_frac=0.1, merge_frac=0.05, seed=0):
    """Closed sphere: poles 0 and 1, rings 1..rings-1 of `slices` vertices."""
    rng = np.random.default_rng(seed)

    def vid(i, j):
        return 2 + (i - 1) * slices + (j % slices)

    faces = [[0, vid(1, j), vid(1, j + 1)] for j in range(slices)]
    for i in range(1, rings - 1):
        bottom = [vid(i, j) for j in range(slices)]
        top = [vid(i + 1, j) for j in range(slices)]
        # band cells here are [b(c), t(c), t(c+1), b(c+1)] reversed w.r.t. _band's
        # orientation; feed the rings swapped so orientation stays consistent
        faces += _band(top, bottom, rng, split_frac, merge_frac, wrap=True)
    faces += [[1, vid(rings - 1, j + 1), vid(rings - 1, j)] for j in range(slices)]
    sizes, verts = _pack(faces)
    V = 2 + (rings - 1) * slices
    pos = np.zeros((V, 3))
    pos[0] = (0, 0, 1)
    pos[1] = (0, 0, -1)
    for i in range(1, rings):
        phi = np.pi * i / rings
        th = 2 * np.pi * np.arange(slices) / slices
        pos[vid(i, 0):vid(i, 0) + slices] = np.stack(
            [np.sin(phi) * np.cos(th), np.sin(phi) * np.sin(th), np.full(slices, np.cos(phi))], 1)
    return sizes, verts, V, pos


def texels_f32(log2n, channels, seed=0):
    """Level-0 texels, U[0,1) float32, all edges concatenated (edge order)."""
    rng = np.random.default_rng(seed)
    count = int(sum((1 << int(n)) ** 2 for n in np.asarray(log2n))) * channels
    return rng.random(count, dtype=np.float32)


def texels_u8(log2n, channels, seed=0):
    """Level-0 texels, uniform random bytes, all edges concatenated."""
    rng = np.random.default_rng(seed)
    count = int(np.sum((np.int64(1) << (2 * np.asarray(log2n, np.int64))))) * channels
    return np.frombuffer(rng.bytes(count), np.uint8).copy()


def texels_smooth(log2n, channels, seed=0, waves=8):
    """Level-0 texels from a sum of random sinusoids in per-texture (x, y).

    Smooth inside every texture; used as a fitting target, not for parity."""
    rng = np.random.default_rng(seed)
    out = []
    k = rng.uniform(-4, 4, (waves, 2)) * np.pi
    ph = rng.uniform(0, 2 * np.pi, (waves, channels))
    amp = rng.uniform(0.05, 0.2, (waves, channels))
    for e, n in enumerate(np.asarray(log2n)):
        N = 1 << int(n)
        x = (np.arange(N) + 0.5) / N
        X, Y = np.meshgrid(x, x)           # row j = y, column i = x
        val = np.full((N, N, channels), 0.5)
        shift = 0.37 * e
        for w in range(waves):
            arg = (k[w, 0] * X + k[w, 1] * Y + shift)[..., None] + ph[w]
            val += amp[w] * np.sin(arg)
        out.append(val.astype(np.float32).reshape(-1))
    return np.concatenate(out)


def queries(H, n, seed=0, footprint="zero", lo=-8.0, hi=0.0):
    """n queries: h ~ U{0..H-1}; (u, v) uniform on the triangle by folding
    (u + v > 1 -> (1 - u, 1 - v)); footprint 0, or 2^U(lo, hi) ('loguniform')."""
    rng = np.random.default_rng(seed)
    h = rng.integers(0, H, n, dtype=np.int64).astype(np.int32)
    u = rng.random(n, dtype=np.float32)
    v = rng.random(n, dtype=np.float32)
    fold = (u + v) > 1.0
    u[fold], v[fold] = 1.0 - u[fold], 1.0 - v[fold]
    if footprint == "zero":
        f = np.zeros(n, np.float32)
    elif footprint == "loguniform":
        f = np.exp2(rng.uniform(lo, hi, n)).astype(np.float32)
    else:
        raise ValueError(footprint)
    return h, u, v, f


def edge_queries(H, N, footprints=(0.0,)):
    """Adversarial queries for every halfedge: (u, v) on the lattice of
    multiples of 1/(2N) inside the closed triangle (texel centres, texel
    borders, the triangle's sides and corners), for each footprint."""
    g = np.arange(2 * N + 1, dtype=np.float64) / (2 * N)
    U, Vv = np.meshgrid(g, g)
    keep = (U + Vv) <= 1.0 + 1e-12
    uu, vv = U[keep], Vv[keep]
    hs, us, vs, fs = [], [], [], []
    for f in footprints:
        for h in range(H):
            hs.append(np.full(uu.shape, h, np.int32))
            us.append(uu)
            vs.append(vv)
            fs.append(np.full(uu.shape, f))
    cat = np.concatenate
    return (cat(hs).astype(np.int32), cat(us).astype(np.float32), cat(vs).astype(np.float32),
            cat(fs).astype(np.float32))


def invalid_queries(H):
    """Queries outside the domain: bad halfedge ids and barycentrics off the triangle."""
    h = np.array([-1, H, 2 ** 31 - 1, 0, 0, 0, 0, H - 1], np.int32)
    u = np.array([0.2, 0.2, 0.2, -0.5, 0.9, 2.0, np.nan, 0.3], np.float32)
    v = np.array([0.2, 0.2, 0.2, 0.3, 0.9, -1.0, 0.1, np.inf], np.float32)
    f = np.array([0, 0, 0, 0, 0, -1.0, np.nan, np.inf], np.float32)
    return h, u, v, f


def cylinder_with_halfedges(target_H, seed=0):
    """An open cylinder (splits and merges as `cylinder`) with about target_H halfedges."""
    around = max(8, int(round((target_H / 4.5) ** 0.5)))
    rows = max(2, int(round(target_H / (4.53 * around))))
    return cylinder(around=around, rows=rows, seed=seed)


def serving_assets(count=8, h_lo=1_000, h_hi=500_000):
    """Serving workload assets: halfedge counts log-spaced over [h_lo, h_hi]
    (both ends included); texture resolution 128, 128, 64, 64, 32, 32, 16, 16
    from the smallest mesh up (total texels stay a few GB), formats
    alternating RGBA8 / FP16.  Returns a list of dicts."""
    hs = np.exp(np.linspace(np.log(h_lo), np.log(h_hi), count))
    res = [128, 128, 64, 64, 32, 32, 16, 16]
    out = []
    for k, H in enumerate(hs):
        fs, fv, V, _ = cylinder_with_halfedges(H, seed=100 + k)
        out.append({"faces": (fs, fv, V), "log2n": int(np.log2(res[k % len(res)])),
                    "dtype": "u8" if k % 2 == 0 else "f16", "seed": 200 + k})
    return out


def poisson_requests(count, rate, num_assets, lo=1_000, hi=4_000_000, seed=0):
    """Request stream: arrival times of a Poisson process with 'rate'
    requests/s, sizes log-uniform over [lo, hi] queries, uniform asset tags."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, count))
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), count)).astype(np.int64)
    assets = rng.integers(0, num_assets, count)
    return arrivals - arrivals[0], sizes, assets


# ----------------------------------------------------------------- cameras

def look_at(eye, target, up):
    """World-to-view matrix (right-handed, looking down -z)."""
    eye, target, up = (np.asarray(a, np.float64) for a in (eye, target, up))
    f = target - eye
    f /= np.linalg.norm(f)
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = s, u, -f
    m[:3, 3] = -m[:3, :3] @ eye
    return m


def perspective(fovy_deg, aspect, near, far):
    """GL-style projection: visible depth z/w in [-1, 1]."""
    t = 1.0 / np.tan(np.radians(fovy_deg) / 2)
    m = np.zeros((4, 4))
    m[0, 0], m[1, 1] = t / aspect, t
    m[2, 2], m[2, 3] = (far + near) / (near - far), 2 * far * near / (near - far)
    m[3, 2] = -1.0
    return m
