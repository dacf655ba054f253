"""Htex FP64 CPU oracle — TEST INFRASTRUCTURE ONLY.

A plain, slow restatement of per-halfedge texturing (Barbier & Dupuy 2022)
in double precision, used to check the CUDA library.  Only ``tests/``, the
``smoke()`` check in ``__graft_entry__`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA path: the
arithmetic lives in ``htex_oracle.c`` (built with gcc, loaded with ctypes);
this module only marshals numpy arrays.

Functions and the passages they follow:
  mesh_from_faces      Section 2 (halfedge operators, Fig. 2), Section 3.2
                       (edges, boundary halfedges paired with themselves)
  prepare_textures     Section 4.3 (one square texture per edge, boundary
                       mirroring), Section 4.4 (corner pre-processing); mip
                       generation and reduced-precision storage are readings
                       of what the paper leaves to the graphics API
  lookup               Section 4.4, Alg. 3 with Alg. 2
  lookup_grad          the derivative of Alg. 3, which is linear in the texels
  triangle_vertices    Alg. 1 (Section 3.1)
  vertex_normals       normals of the input mesh for displacement (Section 5.1)
  rasterize            visibility of the intrinsic triangulation through a
                       pinhole camera, with barycentrics and footprints
                       (the rendering of Section 4.4, written as a plain
                       per-pixel nearest-hit search)
  displace             displaced lattice vertices (Section 5.1)

Every function is pinned by tests in ``tests/test_oracle_*.py`` against the
Fig. 2 table, hand-derived values, closed forms and invariants.  Parity is
unpinned for nothing in this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "htex_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "htex_oracle.so")

FMT = {"f32": 0, "u8": 1, "f16": 2, "bf16": 3, "e4m3": 4}
BUILD_MIPS, MIRROR_BOUNDARY, FIX_CORNERS = 1, 2, 4

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64 = ctypes.c_int32, ctypes.c_int64
            lib.orc_mesh_from_faces.argtypes = [i32, P, P, i32, i32, P, P, P, P, P, P, P]
            lib.orc_mesh_from_faces.restype = ctypes.c_int
            lib.orc_edge_owner.argtypes = [i32, P, P, P]
            lib.orc_texels_in_chain.argtypes = [i32]
            lib.orc_texels_in_chain.restype = i64
            lib.orc_texture_offsets.argtypes = [i32, P, P]
            lib.orc_build_mips.argtypes = [i32, P, P, i32, i32, P]
            lib.orc_mirror_boundary.argtypes = [i32, P, P, i32, P, P, i32, P]
            lib.orc_fix_corners.argtypes = [i32, P, P, i32, i32, i32, P, P, P, P, P, i32, i32, P]
            lib.orc_quantize.argtypes = [i32, P, P, i32, i32, P, P, P]
            lib.orc_lookup.argtypes = [i32, P, P, P, P, P, P, P, i32, i64, P, P, P, P, P, P, i32]
            lib.orc_lookup_grad.argtypes = [i32, P, P, P, P, P, P, P, i32, i64, P, P, P, P, P, P]
            lib.orc_lookup_aniso.argtypes = [i32, P, P, P, P, P, P, P, i32, i64, P, P, P, P, i32, P, i32]
            lib.orc_pool_offsets.argtypes = [i32, P, i32, i32, P]
            lib.orc_pool_offsets.restype = i64
            lib.orc_pack_pool.argtypes = [i32, P, P, P, i32, i32, P, P, P]
            for name in ("orc_round_f16", "orc_round_bf16", "orc_round_e4m3"):
                getattr(lib, name).argtypes = [ctypes.c_double]
                getattr(lib, name).restype = ctypes.c_double
            lib.orc_triangle_vertices.argtypes = [i32, P, P, P, P]
            lib.orc_vertex_normals.argtypes = [i32, i32, i32, P, P, P, P, P, P]
            lib.orc_encode.argtypes = [i32, ctypes.c_double]
            lib.orc_encode.restype = ctypes.c_uint32
            lib.orc_decode.argtypes = [i32, ctypes.c_uint32]
            lib.orc_decode.restype = ctypes.c_double
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleError(ValueError):
    pass


@dataclass
class Mesh:
    twin: np.ndarray
    next: np.ndarray
    prev: np.ndarray
    vert: np.ndarray
    edge: np.ndarray
    face: np.ndarray
    num_verts: int
    num_faces: int
    num_edges: int

    @property
    def H(self) -> int:
        return int(self.twin.shape[0])

    @property
    def num_boundary(self) -> int:
        return int((self.twin < 0).sum())

    def owner(self) -> np.ndarray:
        """Per edge: the larger id of its halfedge pair (Alg. 2), or the boundary halfedge."""
        o = np.empty(self.num_edges, np.int32)
        _load().orc_edge_owner(self.H, _p(self.twin), _p(self.edge), _p(o))
        return o


def mesh_from_faces(face_sizes, face_verts, num_verts: int) -> Mesh:
    fs = np.ascontiguousarray(face_sizes, np.int32)
    fv = np.ascontiguousarray(face_verts, np.int32)
    F, H = int(fs.shape[0]), int(fs.sum())
    if fv.shape[0] != H:
        raise OracleError("face_verts length != sum(face_sizes)")
    arrs = [np.empty(H, np.int32) for _ in range(6)]
    E = ctypes.c_int32(0)
    rc = _load().orc_mesh_from_faces(F, _p(fs), _p(fv), int(num_verts), H, *[_p(a) for a in arrs],
                                     ctypes.byref(E))
    if rc == 1:
        raise OracleError("invalid faces")
    if rc == 2:
        raise OracleError("non-manifold: directed edge used twice")
    return Mesh(*arrs, num_verts=int(num_verts), num_faces=F, num_edges=int(E.value))


def mesh_from_halfedges(twin, next, prev, vert, edge, face, num_verts: int, num_faces: int) -> Mesh:
    a = [np.ascontiguousarray(x, np.int32) for x in (twin, next, prev, vert, edge, face)]
    return Mesh(*a, num_verts=int(num_verts), num_faces=int(num_faces),
                num_edges=int(a[4].max()) + 1 if a[4].size else 0)


@dataclass
class Textures:
    """Oracle-side textures: fp64 values of what is stored, all levels."""
    log2n: np.ndarray          # [E] int32
    toff: np.ndarray           # [E+1] int64 texel offsets (oracle layout)
    values: np.ndarray         # [T*C] float64: the value every stored texel decodes to
    channels: int
    fmt: str
    scales: np.ndarray         # [E] float32 (1 where unused)
    codes: np.ndarray | None = None   # reduced-precision codes, oracle layout
    flags: int = 0
    extra: dict = field(default_factory=dict)

    def level(self, e: int, l: int) -> np.ndarray:
        """View of level l of texture e as [N][N][C] (row j, column i)."""
        n = int(self.log2n[e])
        base = int(self.toff[e]) + sum((1 << (n - k)) ** 2 for k in range(l))
        N = 1 << (n - l)
        return self.values[base * self.channels:(base + N * N) * self.channels].reshape(N, N, self.channels)

    def pool_bytes(self) -> tuple[np.ndarray, np.ndarray]:
        """The stored pool in the documented byte layout, and per-texture byte offsets."""
        lib = _load()
        E = int(self.log2n.shape[0])
        poff = np.empty(E + 1, np.int64)
        total = lib.orc_pool_offsets(E, _p(self.log2n), self.channels, FMT[self.fmt], _p(poff))
        pool = np.zeros(max(int(total), 1), np.uint8)
        raw = self.extra["raw"]        # stored numbers before decoding (bytes or floats)
        codes = self.codes if self.codes is not None else np.zeros(1, np.uint32)
        lib.orc_pack_pool(E, _p(self.log2n), _p(self.toff), _p(poff), self.channels, FMT[self.fmt],
                          _p(raw), _p(codes), _p(pool))
        return pool[:int(total)], poff


def texture_offsets(log2n) -> np.ndarray:
    ln = np.ascontiguousarray(log2n, np.int32)
    toff = np.empty(ln.shape[0] + 1, np.int64)
    _load().orc_texture_offsets(int(ln.shape[0]), _p(ln), _p(toff))
    return toff


def prepare_textures(mesh: Mesh, log2n, texels, channels: int, fmt: str = "f32",
                     flags: int = BUILD_MIPS, levels_given: bool = False) -> Textures:
    """What the stored textures hold, in fp64.

    ``texels``: per edge, in edge order, level 0 only (``levels_given`` False)
    or every level (True), row-major [N][N][C]; float data for f32/f16/bf16/
    e4m3, byte values for u8.  Steps, each optional by flag: boundary
    mirroring of level 0, box mips, mirroring of every level, corner
    pre-processing per resolution, then quantisation with per-texture scale.
    """
    lib = _load()
    C = int(channels)
    ln = np.ascontiguousarray(log2n, np.int32)
    E = int(ln.shape[0])
    if E != mesh.num_edges:
        raise OracleError("one texture per edge")
    toff = texture_offsets(ln)
    tex = np.zeros(int(toff[E]) * C, np.float64)
    src = np.ascontiguousarray(texels).reshape(-1)
    if fmt == "u8":
        src = src.astype(np.uint8).astype(np.float64)
    else:
        src = src.astype(np.float32).astype(np.float64)
    pos = 0
    for e in range(E):
        n = int(ln[e])
        cnt = (int(toff[e + 1] - toff[e]) if levels_given else (1 << n) ** 2) * C
        tex[int(toff[e]) * C:int(toff[e]) * C + cnt] = src[pos:pos + cnt]
        pos += cnt
    if pos != src.shape[0]:
        raise OracleError("texel count does not match the resolutions")
    owner = mesh.owner()
    is_u8 = 1 if fmt == "u8" else 0
    mirrored = 1 if flags & MIRROR_BOUNDARY else 0
    if not levels_given and (flags & BUILD_MIPS):
        if mirrored:
            # level 0 first, so that the built mips inherit the symmetry
            lib.orc_mirror_boundary(E, _p(ln), _p(toff), C, _p(owner), _p(mesh.twin), 1, _p(tex))
        lib.orc_build_mips(E, _p(ln), _p(toff), C, is_u8, _p(tex))
    elif not levels_given:
        raise OracleError("level-0 texels without BUILD_MIPS: levels must be given")
    if mirrored:
        lib.orc_mirror_boundary(E, _p(ln), _p(toff), C, _p(owner), _p(mesh.twin), 0, _p(tex))
    if flags & FIX_CORNERS:
        lib.orc_fix_corners(E, _p(ln), _p(toff), C, is_u8, mirrored, _p(owner), _p(mesh.twin),
                            _p(mesh.next), _p(mesh.vert), _p(mesh.face), mesh.num_verts,
                            mesh.num_faces, _p(tex))
    scales = np.ones(E, np.float32)
    codes = None
    raw = tex.copy()
    if fmt in ("f16", "bf16", "e4m3"):
        codes = np.zeros(tex.shape[0], np.uint32)
        lib.orc_quantize(E, _p(ln), _p(toff), C, FMT[fmt], _p(tex), _p(codes), _p(scales))
        values = tex
    elif fmt == "u8":
        values = tex / 255.0
    elif fmt == "f32":
        values = tex
    else:
        raise OracleError(f"unknown format {fmt}")
    return Textures(ln, toff, values, C, fmt, scales, codes, flags, {"raw": raw})


def _queries(queries):
    h, u, v, f = queries
    h = np.ascontiguousarray(h, np.int32)
    u = np.ascontiguousarray(u, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    f = np.ascontiguousarray(f, np.float64)
    assert h.shape == u.shape == v.shape == f.shape
    return h, u, v, f


def lookup(mesh: Mesh, tex: Textures, queries, nthreads: int = 1, return_weight: bool = False):
    """Alg. 3 for every query (h, u, v, footprint); returns fp64 [n][C]
    (and the summed normalisation weight per query when asked)."""
    h, u, v, f = _queries(queries)
    n = int(h.shape[0])
    out = np.empty((n, tex.channels), np.float64)
    w = np.empty(n, np.float64) if return_weight else None
    _load().orc_lookup(mesh.H, _p(mesh.twin), _p(mesh.next), _p(mesh.prev), _p(mesh.edge),
                       _p(tex.log2n), _p(tex.toff), _p(tex.values), tex.channels, n,
                       _p(h), _p(u), _p(v), _p(f), _p(out), _p(w) if w is not None else None,
                       int(nthreads))
    return (out, w) if return_weight else out


def lookup_aniso(mesh: Mesh, tex: Textures, queries, kmax: int, nthreads: int = 1) -> np.ndarray:
    """Anisotropic lookups (the reading of Section 5.1's anisotropic filter
    written out in ``htex_oracle.c``): queries (h, u, v, du/dx, dv/dx, du/dy,
    dv/dy), the derivatives taken as float32 like the stored query; returns
    fp64 [n][C]."""
    h, u, v, dudx, dvdx, dudy, dvdy = queries
    h = np.ascontiguousarray(h, np.int32)
    u = np.ascontiguousarray(u, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    d = np.ascontiguousarray(np.stack([dudx, dvdx, dudy, dvdy], 1), np.float32)
    n = int(h.shape[0])
    assert u.shape == v.shape == h.shape and d.shape == (n, 4)
    out = np.empty((n, tex.channels), np.float64)
    _load().orc_lookup_aniso(mesh.H, _p(mesh.twin), _p(mesh.next), _p(mesh.prev), _p(mesh.edge),
                             _p(tex.log2n), _p(tex.toff), _p(tex.values), tex.channels, n,
                             _p(h), _p(u), _p(v), _p(d), int(kmax), _p(out), int(nthreads))
    return out


def lookup_grad(mesh: Mesh, tex: Textures, queries, grad_out) -> np.ndarray:
    """d(sum grad_out * lookup)/d(stored texel value), fp64, oracle layout [T*C]."""
    h, u, v, f = _queries(queries)
    g = np.ascontiguousarray(grad_out, np.float64).reshape(h.shape[0], tex.channels)
    grad = np.zeros_like(tex.values)
    _load().orc_lookup_grad(mesh.H, _p(mesh.twin), _p(mesh.next), _p(mesh.prev), _p(mesh.edge),
                            _p(tex.log2n), _p(tex.toff), _p(tex.values), tex.channels,
                            int(h.shape[0]), _p(h), _p(u), _p(v), _p(f), _p(g), _p(grad))
    return grad


def grad_to_pool_layout(tex: Textures, grad: np.ndarray, dtype_bytes: int) -> np.ndarray:
    """Re-index an oracle-layout per-texel array into pool element order.

    The pool holds texture e at byte offset poff[e] (16-byte padded); a
    pool-shaped gradient has one float per stored element at the same
    element index, so padding elements stay zero."""
    E = int(tex.log2n.shape[0])
    poff = np.empty(E + 1, np.int64)
    _load().orc_pool_offsets(E, _p(tex.log2n), tex.channels, FMT[tex.fmt], _p(poff))
    out = np.zeros(int(poff[E]) // dtype_bytes, np.float64)
    C = tex.channels
    for e in range(E):
        a, b = int(tex.toff[e]) * C, int(tex.toff[e + 1]) * C
        s = int(poff[e]) // dtype_bytes
        out[s:s + (b - a)] = grad[a:b]
    return out


def round_format(fmt: str, x: float) -> float:
    lib = _load()
    return {"f16": lib.orc_round_f16, "bf16": lib.orc_round_bf16, "e4m3": lib.orc_round_e4m3}[fmt](float(x))


def encode(fmt: str, rounded: float) -> int:
    return int(_load().orc_encode(FMT[fmt], float(rounded)))


def decode(fmt: str, bits: int) -> float:
    return float(_load().orc_decode(FMT[fmt], int(bits)))


# ----------------------------------------------------------- rendering side

def triangle_vertices(mesh: Mesh, positions) -> np.ndarray:
    """Alg. 1 for every halfedge: [H][3][3] = (v0, v1, v2)."""
    pos = np.ascontiguousarray(positions, np.float64).reshape(-1, 3)
    tri = np.empty((mesh.H, 3, 3), np.float64)
    _load().orc_triangle_vertices(mesh.H, _p(mesh.next), _p(mesh.vert), _p(pos), _p(tri))
    return tri


def vertex_normals(mesh: Mesh, positions):
    pos = np.ascontiguousarray(positions, np.float64).reshape(-1, 3)
    vn = np.empty((mesh.num_verts, 3), np.float64)
    fn = np.empty((mesh.num_faces, 3), np.float64)
    _load().orc_vertex_normals(mesh.H, mesh.num_verts, mesh.num_faces, _p(mesh.next), _p(mesh.vert),
                               _p(mesh.face), _p(pos), _p(vn), _p(fn))
    return vn, fn


def _project(view_proj, pts):
    """Homogeneous clip coordinates of points [..., 3] (row-vector convention: clip = M @ [p, 1])."""
    M = np.asarray(view_proj, np.float64).reshape(4, 4)
    ph = np.concatenate([pts, np.ones(pts.shape[:-1] + (1,))], -1)
    return ph @ M.T


def rasterize(mesh: Mesh, positions, view_proj, width: int, height: int, derivatives: bool = False):
    """Per pixel centre (x + 1/2, y + 1/2), the intrinsic triangle seen
    first: the triangle whose interior (barycentrics >= 0) contains the
    centre with the smallest depth z/w in [-1, 1]; its perspective-correct
    barycentrics (u on Vert(h), v on Vert(Next h), Section 4.2) and the
    footprint max(|d(u,v)/dx|, |d(u,v)/dy|) in uv units per pixel, from the
    same triangle's barycentrics at the centres one pixel right and down.
    Returns h [H_px, W_px] (-1 where empty), u, v, footprint, depth, and the
    barycentric margin and depth gap to the runner-up (for deciding which
    pixels have a unique answer).  With 'derivatives', also the differences
    du/dx, dv/dx, du/dy, dv/dy of the barycentrics at those neighbouring
    centres (the footprint of an anisotropic lookup).  Plain loops over
    pixels, vectorised over triangles: small images only."""
    tri = triangle_vertices(mesh, positions)           # v0 = Vert(Next h), v1 = centroid, v2 = Vert(h)
    clip = _project(view_proj, tri)                    # [H][3][4]
    w = clip[..., 3]
    ndc = clip[..., :3] / w[..., None]
    sx = (ndc[..., 0] * 0.5 + 0.5) * width
    sy = (0.5 - ndc[..., 1] * 0.5) * height
    hh = np.full((height, width), -1, np.int64)
    out = {k: np.full((height, width), np.nan)
           for k in ("u", "v", "f", "depth", "margin", "gap", "dudx", "dvdx", "dudy", "dvdy")}

    def bary(px, py):
        # screen-space barycentrics of (px, py) in every triangle, then perspective-corrected
        x0, y0, x1, y1, x2, y2 = sx[:, 0], sy[:, 0], sx[:, 1], sy[:, 1], sx[:, 2], sy[:, 2]
        den = (y1 - y2) * (x0 - x2) + (x2 - x1) * (y0 - y2)
        with np.errstate(divide="ignore", invalid="ignore"):
            l0 = ((y1 - y2) * (px - x2) + (x2 - x1) * (py - y2)) / den
            l1 = ((y2 - y0) * (px - x2) + (x0 - x2) * (py - y2)) / den
        l2 = 1 - l0 - l1
        lam = np.stack([l0, l1, l2], 1)
        z = (lam * ndc[..., 2]).sum(1)
        pw = lam / w
        pc = pw / pw.sum(1, keepdims=True)
        # (u, v, w) weigh (v2, v0, v1): u = pc[2], v = pc[0]
        return lam, z, pc[:, 2], pc[:, 0]

    valid_tri = np.all(w > 0, 1)
    for y in range(height):
        for x in range(width):
            lam, z, u, v = bary(x + 0.5, y + 0.5)
            inside = valid_tri & np.all(lam >= 0, 1) & (z >= -1) & (z <= 1)
            idx = np.nonzero(inside)[0]
            if idx.size == 0:
                continue
            order = idx[np.lexsort((idx, z[idx]))]
            k = order[0]
            hh[y, x] = k
            out["u"][y, x], out["v"][y, x], out["depth"][y, x] = u[k], v[k], z[k]
            out["margin"][y, x] = lam[k].min()
            out["gap"][y, x] = (z[order[1]] - z[k]) if order.size > 1 else np.inf
            _, _, ux, vx = bary(x + 1.5, y + 0.5)
            _, _, uy, vy = bary(x + 0.5, y + 1.5)
            out["f"][y, x] = max(np.hypot(ux[k] - u[k], vx[k] - v[k]), np.hypot(uy[k] - u[k], vy[k] - v[k]))
            out["dudx"][y, x], out["dvdx"][y, x] = ux[k] - u[k], vx[k] - v[k]
            out["dudy"][y, x], out["dvdy"][y, x] = uy[k] - u[k], vy[k] - v[k]
    res = (hh, out["u"], out["v"], out["f"], out["depth"], out["margin"], out["gap"])
    if derivatives:
        res += (out["dudx"], out["dvdx"], out["dudy"], out["dvdy"])
    return res


def displace(mesh: Mesh, tex: Textures, positions, tess: int, scale: float, channel: int = 0):
    """Displacement (Section 5.1): for every halfedge triangle the lattice
    (u, v) = (i/T, j/T), i + j <= T, of the intrinsic triangle, displaced
    along the interpolated normal (vertex normals at Vert(h) and Vert(Next h),
    the face normal at the centroid) by scale times the lookup (level 0).
    Returns [H][K][3] positions, K = (T+1)(T+2)/2, lattice in (i, j) order."""
    tri = triangle_vertices(mesh, positions)
    vn, fn = vertex_normals(mesh, positions)
    ij = [(i, j) for i in range(tess + 1) for j in range(tess + 1 - i)]
    K = len(ij)
    u = np.array([i / tess for i, _ in ij])
    v = np.array([j / tess for _, j in ij])
    hs = np.repeat(np.arange(mesh.H, dtype=np.int32), K)
    uu, vv = np.tile(u, mesh.H), np.tile(v, mesh.H)
    d = lookup(mesh, tex, (hs, uu, vv, np.zeros_like(uu)))[:, channel].reshape(mesh.H, K)
    wgt = np.stack([u, v, 1 - u - v], 1)                               # weights of v2, v0, v1
    P = (wgt[None, :, 0, None] * tri[:, None, 2] + wgt[None, :, 1, None] * tri[:, None, 0]
         + wgt[None, :, 2, None] * tri[:, None, 1])
    n2 = vn[mesh.vert]                       # at Vert(h)
    n0 = vn[mesh.vert[mesh.next]]            # at Vert(Next h)
    n1 = fn[mesh.face]                       # at the centroid
    N = wgt[None, :, 0, None] * n2[:, None] + wgt[None, :, 1, None] * n0[:, None] + wgt[None, :, 2, None] * n1[:, None]
    N = N / np.linalg.norm(N, axis=-1, keepdims=True)
    return P + scale * d[..., None] * N
