"""Rendering the intrinsic triangulation (htex_geometry_*, htex_rasterize,
htex_displace): argument marshalling for the CUDA kernels, plus camera
matrices."""
from __future__ import annotations

import ctypes

import numpy as np

from . import Mesh, Textures, _stream
from ._lib import check, load


class Geometry:
    def __init__(self, mesh: Mesh, positions, stream=None):
        self._lib = load()
        pos = np.ascontiguousarray(positions, np.float32).reshape(-1, 3)
        h = ctypes.c_void_p()
        check(self._lib.htex_geometry_create(mesh._h, pos.ctypes.data_as(ctypes.c_void_p), _stream(stream),
                                             ctypes.byref(h)), "htex_geometry_create")
        self._h = h
        self.H = mesh.H

    def triangle_vertices(self, stream=None):
        import torch
        out = torch.empty((self.H, 3, 3), dtype=torch.float32, device="cuda")
        check(self._lib.htex_triangle_vertices(self._h, ctypes.c_void_p(out.data_ptr()), _stream(stream)),
              "htex_triangle_vertices")
        return out

    def rasterize(self, view_proj, width: int, height: int, queries=None, depth=None, stream=None):
        """Queries (int32 [height * width, 4], CUDA) and optional depth."""
        import torch
        m = np.ascontiguousarray(view_proj, np.float32).reshape(16)
        if queries is None:
            queries = torch.empty((width * height, 4), dtype=torch.int32, device="cuda")
        dptr = ctypes.c_void_p(depth.data_ptr()) if depth is not None else None
        check(self._lib.htex_rasterize(self._h, m.ctypes.data_as(ctypes.c_void_p), int(width), int(height),
                                       ctypes.c_void_p(queries.data_ptr()), dptr, _stream(stream)),
              "htex_rasterize")
        return queries

    def rasterize_aniso(self, view_proj, width: int, height: int, queries=None, depth=None, stream=None):
        """Anisotropic queries (int32 [height * width, 8], CUDA, laid out as
        htex_query_aniso) and optional depth."""
        import torch
        m = np.ascontiguousarray(view_proj, np.float32).reshape(16)
        if queries is None:
            queries = torch.empty((width * height, 8), dtype=torch.int32, device="cuda")
        dptr = ctypes.c_void_p(depth.data_ptr()) if depth is not None else None
        check(self._lib.htex_rasterize_aniso(self._h, m.ctypes.data_as(ctypes.c_void_p), int(width), int(height),
                                             ctypes.c_void_p(queries.data_ptr()), dptr, _stream(stream)),
              "htex_rasterize_aniso")
        return queries

    def displace(self, tex: Textures, tess: int, scale: float, channel: int = 0, stream=None):
        import torch
        K = (tess + 1) * (tess + 2) // 2
        out = torch.empty((self.H, K, 3), dtype=torch.float32, device="cuda")
        check(self._lib.htex_displace(self._h, tex._h, int(tess), float(scale), int(channel),
                                      ctypes.c_void_p(out.data_ptr()), _stream(stream)), "htex_displace")
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.htex_geometry_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def camera(eye, target, up, fovy_deg, aspect, near, far):
    """Row-major view-projection matrix (see htex_synth.look_at / perspective)."""
    import htex_synth as syn
    return syn.perspective(fovy_deg, aspect, near, far) @ syn.look_at(eye, target, up)
