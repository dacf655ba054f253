"""Htex batched seamless filtered lookups on GB300 (sm_103a).

Python face of libhtex (C ABI in include/htex.h): argument marshalling
only, every step of the lookup runs in the library's CUDA kernels.
PyTorch supplies device memory and streams.

    mesh = Mesh(face_sizes, face_verts, num_verts)          # Section 2, Fig. 2
    tex = Textures.upload(mesh, log2_res, texels, channels=4, dtype="u8")
    out = lookup(tex, queries)          # queries: int32 [n, 4] (h, u, v, footprint bits)
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import (BUILD_MIPS, DTYPES, ELEM_SIZE, FIX_CORNERS, LEVELS_GIVEN, LOOKUP_BIN,
                   LOOKUP_GLOBAL, MIRROR_BOUNDARY, HtexError, check, load)

__all__ = ["Mesh", "Textures", "lookup", "lookup_host", "lookup_backward", "lookup_aniso", "sort_queries",
           "gather_results", "pack_queries", "pack_queries_aniso", "HtexLookup",
           "HtexError", "BUILD_MIPS", "MIRROR_BOUNDARY", "FIX_CORNERS", "LEVELS_GIVEN",
           "LOOKUP_BIN", "LOOKUP_GLOBAL"]


def _np(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Mesh:
    """Host-side halfedge mesh (htex_mesh_create / _create_from_halfedges)."""

    def __init__(self, face_sizes=None, face_verts=None, num_verts: int = 0, *, _handle=None):
        self._lib = load()
        if _handle is not None:
            self._h = _handle
        else:
            fs, fv = _np(face_sizes, np.int32), _np(face_verts, np.int32)
            h = ctypes.c_void_p()
            check(self._lib.htex_mesh_create(_ptr(fs), int(fs.shape[0]), _ptr(fv), int(num_verts),
                                             ctypes.byref(h)), "htex_mesh_create")
            self._h = h
        vals = [ctypes.c_int32() for _ in range(5)]
        check(self._lib.htex_mesh_info(self._h, *[ctypes.byref(v) for v in vals]), "htex_mesh_info")
        self.H, self.E, self.num_boundary, self.num_verts, self.num_faces = [v.value for v in vals]

    @classmethod
    def from_halfedges(cls, twin, next, prev, vert, edge, face, num_verts: int, num_faces: int):
        lib = load()
        arrs = [_np(a, np.int32) for a in (twin, next, prev, vert, edge, face)]
        h = ctypes.c_void_p()
        check(lib.htex_mesh_create_from_halfedges(*[_ptr(a) for a in arrs], int(arrs[0].shape[0]),
                                                  int(num_verts), int(num_faces), ctypes.byref(h)),
              "htex_mesh_create_from_halfedges")
        return cls(_handle=h)

    def halfedges(self) -> dict:
        arrs = {k: np.empty(self.H, np.int32) for k in ("twin", "next", "prev", "vert", "edge", "face")}
        check(self._lib.htex_mesh_get_halfedges(self._h, *[_ptr(a) for a in arrs.values()]),
              "htex_mesh_get_halfedges")
        return arrs

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.htex_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def _texel_array(texels, dtype: str) -> np.ndarray:
    return _np(texels, np.uint8 if dtype == "u8" else np.float32).reshape(-1)


class Textures:
    """Device-resident mesh + textures (htex_textures_*)."""

    def __init__(self, handle, mesh: Mesh):
        self._lib = load()
        self._h = handle
        ch, dt, H, E = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        pb, db = ctypes.c_int64(), ctypes.c_int64()
        check(self._lib.htex_textures_info(handle, ctypes.byref(ch), ctypes.byref(dt), ctypes.byref(H),
                                           ctypes.byref(E), ctypes.byref(pb), ctypes.byref(db)),
              "htex_textures_info")
        self.channels, self.H, self.E = ch.value, H.value, E.value
        self.dtype = {v: k for k, v in DTYPES.items()}[dt.value]
        self.pool_bytes, self.device_bytes = pb.value, db.value
        self.mesh = mesh

    @staticmethod
    def layout(mesh: Mesh, log2_res, channels: int, dtype: str):
        lib = load()
        ln = _np(log2_res, np.int32)
        total = ctypes.c_int64()
        offs = np.empty(mesh.E + 1, np.int64)
        check(lib.htex_textures_layout(mesh._h, int(channels), DTYPES[dtype], _ptr(ln), ctypes.byref(total),
                                       _ptr(offs)), "htex_textures_layout")
        return int(total.value), offs

    @staticmethod
    def prepare(mesh: Mesh, log2_res, texels, channels: int, dtype: str = "f32", flags: int = BUILD_MIPS):
        """Host-side preparation: the stored pool bytes and per-texture scales."""
        lib = load()
        ln = _np(log2_res, np.int32)
        total, _ = Textures.layout(mesh, ln, channels, dtype)
        pool = np.empty(max(total, 1), np.uint8)
        scales = np.empty(max(mesh.E, 1), np.float32)
        tx = _texel_array(texels, dtype)
        check(lib.htex_textures_prepare(mesh._h, int(channels), DTYPES[dtype], _ptr(ln), _ptr(tx), int(flags),
                                        _ptr(pool), _ptr(scales)), "htex_textures_prepare")
        return pool[:total], scales[:mesh.E]

    @classmethod
    def upload(cls, mesh: Mesh, log2_res, texels, channels: int, dtype: str = "f32",
               flags: int = BUILD_MIPS, stream=None):
        lib = load()
        ln = _np(log2_res, np.int32)
        tx = _texel_array(texels, dtype)
        h = ctypes.c_void_p()
        check(lib.htex_textures_upload(mesh._h, int(channels), DTYPES[dtype], _ptr(ln), _ptr(tx), int(flags),
                                       _stream(stream), ctypes.byref(h)), "htex_textures_upload")
        return cls(h, mesh)

    @classmethod
    def upload_levels(cls, mesh: Mesh, log2_res, texels, channels: int, dtype: str = "f32",
                      flags: int = 0, stream=None):
        lib = load()
        ln = _np(log2_res, np.int32)
        tx = _texel_array(texels, dtype)
        h = ctypes.c_void_p()
        check(lib.htex_textures_upload_levels(mesh._h, int(channels), DTYPES[dtype], _ptr(ln), _ptr(tx),
                                              int(flags), _stream(stream), ctypes.byref(h)),
              "htex_textures_upload_levels")
        return cls(h, mesh)

    @classmethod
    def upload_pool(cls, mesh: Mesh, log2_res, pool, scales, channels: int, dtype: str, stream=None):
        lib = load()
        ln = _np(log2_res, np.int32)
        pool = _np(pool, np.uint8)
        sc = _np(scales, np.float32) if scales is not None else None
        h = ctypes.c_void_p()
        check(lib.htex_textures_upload_pool(mesh._h, int(channels), DTYPES[dtype], _ptr(ln), _ptr(pool),
                                            _ptr(sc) if sc is not None else None, _stream(stream),
                                            ctypes.byref(h)), "htex_textures_upload_pool")
        return cls(h, mesh)

    def download_pool(self, stream=None):
        pool = np.empty(max(self.pool_bytes, 1), np.uint8)
        scales = np.empty(max(self.E, 1), np.float32)
        check(self._lib.htex_textures_download_pool(self._h, _ptr(pool), _ptr(scales), _stream(stream)),
              "htex_textures_download_pool")
        return pool[:self.pool_bytes], scales[:self.E]

    def write_pool(self, src, offset: int = 0, stream=None) -> None:
        """Overwrite pool bytes from a CUDA tensor or host array (raw stored values)."""
        import torch
        if isinstance(src, torch.Tensor):
            if not src.is_contiguous():
                raise ValueError("src must be contiguous")
            nbytes = src.numel() * src.element_size()
            ptr = ctypes.c_void_p(src.data_ptr())
        else:
            arr = np.ascontiguousarray(src)
            nbytes, ptr = arr.nbytes, _ptr(arr)
        check(self._lib.htex_textures_write_pool(self._h, int(offset), int(nbytes), ptr, _stream(stream)),
              "htex_textures_write_pool")

    def adam_step(self, master, grad, m, v, step: int, lr: float, betas=(0.9, 0.999), eps: float = 1e-8,
                  stream=None) -> None:
        """htex_textures_adam_step: one Adam step on an FP32 asset's texels;
        updates master, m and v, writes the new values into the pool and
        clears grad (all float32 CUDA tensors of pool_elements).  master
        None: the pool's own values are optimised in place."""
        import torch
        for name, x in (("master", master), ("grad", grad), ("m", m), ("v", v)):
            if x is None and name == "master":
                continue
            if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
                    and x.numel() == self.pool_elements):
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of pool_elements")
        ptrs = [ctypes.c_void_p(x.data_ptr() if x is not None else None) for x in (master, grad, m, v)]
        check(self._lib.htex_textures_adam_step(self._h, *ptrs,
                                                self.pool_elements, float(lr), float(betas[0]), float(betas[1]),
                                                float(eps), int(step), _stream(stream)), "htex_textures_adam_step")

    @property
    def pool_elements(self) -> int:
        return self.pool_bytes // ELEM_SIZE[self.dtype]

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.htex_textures_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def pack_queries(h, u, v, footprint=None):
    """AoS queries as an int32 numpy array [n, 4]: h, then the float32 bits of u, v, footprint."""
    h = _np(h, np.int32)
    n = h.shape[0]
    q = np.empty((n, 4), np.int32)
    q[:, 0] = h
    q[:, 1] = _np(u, np.float32).view(np.int32)
    q[:, 2] = _np(v, np.float32).view(np.int32)
    f = np.zeros(n, np.float32) if footprint is None else _np(footprint, np.float32)
    q[:, 3] = f.view(np.int32)
    return q


def _check_tensor(t, name, dtype, cols):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.dim() != 2 or t.shape[1] != cols:
        raise ValueError(f"{name} must be contiguous {dtype} [n, {cols}]")


def lookup(tex: Textures, queries, out=None, flags: int = 0, stream=None, status=None):
    """htex_lookup: queries int32 CUDA tensor [n, 4] -> float32 [n, channels]."""
    import torch
    _check_tensor(queries, "queries", torch.int32, 4)
    n = queries.shape[0]
    if out is None:
        out = torch.empty((n, tex.channels), dtype=torch.float32, device=queries.device)
    else:
        _check_tensor(out, "out", torch.float32, tex.channels)
    st = ctypes.c_void_p(status.data_ptr()) if status is not None else None
    check(tex._lib.htex_lookup(tex._h, ctypes.c_void_p(queries.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                               int(flags), _stream(stream), st), "htex_lookup")
    return out


def pack_queries_aniso(h, u, v, dudx, dvdx, dudy, dvdy) -> np.ndarray:
    """int32 [n, 8] rows laid out as htex_query_aniso (h, u, v, pad, du/dx,
    dv/dx, du/dy, dv/dy; the floats bit-cast)."""
    h = np.ascontiguousarray(h, np.int32)
    cols = [np.ascontiguousarray(a, np.float32).view(np.int32) for a in (u, v)]
    d = [np.ascontiguousarray(a, np.float32).view(np.int32) for a in (dudx, dvdx, dudy, dvdy)]
    return np.ascontiguousarray(np.stack([h, cols[0], cols[1], np.zeros_like(h)] + d, 1))


def lookup_aniso(tex: Textures, queries, max_aniso: int = 16, out=None, stream=None, status=None, flags: int = 0):
    """htex_lookup_aniso: queries int32 CUDA tensor [n, 8] -> float32 [n, channels]
    (flags: LOOKUP_BIN sorts the queries by halfedge range first)."""
    import torch
    _check_tensor(queries, "queries", torch.int32, 8)
    n = queries.shape[0]
    if out is None:
        out = torch.empty((n, tex.channels), dtype=torch.float32, device=queries.device)
    else:
        _check_tensor(out, "out", torch.float32, tex.channels)
    st = ctypes.c_void_p(status.data_ptr()) if status is not None else None
    check(tex._lib.htex_lookup_aniso(tex._h, ctypes.c_void_p(queries.data_ptr()), n, int(max_aniso), int(flags),
                                     ctypes.c_void_p(out.data_ptr()), _stream(stream), st), "htex_lookup_aniso")
    return out


def sort_queries(tex: Textures, queries, sorted_queries=None, pos=None, stream=None):
    """htex_queries_sort: queries int32 CUDA tensor [n, 4] -> (the queries
    sorted by halfedge range, int32 [n, 4]; pos int32 [n], where each query went)."""
    import torch
    _check_tensor(queries, "queries", torch.int32, 4)
    n = queries.shape[0]
    if sorted_queries is None:
        sorted_queries = torch.empty_like(queries)
    else:
        _check_tensor(sorted_queries, "sorted_queries", torch.int32, 4)
    if pos is None:
        pos = torch.empty(n, dtype=torch.int32, device=queries.device)
    if not (pos.is_cuda and pos.dtype == torch.int32 and pos.is_contiguous() and pos.numel() == n):
        raise ValueError("pos must be a contiguous CUDA int32 tensor of n elements")
    check(tex._lib.htex_queries_sort(tex._h, ctypes.c_void_p(queries.data_ptr()), n,
                                     ctypes.c_void_p(sorted_queries.data_ptr()), ctypes.c_void_p(pos.data_ptr()),
                                     _stream(stream)), "htex_queries_sort")
    return sorted_queries, pos


def gather_results(sorted_out, pos, out=None, stream=None):
    """htex_results_gather: float32 CUDA [n, channels] in sorted order -> query order."""
    import torch
    if not isinstance(sorted_out, torch.Tensor) or sorted_out.dim() != 2:
        raise ValueError("sorted_out must be a float32 CUDA tensor [n, channels]")
    n, c = sorted_out.shape
    _check_tensor(sorted_out, "sorted_out", torch.float32, c)
    if not (pos.is_cuda and pos.dtype == torch.int32 and pos.is_contiguous() and pos.numel() == n):
        raise ValueError("pos must be a contiguous CUDA int32 tensor of n elements")
    if out is None:
        out = torch.empty_like(sorted_out)
    else:
        _check_tensor(out, "out", torch.float32, c)
    lib = load()
    check(lib.htex_results_gather(ctypes.c_void_p(sorted_out.data_ptr()), ctypes.c_void_p(pos.data_ptr()), n, c,
                                  ctypes.c_void_p(out.data_ptr()), _stream(stream)), "htex_results_gather")
    return out


def lookup_host(tex: Textures, queries, out=None, flags: int = 0, stream=None, status=None):
    """htex_lookup_host: queries in host memory (int32 [n, 4], numpy or CPU
    tensor, ideally pinned) -> float32 [n, channels] in host memory.  The
    results are complete once 'stream' is synchronised."""
    import torch
    qt = torch.as_tensor(queries)
    if qt.is_cuda or qt.dtype != torch.int32 or qt.dim() != 2 or qt.shape[1] != 4 or not qt.is_contiguous():
        raise ValueError("queries must be a contiguous host int32 [n, 4] array")
    n = qt.shape[0]
    if out is None:
        out = torch.empty((n, tex.channels), dtype=torch.float32, pin_memory=True)
    if out.is_cuda or out.dtype != torch.float32 or tuple(out.shape) != (n, tex.channels) or not out.is_contiguous():
        raise ValueError("out must be a contiguous host float32 [n, channels] tensor")
    st = ctypes.c_void_p(status.data_ptr()) if status is not None else None
    check(tex._lib.htex_lookup_host(tex._h, ctypes.c_void_p(qt.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                    int(flags), _stream(stream), st), "htex_lookup_host")
    return out


def lookup_backward(tex: Textures, queries, grad_out, grad_texels=None, flags: int = 0, stream=None,
                    status=None):
    """htex_lookup_backward: accumulates into a pool-shaped float32 gradient and returns it."""
    import torch
    _check_tensor(queries, "queries", torch.int32, 4)
    _check_tensor(grad_out, "grad_out", torch.float32, tex.channels)
    if grad_texels is None:
        grad_texels = torch.zeros(tex.pool_elements, dtype=torch.float32, device=queries.device)
    st = ctypes.c_void_p(status.data_ptr()) if status is not None else None
    check(tex._lib.htex_lookup_backward(tex._h, ctypes.c_void_p(queries.data_ptr()), queries.shape[0],
                                        ctypes.c_void_p(grad_out.data_ptr()),
                                        ctypes.c_void_p(grad_texels.data_ptr()), int(flags), _stream(stream),
                                        st), "htex_lookup_backward")
    return grad_texels


def _autograd():
    import torch

    class HtexLookup(torch.autograd.Function):
        """Differentiable lookups of an FP32 asset:
        ``out = HtexLookup.apply(texels, tex, queries, flags)``.

        ``texels``: contiguous float32 CUDA tensor of ``tex.pool_elements``
        values, the stored texels in pool order (every texture at its pool
        offset, levels consecutive, row-major [N][N][C]; padding elements are
        ignored).  The forward pass writes them into the resident pool
        (htex_textures_write_pool, a device-to-device copy on the current
        stream) and runs htex_lookup, so the result is always the lookup of
        exactly these values; the backward pass returns d loss / d texels in
        the same layout (htex_lookup_backward).  ``flags``: HTEX_LOOKUP_BIN
        sorts the queries in both passes.  The queries get no gradient."""

        @staticmethod
        def forward(ctx, texels, tex, queries, flags=0):
            if tex.dtype != "f32":
                raise ValueError("HtexLookup needs an FP32 asset (its texels are the stored values)")
            if not (isinstance(texels, torch.Tensor) and texels.is_cuda and texels.dtype == torch.float32
                    and texels.is_contiguous() and texels.numel() == tex.pool_elements):
                raise ValueError("texels must be a contiguous float32 CUDA tensor of tex.pool_elements values")
            tex.write_pool(texels.detach())
            ctx.tex = tex
            ctx.flags = int(flags)
            ctx.save_for_backward(queries)
            return lookup(tex, queries, flags=flags)

        @staticmethod
        def backward(ctx, grad_out):
            (queries,) = ctx.saved_tensors
            g = None
            if ctx.needs_input_grad[0]:
                g = lookup_backward(ctx.tex, queries, grad_out.contiguous().float(), flags=ctx.flags)
            return g, None, None, None

    return HtexLookup


class _LazyFn:
    """HtexLookup, created on first use (torch is imported lazily)."""
    _fn = None

    def apply(self, *a):
        if _LazyFn._fn is None:
            _LazyFn._fn = _autograd()
        return _LazyFn._fn.apply(*a)


HtexLookup = _LazyFn()
