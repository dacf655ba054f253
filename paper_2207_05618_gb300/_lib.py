"""ctypes declarations of libhtex's C ABI (include/htex.h).

Argument marshalling only.  Loading fails loudly when the library has not
been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

from .build import INCLUDE, LIB

HTEX_OK = 0
STATUS_NAMES = {0: "HTEX_OK", 1: "HTEX_ERR_INVALID_ARG", 2: "HTEX_ERR_NONMANIFOLD",
                3: "HTEX_ERR_BAD_TEXTURE", 4: "HTEX_ERR_OUT_OF_MEMORY", 5: "HTEX_ERR_CUDA",
                6: "HTEX_ERR_QUERY_OUT_OF_RANGE", 7: "HTEX_ERR_TIMEOUT", 8: "HTEX_ERR_UNSUPPORTED"}

DTYPES = {"f32": 0, "u8": 1, "f16": 2, "bf16": 3, "e4m3": 4}
ELEM_SIZE = {"f32": 4, "u8": 1, "f16": 2, "bf16": 2, "e4m3": 1}
BUILD_MIPS, MIRROR_BOUNDARY, FIX_CORNERS, LEVELS_GIVEN = 1, 2, 4, 8
LOOKUP_BIN, LOOKUP_GLOBAL = 1, 2


class HtexError(RuntimeError):
    def __init__(self, code: int, call: str):
        self.code = code
        super().__init__(f"{call} failed: {STATUS_NAMES.get(code, code)}")


def check(code: int, call: str) -> None:
    if code != HTEX_OK:
        raise HtexError(code, call)


P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
U32 = ctypes.c_uint32
PP = ctypes.POINTER(ctypes.c_void_p)

_SIGNATURES = {
    "htex_status_string": ([I32], ctypes.c_char_p),
    "htex_mesh_create": ([P, I32, P, I32, PP], I32),
    "htex_mesh_create_from_halfedges": ([P, P, P, P, P, P, I32, I32, I32, PP], I32),
    "htex_mesh_info": ([P, P, P, P, P, P], I32),
    "htex_mesh_get_halfedges": ([P, P, P, P, P, P, P], I32),
    "htex_mesh_destroy": ([P], None),
    "htex_textures_layout": ([P, I32, I32, P, P, P], I32),
    "htex_textures_prepare": ([P, I32, I32, P, P, U32, P, P], I32),
    "htex_textures_upload": ([P, I32, I32, P, P, U32, P, PP], I32),
    "htex_textures_upload_levels": ([P, I32, I32, P, P, U32, P, PP], I32),
    "htex_textures_upload_pool": ([P, I32, I32, P, P, P, P, PP], I32),
    "htex_textures_info": ([P, P, P, P, P, P, P], I32),
    "htex_textures_download_pool": ([P, P, P, P], I32),
    "htex_textures_write_pool": ([P, I64, I64, P, P], I32),
    "htex_textures_destroy": ([P], None),
    "htex_lookup": ([P, P, I64, P, U32, P, P], I32),
    "htex_lookup_aniso": ([P, P, I64, I32, U32, P, P, P], I32),
    "htex_queries_sort": ([P, P, I64, P, P, P], I32),
    "htex_results_gather": ([P, P, I64, I32, P, P], I32),
    "htex_lookup_backward": ([P, P, I64, P, P, U32, P, P], I32),
    "htex_textures_adam_step": ([P, P, P, P, P, I64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, I32, P], I32),
    "htex_lookup_host": ([P, P, I64, P, U32, P, P], I32),
    "htex_geometry_create": ([P, P, P, PP], I32),
    "htex_geometry_destroy": ([P], None),
    "htex_triangle_vertices": ([P, P, P], I32),
    "htex_rasterize": ([P, P, I32, I32, P, P, P], I32),
    "htex_rasterize_aniso": ([P, P, I32, I32, P, P, P], I32),
    "htex_displace": ([P, P, I32, ctypes.c_float, I32, P, P], I32),
    "htex_server_create": ([P, PP], I32),
    "htex_server_add_asset": ([P, P, I32, I32, P, P, P, P], I32),
    "htex_server_submit": ([P, I32, P, I64, P, P], I32),
    "htex_server_poll": ([P, P, P, I32, P], I32),
    "htex_server_drain": ([P, ctypes.c_double], I32),
    "htex_server_get_stats": ([P, P], I32),
    "htex_server_destroy": ([P], None),
    "htex_lookup_noalloc": ([P, P, I64, P, P, P], I32),
    "htex_lookup_noalloc_max_queries": ([], I64),
}

_lib = None


def header_functions() -> list[str]:
    """Every function name declared in include/*.h."""
    names = []
    for fn in sorted(os.listdir(INCLUDE)):
        if fn.endswith(".h"):
            text = open(os.path.join(INCLUDE, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(htex_\w+)\s*\(", text)
    return sorted(set(names))


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libhtex.so (built by paper_2207_05618_gb300.build)."""
    global _lib
    if _lib is None:
        path = path or LIB
        if not os.path.exists(path):
            raise ImportError(f"libhtex.so not built ({path}); run paper_2207_05618_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib
