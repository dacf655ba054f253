"""Multi-asset lookup serving (htex_server_*): ctypes wrapper and a stream driver.

The server (native, in libhtex) keeps assets resident under a device-memory
budget and serves requests by continuous batching in CUDA-graph launches;
this module only marshals arguments and replays request streams.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import DTYPES, Mesh, Textures
from ._lib import check, load


class Config(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("batch_queries", ctypes.c_int64),
                ("batch_slots", ctypes.c_int32), ("max_items", ctypes.c_int32),
                ("request_chunk", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("queries", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("uploads", ctypes.c_int64), ("evictions", ctypes.c_int64), ("resident_bytes", ctypes.c_int64),
                ("host_queries", ctypes.c_int64)]


class Server:
    def __init__(self, budget_bytes: int, batch_queries: int = 1 << 22, batch_slots: int = 3,
                 max_items: int = 256, request_chunk: int = 1 << 20):
        self._lib = load()
        cfg = Config(int(budget_bytes), int(batch_queries), int(batch_slots), int(max_items), int(request_chunk))
        h = ctypes.c_void_p()
        check(self._lib.htex_server_create(ctypes.byref(cfg), ctypes.byref(h)), "htex_server_create")
        self._h = h
        self._keep = {}

    def add_asset(self, mesh: Mesh, log2_res, pool, scales, channels: int, dtype: str) -> int:
        ln = np.ascontiguousarray(log2_res, np.int32)
        pool = np.ascontiguousarray(pool, np.uint8)
        sc = np.ascontiguousarray(scales, np.float32)
        aid = ctypes.c_int32()
        check(self._lib.htex_server_add_asset(self._h, mesh._h, int(channels), DTYPES[dtype],
                                              ln.ctypes.data_as(ctypes.c_void_p), pool.ctypes.data_as(ctypes.c_void_p),
                                              sc.ctypes.data_as(ctypes.c_void_p), ctypes.byref(aid)),
              "htex_server_add_asset")
        return aid.value

    def submit(self, asset: int, q_ptr: int, n: int, out_ptr: int) -> int:
        """Queue n queries at host address q_ptr; results to host address out_ptr."""
        rid = ctypes.c_int64()
        check(self._lib.htex_server_submit(self._h, int(asset), ctypes.c_void_p(q_ptr), int(n),
                                           ctypes.c_void_p(out_ptr), ctypes.byref(rid)), "htex_server_submit")
        return rid.value

    def poll(self, capacity: int = 4096):
        ids = np.empty(capacity, np.int64)
        lat = np.empty(capacity, np.float64)
        cnt = ctypes.c_int32()
        check(self._lib.htex_server_poll(self._h, ids.ctypes.data_as(ctypes.c_void_p),
                                         lat.ctypes.data_as(ctypes.c_void_p), capacity, ctypes.byref(cnt)),
              "htex_server_poll")
        return ids[:cnt.value].copy(), lat[:cnt.value].copy()

    def drain(self, timeout_s: float = 60.0) -> None:
        check(self._lib.htex_server_drain(self._h, float(timeout_s)), "htex_server_drain")

    def stats(self) -> dict:
        st = Stats()
        check(self._lib.htex_server_get_stats(self._h, ctypes.byref(st)), "htex_server_get_stats")
        return {k: getattr(st, k) for k, _ in Stats._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.htex_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def replay(server: Server, arrivals, sizes, assets, query_src, out_ptr_of):
    """Submit requests at their arrival times (seconds from start).

    query_src(asset, n) -> host address of n queries; out_ptr_of(k, asset, n)
    -> host address for request k's results.  Returns per-request latencies
    (seconds, submission to completion, request order) and the wall time
    from the first submission to the last completion."""
    ids = np.zeros(len(sizes), np.int64)
    t0 = time.perf_counter()
    for k in range(len(sizes)):
        target = t0 + float(arrivals[k])
        while time.perf_counter() < target:
            pass
        ids[k] = server.submit(int(assets[k]), query_src(int(assets[k]), int(sizes[k])), int(sizes[k]),
                               out_ptr_of(k, int(assets[k]), int(sizes[k])))
    server.drain(600.0)
    wall = time.perf_counter() - t0
    got_ids, lat = server.poll(len(sizes) + 16)
    order = {int(i): float(t) for i, t in zip(got_ids, lat)}
    return np.array([order[int(i)] for i in ids]), wall
