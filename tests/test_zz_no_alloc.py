"""The allocation-free lookup, htex_lookup_noalloc, called through the C ABI.

Callers that may not allocate device memory (an engine or plug-in host that
owns every allocation, a frame loop that cannot absorb the synchronisation
cudaMalloc/cudaFree may cause) use this entry point; its scratch is a fixed
device array inside the library.  This file is collected last so that a run
stopping at the first failure has run every other test first; it also
passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import htex_synth as syn
import paper_2207_05618_gb300 as hx
from paper_2207_05618_gb300 import _lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def asset():
    from paper_2207_05618_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    # about 97 MB of 32x32 RGBA8 texels: large enough for the binned path
    fs, fv, V, _ = syn.cylinder(around=128, rows=60, seed=14)
    mesh = hx.Mesh(fs, fv, V)
    log2n = np.full(mesh.E, 5, np.int32)
    tex = hx.Textures.upload(mesh, log2n, syn.texels_u8(log2n, 4, seed=15), 4, "u8",
                             hx.BUILD_MIPS | hx.MIRROR_BOUNDARY)
    assert tex.pool_bytes > (64 << 20)
    return mesh, tex


def _noalloc(tex, q, out, status):
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.htex_lookup_noalloc(tex._h, ctypes.c_void_p(q.data_ptr()), q.shape[0],
                                   ctypes.c_void_p(out.data_ptr()), stream,
                                   ctypes.c_void_p(status.data_ptr()))


def test_noalloc_matches_binned_lookup_twice(asset):
    mesh, tex = asset
    lib = _lib.load()
    nmax = int(lib.htex_lookup_noalloc_max_queries())
    assert nmax == 1 << 20
    for call, (n, seed) in enumerate(((300007, 31), (nmax, 32))):
        h, u, v, f = syn.queries(mesh.H, n, seed=seed, footprint="loguniform")
        h[:3] = (-1, mesh.H, 5)                    # two invalid ids
        q = torch.from_numpy(hx.pack_queries(h, u, v, f)).cuda()
        ref_status = torch.zeros(1, dtype=torch.int32, device="cuda")
        ref = hx.lookup(tex, q, flags=hx.LOOKUP_BIN, status=ref_status)
        out = torch.full((n, 4), 7.0, dtype=torch.float32, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        assert _noalloc(tex, q, out, status) == 0, f"call {call}"
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        # the same per-query filter code in both: equal bit for bit, NaN
        # rows (invalid ids) included
        np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
        assert int(status.item()) == int(ref_status.item()) == 2


def test_noalloc_rejects_more_than_its_capacity(asset):
    mesh, tex = asset
    lib = _lib.load()
    n = int(lib.htex_lookup_noalloc_max_queries()) + 1
    q = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _noalloc(tex, q, out, status) == 8            # HTEX_ERR_UNSUPPORTED
