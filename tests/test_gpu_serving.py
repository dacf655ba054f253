"""GPU tests of the lookup server (htex_server_*): every request's results
are the same alone and in the mix, while the device budget forces assets
to be evicted and uploaded again (requests for an asset that is not
resident read its host copy meanwhile), for requests served in place from
pinned buffers and for requests staged through device copies."""
import numpy as np
import pytest

import htex_synth as syn
import paper_2207_05618_gb300 as hx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2207_05618_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _assets():
    specs = [(syn.cylinder(around=24, rows=10, seed=1), 5, "u8", 4),
             (syn.uv_sphere(slices=20, rings=12, seed=2), 5, "f16", 4),
             (syn.cylinder(around=16, rows=8, seed=3), 4, "f32", 3),
             (syn.cylinder(around=40, rows=12, seed=4), 4, "e4m3", 2)]
    out = []
    for k, ((fs, fv, V, _), n, fmt, C) in enumerate(specs):
        mesh = hx.Mesh(fs, fv, V)
        log2n = np.full(mesh.E, n, np.int32)
        tex = (syn.texels_u8 if fmt == "u8" else syn.texels_f32)(log2n, C, seed=10 + k)
        pool, scales = hx.Textures.prepare(mesh, log2n, tex, C, fmt, hx.BUILD_MIPS | hx.MIRROR_BOUNDARY)
        alone = hx.Textures.upload_pool(mesh, log2n, pool, scales, C, fmt)
        out.append({"mesh": mesh, "log2n": log2n, "pool": pool, "scales": scales, "C": C, "fmt": fmt,
                    "alone": alone})
    return out


def test_server_results_equal_standalone_lookups():
    from paper_2207_05618_gb300 import serve
    assets = _assets()
    sizes_b = sorted(a["alone"].device_bytes for a in assets)
    budget = sizes_b[-1] + sizes_b[-2] // 2          # the two largest never fit together
    server = serve.Server(budget, batch_queries=1 << 18, batch_slots=3, max_items=64, request_chunk=1 << 16)
    ids = [server.add_asset(a["mesh"], a["log2n"], a["pool"], a["scales"], a["C"], a["fmt"]) for a in assets]
    assert ids == [0, 1, 2, 3]
    rng = np.random.default_rng(0)
    reqs = []
    order = np.concatenate([np.repeat(np.arange(4), 10), rng.integers(0, 4, 40)])   # runs force re-uploads
    for k, a_id in enumerate(order):
        a = assets[int(a_id)]
        n = int(np.exp(rng.uniform(0, np.log(300_000))))
        qs = syn.queries(a["mesh"].H, n, seed=1000 + k, footprint="loguniform")
        if k % 7 == 3:
            qs[0][: min(n, 2)] = -5                  # invalid ids in the mix
        q = torch.from_numpy(hx.pack_queries(*qs))
        out = torch.full((n, a["C"]), 3.0, dtype=torch.float32)
        if k % 5 != 1:                               # pinned: served in place; else staged copies
            q, out = q.pin_memory(), out.pin_memory()
        rid = server.submit(int(a_id), q.data_ptr(), n, out.data_ptr())
        reqs.append((rid, int(a_id), q, out))
    assert server.submit(0, 0, 0, 0) > 0             # an empty request completes at once
    server.drain(120.0)
    got, lat = server.poll(1000)
    assert len(got) == len(reqs) + 1 and np.all(lat >= 0)
    for rid, a_id, q, out in reqs:
        ref = hx.lookup(assets[a_id]["alone"], q.cuda()).cpu()
        assert torch.equal(torch.isnan(out), torch.isnan(ref))
        assert torch.equal(torch.nan_to_num(out, nan=0.0), torch.nan_to_num(ref, nan=0.0)), rid
    st = server.stats()
    assert st["completed"] == len(reqs) + 1
    assert st["evictions"] > 0 and st["uploads"] > len(assets)
    assert st["resident_bytes"] <= budget
    assert 0 < st["host_queries"] < st["queries"]   # some batches read a non-resident asset's host copy
    with pytest.raises(hx.HtexError):
        server.submit(17, 0, 1, 0)
    server.close()


def test_server_rejects_asset_over_budget():
    from paper_2207_05618_gb300 import serve
    a = _assets()[0]
    server = serve.Server(a["alone"].device_bytes // 2, batch_queries=1 << 16)
    with pytest.raises(hx.HtexError):
        server.add_asset(a["mesh"], a["log2n"], a["pool"], a["scales"], a["C"], a["fmt"])
    server.close()
