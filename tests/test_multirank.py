"""Multi-GPU logic of bench.py on CPU (gloo, world size 2): every rank
holds its own replica and queries (weak scaling, no data-path collective);
the job is timed by its slowest rank and its throughput counts every
rank's lookups.  Each rank also filters its own shard on its replica (the
FP64 oracle stands in for the device here), and the shards' results,
gathered after the fact, equal one process filtering the union: replicas
need no exchange."""
import os
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import htex_synth as syn
    # each rank's queries differ (own seed), same count
    h, u, v, f = syn.queries(1000, 64, seed=bench.rank_seed(rank), footprint="loguniform")
    local_ms = 10.0 + 5.0 * rank                   # rank 1 is the slower one
    slowest = bench.reduce_max(local_ms, dist, "cpu")
    rate = bench.job_rate(1 << 24, 10, world, slowest)
    # this rank's replica of a small asset and its own shard of queries
    import oracle
    fs, fv, V, _ = syn.cylinder(around=8, rows=3, seed=5)
    mo = oracle.mesh_from_faces(fs, fv, V)
    log2n = np.full(mo.num_edges, 2, np.int32)
    to = oracle.prepare_textures(mo, log2n, syn.texels_f32(log2n, 2, seed=6), 2, "f32", oracle.BUILD_MIPS)
    shard = syn.queries(mo.H, 500, seed=bench.rank_seed(rank), footprint="loguniform")
    out = oracle.lookup(mo, to, shard)
    q.put((rank, int(h[:8].sum()), slowest, rate, out.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, v0, o0), (r1, s1, t1, v1, o1) = res
    assert s0 != s1                                 # independent query shards
    assert t0 == t1 == 15.0                         # both ranks report the slowest rank's time
    assert v0 == v1 == pytest.approx((1 << 24) * 10 * 2 / 0.015)
    # one process over the union of both shards gives the same values
    sys.path.insert(0, ROOT)
    import bench
    import htex_synth as syn
    import oracle
    fs, fv, V, _ = syn.cylinder(around=8, rows=3, seed=5)
    mo = oracle.mesh_from_faces(fs, fv, V)
    log2n = np.full(mo.num_edges, 2, np.int32)
    to = oracle.prepare_textures(mo, log2n, syn.texels_f32(log2n, 2, seed=6), 2, "f32", oracle.BUILD_MIPS)
    shards = [syn.queries(mo.H, 500, seed=bench.rank_seed(r), footprint="loguniform") for r in range(2)]
    union = tuple(np.concatenate([a, b]) for a, b in zip(*shards))
    np.testing.assert_array_equal(np.concatenate([np.array(o0), np.array(o1)]), oracle.lookup(mo, to, union))
