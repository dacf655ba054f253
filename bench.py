#!/usr/bin/env python3
"""Benchmark of batched seamless filtered Htex lookups (libhtex, GB300).

Default workload (one step = one htex_lookup over every query of the
batch): the asset-scale mesh, an open cylinder of 256 quads around and 460
rows with about 30% of quads split into triangles and about 5% of faces
merged into 5- to 8-gons (522,126 halfedges, 261k edges), one 64x64 RGBA8
UNORM texture per edge with its mip chain (5.7 GB), 16,777,216 queries per
GPU with uniform halfedge ids and barycentrics and log-uniform footprints
2^-8..1 (trilinear).  Inputs are seeded and synthetic.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead, on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "filtered Htex lookups/s"
UNIT = "lookups/s"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=500)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--queries", type=int, default=1 << 24)
    p.add_argument("--no-bin", action="store_true",
                   help="filter the queries in their given order (no sort by halfedge range)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cube", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the precision and backward measurements")
    p.add_argument("--rows", type=int, default=460, help="cylinder rows (460: the asset-scale mesh)")
    p.add_argument("--only", choices=["backward", "aniso", "cube"],
                   help="run one workload alone (sorted adjoint on the differentiation workload; anisotropic "
                        "lookups on the --rows asset with --queries queries; cube streaming), warm-up and timed "
                        "launches only, and print its timing: for profiling one kernel")
    return p.parse_args()


def run_only(args, hx, torch):
    """One workload's launches alone (for ncu captures of one kernel)."""
    import htex_synth as syn
    stream = torch.cuda.current_stream()
    if args.only == "backward":
        fs, fv, V, _ = syn.uv_sphere()
        mesh = hx.Mesh(fs, fv, V)
        log2n = np.full(mesh.E, 5, np.int32)
        tex = hx.Textures.upload(mesh, log2n, syn.texels_f32(log2n, 3, seed=2), 3, "f32", hx.BUILD_MIPS)
        gen = torch.Generator(device="cuda")
        gen.manual_seed(4)
        n = 2_000_000
        q = device_queries(torch, mesh.H, n, gen)
        g = torch.randn((n, 3), device="cuda", generator=gen)
        grad = torch.zeros(tex.pool_elements, dtype=torch.float32, device="cuda")
        fn = lambda: hx.lookup_backward(tex, q, g, grad_texels=grad, flags=hx.LOOKUP_BIN, stream=stream)
        units = n
    elif args.only == "aniso":
        fs, fv, V, _ = syn.cylinder(rows=args.rows)
        mesh = hx.Mesh(fs, fv, V)
        log2n = np.full(mesh.E, 6, np.int32)
        tex = hx.Textures.upload(mesh, log2n, syn.texels_u8(log2n, 4, seed=21), 4, "u8", hx.BUILD_MIPS)
        r = aniso_bench(hx, torch, stream, mesh, tex, n=args.queries, reps=args.steps, warm=args.warmup,
                        sorted_too=False)
        print(json.dumps({"only": "aniso", **r}), flush=True)
        return
    else:
        fs, fv, V, _ = syn.cube()
        mesh = hx.Mesh(fs, fv, V)
        log2n = np.full(mesh.E, 4, np.int32)
        tex = hx.Textures.upload(mesh, log2n, syn.texels_f32(log2n, 4, seed=1), 4, "f32", hx.BUILD_MIPS)
        n = 1 << 24
        q = torch.from_numpy(hx.pack_queries(*syn.queries(mesh.H, n, seed=2))).cuda()
        out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        fn = lambda: hx.lookup(tex, q, out=out, stream=stream)
        units = n
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    print(json.dumps({"only": args.only, "ms": ms, "units_per_s": units / (ms / 1e3)}), flush=True)


# ----------------------------------------------------------------- workload

def rank_seed(rank: int) -> int:
    """Each rank draws its own queries (weak scaling: the same count per GPU)."""
    return 1000 + rank


def reduce_max(x: float, dist, device) -> float:
    """Max over ranks (the slowest rank times the whole job)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * steps * world / (max_ms / 1e3)


def asset_inputs(rank: int, nq: int, rows: int = 460):
    import htex_synth as syn
    fs, fv, V, pos = syn.cylinder(rows=rows)
    return fs, fv, V, pos, syn.queries(int(fs.sum()), nq, seed=rank_seed(rank), footprint="loguniform")


def workload_config(H, E, nq, flags_name):
    return {
        "workload": "asset-scale open cylinder 256x460 quads with splits and merges; "
                    "64x64 RGBA8 UNORM edge textures with mip chains; log-uniform footprints 2^-8..1",
        "halfedges": int(H), "edges": int(E), "texel_format": "rgba8_unorm", "texture_res": 64,
        "queries_per_gpu": int(nq), "lookup_flags": flags_name,
        "l2": "inputs larger than L2: 256 MB queries, 256 MB outputs, 5.7 GB texels per step",
    }


def arm_flags_name(args) -> str:
    return ("none" if args.no_bin else
            "sorted by halfedge range (htex_queries_sort, htex_lookup, htex_results_gather)")


def source_hash() -> str:
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_2207_05618_gb300", "csrc", "*"))):
        with open(p, "rb") as fh:
            h.update(os.path.basename(p).encode())
            h.update(fh.read())
    return h.hexdigest()[:12]


# the files the filter kernel is compiled from (and the build flags), and lookup.cu, whose sort sets the
# order (hence the DRAM traffic) of the queries it filters
FILTER_SOURCES = ("csrc/lookup_kernels.cuh", "csrc/lookup_u8.cu", "csrc/lookup_core.cuh", "csrc/fetch.cuh",
                  "csrc/htex_internal.h", "build.py", "csrc/lookup.cu")


def filter_source_hash() -> str:
    h = hashlib.sha256()
    for rel in FILTER_SOURCES:
        with open(os.path.join(ROOT, "paper_2207_05618_gb300", rel), "rb") as fh:
            h.update(rel.encode())
            h.update(fh.read())
    return h.hexdigest()[:12]


def profiled_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, when it was
    taken on the filter kernel's current sources; else None."""
    path = os.path.join(ROOT, "profiles", "lookup_asset_scale.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"filter_source_hash:\s*([0-9a-f]+)", text)
    t = re.search(rf"{kernel}_dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if m and t and m.group(1) == filter_source_hash():
        return float(t.group(1))
    return None


# the files the anisotropic kernel and the adjoint are compiled from (and the build flags)
ANISO_SOURCES = ("csrc/aniso.cu", "csrc/aniso_launch.h", "csrc/fetch.cuh", "csrc/htex_internal.h", "build.py")
BACKWARD_SOURCES = ("csrc/backward.cu", "csrc/fetch.cuh", "csrc/htex_internal.h", "build.py")


def sources_hash(rels) -> str:
    h = hashlib.sha256()
    for rel in rels:
        with open(os.path.join(ROOT, "paper_2207_05618_gb300", rel), "rb") as fh:
            h.update(rel.encode())
            h.update(fh.read())
    return h.hexdigest()[:12]


def profiled_values(name: str, rels):
    """'key: value' numbers of a committed ncu summary, when its
    source_files_hash matches the current sources of the kernel; else None."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"source_files_hash:\s*([0-9a-f]+)", text)
    if not m or m.group(1) != sources_hash(rels):
        return None
    vals = {}
    for k, v in re.findall(r"^(\w+):\s*(\S+)\s*$", text, flags=re.M):
        try:
            vals[k] = float(v)
        except ValueError:
            pass
    return vals


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy kernel)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (6.8 TB/s, no MEASURED_PEAKS.json)"


def mean_taps(he, n_uniform: int, qs, sample: int = 1 << 20) -> float:
    """Texel taps one lookup must read, averaged over a sample of the
    queries: every tap with nonzero weight that falls inside its texture
    (own, Next and Prev fetches, one or two levels each) on an asset whose
    textures are all 2^n_uniform a side."""
    h, u, v, f = (np.asarray(x)[:sample] for x in qs)
    u = np.maximum(u.astype(np.float64), 0)
    v = np.maximum(v.astype(np.float64), 0)
    s = u + v
    over = s > 1
    u[over] /= s[over]
    v[over] /= s[over]
    with np.errstate(divide="ignore"):
        lam = np.where(f > 0, np.log2(np.where(f > 0, f, 1.0)) + n_uniform, -1.0)
    d = np.floor(lam)
    taps = np.zeros(h.shape[0])
    twin, nxt, prv = he["twin"], he["next"], he["prev"]
    for g, a, b in ((h, u, v), (nxt[h], v, -u), (prv[h], -v, u)):
        flip = g < twin[g]
        x = np.where(flip, 1 - a, a)
        y = np.where(flip, 1 - b, b)
        single = ~(lam > 0) | (d >= n_uniform)
        l0 = np.where(~(lam > 0), 0, np.minimum(d, n_uniform)).astype(np.int64)
        for lev, active, w in ((l0, np.ones_like(single), np.where(single, 1.0, 1 - (lam - d))),
                               (l0 + 1, ~single, lam - d)):
            N = np.left_shift(1, np.clip(n_uniform - lev, 0, 30)).astype(np.float64)
            sx, sy = x * N - 0.5, y * N - 0.5
            i0, j0 = np.floor(sx), np.floor(sy)
            ax, by = sx - i0, sy - j0
            for di, wx in ((0, 1 - ax), (1, ax)):
                for dj, wy in ((0, 1 - by), (1, by)):
                    ii, jj = i0 + di, j0 + dj
                    ok = (ii >= 0) & (ii < N) & (jj >= 0) & (jj < N) & (wx * wy * w > 0) & active
                    taps += ok
    return float(taps.mean())


def algorithmic_bytes(taps: float, texel_bytes: int) -> dict:
    """Bytes one lookup must move on a one-resolution asset (no texture
    headers), two ways.  'hot_path': the hot-path table's count -- the 16-byte
    query, the 16-byte output, the 16-byte halfedge records of h, Next(h)
    and Prev(h), and the in-bounds taps.  'packed': this library's layout,
    where the three records are pre-evaluated into one 16-byte record of h
    (the same operators, evaluated at upload)."""
    tex = taps * texel_bytes
    return {"hot_path": 16 + 16 + 3 * 16 + tex, "packed": 16 + 16 + 16 + tex, "taps": taps}


# ------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons, timestamped on receipt."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device_index: int):
        self.samples = []
        self.proc = None
        sel = []
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            sel = ["-i", uuid if uuid.startswith("GPU-") else "GPU-" + uuid]
        except Exception:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES")
            sel = ["-i", vis.split(",")[device_index]] if vis else ["-i", str(device_index)]
        self.cmd = ["nvidia-smi", *sel, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                    "-lms", "100"]

    def start(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        def read():
            for line in self.proc.stdout:
                self.samples.append((time.time(), line.strip()))
        self.thread = threading.Thread(target=read, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        """Samples taken during [t0, t1]; when the timed region was shorter
        than the sampling period, the samples within 0.25 s of it."""
        window = "timed region"
        picked = [(ts, line) for ts, line in self.samples if t0 <= ts <= t1 + 0.15]
        if not picked:
            window = "within 0.25 s of the timed region"
            picked = [(ts, line) for ts, line in self.samples if t0 - 0.25 <= ts <= t1 + 0.25]
        sm, mx, reasons = [], [], set()
        for ts, line in picked:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "window": window}


# ------------------------------------------------------------ oracle sample

def oracle_sample(nq_sample: int, seed: int = 7, slice_h: int = 4096):
    """A bounded oracle workload: the same mesh, textures and query
    distribution, with queries restricted to halfedges [0, slice_h) so the
    oracle's FP64 copy of the touched textures fits host memory."""
    import htex_synth as syn
    import oracle
    fs, fv, V, _ = syn.cylinder()
    mo = oracle.mesh_from_faces(fs, fv, V)
    log2n = np.full(mo.num_edges, 6, np.int32)
    h, u, v, f = syn.queries(slice_h, nq_sample, seed=seed, footprint="loguniform")
    hs = np.arange(slice_h)
    edges = np.unique(np.concatenate([mo.edge[hs], mo.edge[mo.next[hs]], mo.edge[mo.prev[hs]]]))
    keep = np.zeros(mo.num_edges, bool)
    keep[edges] = True
    rng = np.random.default_rng(21)
    ln = np.where(keep, log2n, 0).astype(np.int32)
    counts = (np.int64(1) << (2 * ln.astype(np.int64))) * 4
    tex = np.frombuffer(rng.bytes(int(counts.sum())), np.uint8)
    to = oracle.prepare_textures(mo, ln, tex, 4, "u8", oracle.BUILD_MIPS)
    return mo, to, (h, u, v, f)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def time_oracle(budget_s: float):
    """Oracle lookups/s on all host cores, sample sized to about budget_s."""
    import oracle
    cores = host_cores()
    mo, to, qs = oracle_sample(1 << 21)
    oracle.lookup(mo, to, tuple(x[:1 << 14] for x in qs), nthreads=cores)   # warm the caches
    n = 0
    t = time.perf_counter()
    while True:                     # whole passes over the sample until the budget is spent
        oracle.lookup(mo, to, qs, nthreads=cores)
        n += qs[0].shape[0]
        dt = time.perf_counter() - t
        if dt >= budget_s:
            break
    return n / dt, cores, n, (mo, to, qs)


# ---------------------------------------------------------------- reference

def run_reference(args, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = host_cores()
    mo, to, qs = oracle_sample(1 << 21)
    budget = max(0.05, 150.0 / max(args.steps + args.warmup, 1))
    probe = 1 << 13
    t = time.perf_counter()
    oracle.lookup(mo, to, tuple(x[:probe] for x in qs), nthreads=cores)
    rate = probe / max(time.perf_counter() - t, 1e-6)
    n = int(min(qs[0].shape[0], max(1024, rate * budget)))
    sub = tuple(x[:n] for x in qs)
    for _ in range(args.warmup):
        oracle.lookup(mo, to, sub, nthreads=cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.lookup(mo, to, sub, nthreads=cores)
    dt = time.perf_counter() - t
    value = n * args.steps / dt
    # the same config object as this bench's own arm; the bounded sample is described in cpu_baseline
    cfg = workload_config(mo.H, mo.num_edges, args.queries, arm_flags_name(args))
    sample = (f"{n} queries per step with h uniform on halfedges [0, 4096) of the asset, "
              f"barycentrics and footprints as the workload; FP64 oracle on {cores} host threads; "
              f"optimistic: the textures of that subset stay in the host caches, unlike the whole asset's")
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------- ours

def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2207_05618_gb300 import build as b
    if rank == 0:
        b.build()
    if dist:
        dist.barrier()
    import paper_2207_05618_gb300 as hx
    if args.only:
        run_only(args, hx, torch)
        return

    nq = args.queries
    fs, fv, V, positions, qs = asset_inputs(rank, nq, args.rows)
    mesh = hx.Mesh(fs, fv, V)
    log2n = np.full(mesh.E, 6, np.int32)
    import htex_synth as syn
    texels = syn.texels_u8(log2n, 4, seed=21)
    tex = hx.Textures.upload(mesh, log2n, texels, 4, "u8", hx.BUILD_MIPS)
    del texels
    use_bin = not args.no_bin
    flags = hx.LOOKUP_BIN if use_bin else 0
    q_host = torch.from_numpy(hx.pack_queries(*qs)).pin_memory()
    q = q_host.cuda()
    out = torch.empty((nq, 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    taps = mean_taps(mesh.halfedges(), 6, qs)
    ab = algorithmic_bytes(taps, 4)
    if use_bin:
        sq = torch.empty_like(q)
        pos = torch.empty(nq, dtype=torch.int32, device="cuda")
        sout = torch.empty_like(out)
    sort_chunk = 1 << 24
    launches_per_step = (2 * -(-nq // sort_chunk) + 2) if use_bin else 1

    def step(ev=None):
        # a0 (sort by halfedge range), a1..a6 (the filter kernel), results back in query order
        if use_bin:
            hx.sort_queries(tex, q, sq, pos, stream=stream)
        if ev is not None:
            ev[0].record(stream)
        hx.lookup(tex, sq if use_bin else q, out=sout if use_bin else out, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        if use_bin:
            hx.gather_results(sout, pos, out=out, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.5)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    filt = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        starts[k].record(stream)
        step(filt[k])
        ends[k].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t1 = time.time()
    sampler.stop()
    total_ms = reduce_max(starts[0].elapsed_time(ends[-1]), dist, "cuda")
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    launch_ms = [a.elapsed_time(b) for a, b in filt]
    value = job_rate(nq, args.steps, world, total_ms)
    clocks = sampler.summary(t0, t1)

    # end to end through the public API: pinned host queries in, host results out
    e2e = None
    if not args.no_e2e:
        out_host = torch.empty((nq, 4), dtype=torch.float32).pin_memory()
        def e2e_step():
            # the C-ABI host-buffer call: copies in, lookups, copies out, pipelined in chunks
            # pinned buffers: the lookup kernel reads the queries and writes the results
            # across the CPU-GPU link in place (no staging copies)
            hx.lookup_host(tex, q_host, out=out_host, stream=stream)
        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ksteps = max(1, min(args.steps, 50))
        e0.record(stream)
        for _ in range(ksteps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        ems = reduce_max(e0.elapsed_time(e1), dist, "cuda")
        e2e = {"value": job_rate(nq, ksteps, world, ems), "unit": UNIT,
               "h2d_bytes_per_step": int(q_host.numel() * 4), "d2h_bytes_per_step": int(out_host.numel() * 4),
               "steps": ksteps, "path": "htex_lookup_host on pinned host buffers: the lookup kernel reads the "
                                        "queries from and writes the results to host memory across the link, "
                                        "queries in their given order",
               "link": link_roofline(torch, q_host, out_host, q, out, ems / ksteps)}

    # the spec streaming case: the closed cube, 16x16 RGBA FP32, 2^24 queries
    cube = None if args.no_cube else cube_stream(hx, torch, stream, args)
    serving = None if args.no_serving else serving_bench(hx, torch)
    frame = None if args.no_extras else frame_bench(hx, torch, stream, mesh, tex, positions, args.rows)
    precision = None if args.no_extras else precision_bench(hx, torch, stream)
    precision_asset = None if args.no_extras else precision_asset_bench(hx, torch, stream)
    backward = None if args.no_extras else backward_bench(hx, torch, stream)
    aniso = None if args.no_extras else aniso_bench(hx, torch, stream, mesh, tex)

    peak, peak_src = hbm_peak()
    avg_ms = float(np.mean(launch_ms))
    stages = {"filter_ms": avg_ms, "sort_and_gather_ms": float(np.mean(step_ms)) - avg_ms}
    rate = lambda b: b * nq / (avg_ms / 1e3) / 1e9
    traffic = profiled_traffic("lookup")
    roofline = {"bound": "hbm", "achieved": rate(ab["hot_path"]), "peak": peak, "unit": "GB/s",
                "frac": rate(ab["hot_path"]) / peak, "traffic": traffic, "peak_source": peak_src,
                "algorithmic_bytes_per_lookup": ab["hot_path"],
                "definition": "algorithmic bytes of the hot-path table: 16 query + 16 output + 3 x 16 halfedge "
                              "records + 4 B per in-bounds tap of nonzero weight (mean taps counted on the "
                              "queries); no texture headers (one resolution)",
                "mean_taps": taps, "kernel": "k_lookup_global<u8,4> (lookup_u8.cu)", "avg_launch_ms": avg_ms,
                "packed_record": {"algorithmic_bytes_per_lookup": ab["packed"], "achieved": rate(ab["packed"]),
                                  "frac": rate(ab["packed"]) / peak,
                                  "definition": "the same with this library's one 16-byte pre-evaluated record "
                                                "per halfedge instead of three"},
                "dram": ({"bytes_per_launch": traffic, "achieved": traffic / (avg_ms / 1e3) / 1e9,
                          "frac": traffic / (avg_ms / 1e3) / 1e9 / peak,
                          "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum (profiles/)"}
                         if traffic else None)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        rate, cores, n_s, _ = time_oracle(15.0)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n_s} lookups (passes over 2,097,152 queries) with h uniform on halfedges "
                         f"[0, 4096) of the asset, barycentrics "
                         f"and footprints as the workload (the FP64 copy of all 5.7 GB of texels does not "
                         f"fit host memory); optimistic: the textures of that subset stay in the host caches, "
                         f"unlike the whole asset's"}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(mesh.H, mesh.E, nq, arm_flags_name(args)),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": args.steps * launches_per_step, "step_ms_stages": stages,
            "cube_stream": cube, "serving": serving,
            "precision": precision, "precision_asset": precision_asset, "backward": backward, "frame": frame, "aniso": aniso,
            "source_hash": source_hash(),
        }), flush=True)
    if dist:
        dist.destroy_process_group()


SERVER_CONFIG = {"batch_queries": 1 << 22, "batch_slots": 3, "max_items": 256, "request_chunk": 1 << 20}


def link_roofline(torch, q_host, out_host, q_dev, out_dev, step_ms):
    """The CPU-GPU link as the end-to-end bound: the same bytes the step
    moves (queries in, results out) copied by the copy engines alone,
    host-to-device and device-to-host concurrently on two streams, from
    and to the same pinned buffers; 'frac' = that copy time over the step
    time."""
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def both():
        with torch.cuda.stream(s1):
            q_dev.copy_(q_host, non_blocking=True)
        with torch.cuda.stream(s2):
            out_host.copy_(out_dev, non_blocking=True)

    for _ in range(2):
        both()
    torch.cuda.synchronize()
    reps = 5
    cur = torch.cuda.current_stream()
    ev[0].record(cur)
    for _ in range(reps):
        s1.wait_stream(cur)
        s2.wait_stream(cur)
        both()
        cur.wait_stream(s1)
        cur.wait_stream(s2)
    ev[1].record(cur)
    torch.cuda.synchronize()
    copy_ms = ev[0].elapsed_time(ev[1]) / reps
    nbytes = q_host.numel() * 4 + out_host.numel() * 4
    return {"bound": "cpu-gpu link", "bytes_per_step": int(nbytes), "copy_ms": copy_ms,
            "copy_gbs": nbytes / (copy_ms / 1e3) / 1e9, "achieved_gbs": nbytes / (step_ms / 1e3) / 1e9,
            "frac": copy_ms / step_ms}


def serving_bench(hx, torch, n_requests: int = 2000, load: float = 0.7, repeats: int = 3, server_configs=None):
    """The serving workload: 8 resident assets (halfedges log-spaced over
    [1k, 500k], 128^2..16^2 RGBA8 / FP16 textures), a Poisson stream of
    requests of log-uniform 1k..4M queries with uniform asset tags, offered
    at 'load' times the plain path's back-to-back throughput (one
    htex_lookup_host per request, requests back to back: a fixed measure of
    what the device and the host link deliver), under a device budget of 60%
    of the assets' bytes.  For each of 'repeats' arrival streams (different
    seeds): p50/p99 latency and aggregate lookups/s for the server at that
    budget and with every asset resident, and, on the same arrivals, for the
    plain path (one htex_lookup_host per request in arrival order, all
    assets resident).  Reports the median over the streams and every
    stream's figures; with a list of server configurations, one such result
    per configuration (the same streams)."""
    import htex_synth as syn
    from paper_2207_05618_gb300 import serve
    cfgs = [dict(SERVER_CONFIG, **c) for c in (server_configs or [{}])]
    specs = syn.serving_assets()
    assets = []
    for a in specs:
        fs, fv, V = a["faces"]
        mesh = hx.Mesh(fs, fv, V)
        log2n = np.full(mesh.E, a["log2n"], np.int32)
        tex = (syn.texels_u8 if a["dtype"] == "u8" else syn.texels_f32)(log2n, 4, seed=a["seed"])
        pool, scales = hx.Textures.prepare(mesh, log2n, tex, 4, a["dtype"], hx.BUILD_MIPS | hx.MIRROR_BOUNDARY)
        alone = hx.Textures.upload_pool(mesh, log2n, pool, scales, 4, a["dtype"])
        assets.append({"mesh": mesh, "log2n": log2n, "pool": pool, "scales": scales, "dtype": a["dtype"],
                       "alone": alone})
    total = sum(a["alone"].device_bytes for a in assets)
    qmax = 4_000_000
    qpool = []
    for k, a in enumerate(assets):
        q = torch.from_numpy(hx.pack_queries(*syn.queries(a["mesh"].H, qmax, seed=300 + k,
                                                          footprint="loguniform"))).pin_memory()
        qpool.append(q)
    out_arena = torch.empty((qmax, 4), dtype=torch.float32).pin_memory()
    rng = np.random.default_rng(9)

    def qsrc(a, n):
        off = int(rng.integers(0, qmax - n + 1))
        return qpool[a].data_ptr() + off * 16

    # plain path throughput, requests back to back (sets the offered load)
    _, sizes, tags = syn.poisson_requests(n_requests, 1.0, len(assets), seed=11)
    stream = torch.cuda.current_stream()
    warm = min(50, n_requests)
    for k in range(warm):
        n = int(sizes[k])
        hx.lookup_host(assets[tags[k]]["alone"], qpool[tags[k]][:n], out=out_arena[:n], stream=stream)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for k in range(n_requests):
        n = int(sizes[k])
        hx.lookup_host(assets[tags[k]]["alone"], qpool[tags[k]][:n], out=out_arena[:n], stream=stream)
    torch.cuda.synchronize()
    plain_rate = float(sizes.sum()) / (time.perf_counter() - t)
    rate = load * plain_rate / float(sizes.mean())
    pct = lambda x, p: float(np.percentile(x, p) * 1e3)

    def new_server(cfg, budget):
        server = serve.Server(int(budget), **cfg)
        for a in assets:
            server.add_asset(a["mesh"], a["log2n"], a["pool"], a["scales"], 4, a["dtype"])
        return server

    def run_server(cfg, budget, arrivals, sizes, tags):
        server = new_server(cfg, budget)
        # warm-up: one request per asset (large enough to wait for its asset's upload), served before the
        # timed stream
        serve.replay(server, np.zeros(len(assets)), np.full(len(assets), 131072), np.arange(len(assets)), qsrc,
                     lambda k, a, n: out_arena.data_ptr())
        lat, wall = serve.replay(server, arrivals, sizes, tags, qsrc, lambda k, a, n: out_arena.data_ptr())
        st = server.stats()
        server.close()
        return {"budget_bytes": int(budget), "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                "lookups_per_s": float(sizes.sum()) / wall, "batches": st["batches"], "uploads": st["uploads"],
                "evictions": st["evictions"]}

    def run_plain(arrivals, sizes, tags):
        # one request at a time, first come first served
        lat = np.zeros(n_requests)
        t0 = time.perf_counter()
        for k in range(n_requests):
            while time.perf_counter() < t0 + arrivals[k]:
                pass
            n = int(sizes[k])
            hx.lookup_host(assets[tags[k]]["alone"], qpool[tags[k]][:n], out=out_arena[:n], stream=stream)
            stream.synchronize()
            lat[k] = time.perf_counter() - (t0 + arrivals[k])
        wall = time.perf_counter() - t0
        return {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "lookups_per_s": float(sizes.sum()) / wall}

    streams = [syn.poisson_requests(n_requests, rate, len(assets), seed=12 + r) for r in range(repeats)]
    plain = [run_plain(*st) for st in streams]
    results = []
    for cfg in cfgs:
        # the server's back-to-back capacity at the budget (the same requests, all at once)
        server = new_server(cfg, 0.6 * total)
        _, cap_wall = serve.replay(server, np.zeros(n_requests), sizes, tags, qsrc,
                                   lambda k, a, n: out_arena.data_ptr())
        server.close()
        runs = [{"budget": run_server(cfg, 0.6 * total, *st), "all_resident": run_server(cfg, 2 * total, *st),
                 "plain_path": pl} for st, pl in zip(streams, plain)]
        med = lambda key, sub: float(np.median([x[key][sub] for x in runs]))
        res = {"requests": int(n_requests), "repeats": repeats, "offered_load": load,
               "offered_lookups_per_s": float(rate * sizes.mean()), "plain_back_to_back_lookups_per_s": plain_rate,
               "server_back_to_back_lookups_per_s": float(sizes.sum()) / cap_wall,
               "assets": len(assets), "asset_bytes": int(total), "server_config": cfg,
               "budget_bytes": int(0.6 * total)}
        for key in ("budget", "all_resident", "plain_path"):
            res[key] = {"p50_ms": med(key, "p50_ms"), "p99_ms": med(key, "p99_ms"),
                        "lookups_per_s": med(key, "lookups_per_s"),
                        "p99_ms_each_stream": [x[key]["p99_ms"] for x in runs],
                        "p50_ms_each_stream": [x[key]["p50_ms"] for x in runs]}
        res["budget"]["uploads_each_stream"] = [x["budget"]["uploads"] for x in runs]
        res["budget"]["batches_each_stream"] = [x["budget"]["batches"] for x in runs]
        res["all_resident"]["batches_each_stream"] = [x["all_resident"]["batches"] for x in runs]
        results.append(res)
    for a in assets:
        a["alone"].close()
    return results if server_configs else results[0]


def device_queries(torch, H, n, gen, footprint=False):
    """Uniform queries drawn on the device (h uniform, (u, v) folded-uniform);
    elementwise ops only, so nothing waits for the host."""
    h = torch.randint(0, H, (n,), device="cuda", dtype=torch.int32, generator=gen)
    uv = torch.rand((n, 2), device="cuda", generator=gen)
    uv = torch.where((uv.sum(1) > 1)[:, None], 1 - uv, uv)
    f = (torch.exp2(torch.rand(n, device="cuda", generator=gen) * 8 - 8) if footprint
         else torch.zeros(n, device="cuda"))
    q = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    q[:, 0] = h
    q[:, 1:3] = uv.contiguous().view(torch.int32)
    q[:, 3] = f.contiguous().view(torch.int32)
    return q


def timed(torch, stream, fn, reps, warm=3):
    for _ in range(warm):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def frame_bench(hx, torch, stream, mesh, tex, positions, rows):
    """The paper's workload shape: render the asset's intrinsic
    triangulation at 1920x1080 (one query per pixel: halfedge,
    perspective-correct barycentrics, footprint) and look every pixel up."""
    import htex_synth as syn
    from paper_2207_05618_gb300 import render
    W, H = 1920, 1080
    g = render.Geometry(mesh, positions)
    zc = 0.5 * rows / 256
    M = syn.perspective(45.0, W / H, 0.2, 20.0) @ syn.look_at([2.6, 0.0, zc], [0.0, 0.0, zc], [0, 0, 1])
    q = torch.empty((W * H, 4), dtype=torch.int32, device="cuda")
    out = torch.empty((W * H, 4), dtype=torch.float32, device="cuda")
    raster_ms = timed(torch, stream, lambda: g.rasterize(M, W, H, queries=q, stream=stream), 20)
    lookup_ms = timed(torch, stream, lambda: hx.lookup(tex, q, out=out, stream=stream), 50)
    covered = float((q[:, 0] >= 0).float().mean().item())
    qa = torch.empty((W * H, 8), dtype=torch.int32, device="cuda")
    raster_aniso_ms = timed(torch, stream, lambda: g.rasterize_aniso(M, W, H, queries=qa, stream=stream), 20)
    aniso_ms = timed(torch, stream, lambda: hx.lookup_aniso(tex, qa, 16, out=out, stream=stream), 20)
    g.close()
    return {"width": W, "height": H, "covered_fraction": covered, "raster_ms": raster_ms,
            "lookup_ms": lookup_ms, "frame_ms": raster_ms + lookup_ms,
            "lookups_per_s": W * H * covered / (lookup_ms / 1e3),
            "aniso16_frame_ms": raster_aniso_ms + aniso_ms, "aniso16_lookup_ms": aniso_ms,
            "context": "the paper's Htex RGB frame (GL tessellation + raster + fragment lookup) took "
                       "0.42 ms on an RTX 3090 for a different asset; not a like-for-like figure"}


def precision_bench(hx, torch, stream):
    """Config-1 cube and 2^24 queries with FP32 / FP16 / BF16 / E4M3 texels."""
    import htex_synth as syn
    fs, fv, V, _ = syn.cube()
    mesh = hx.Mesh(fs, fv, V)
    log2n = np.full(mesh.E, 4, np.int32)
    tex32 = syn.texels_f32(log2n, 4, seed=1)
    n = 1 << 24
    q = torch.from_numpy(hx.pack_queries(*syn.queries(mesh.H, n, seed=2))).cuda()
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    res = {}
    for fmt in ("f32", "f16", "bf16", "e4m3"):
        tex = hx.Textures.upload(mesh, log2n, tex32, 4, fmt, hx.BUILD_MIPS)
        ms = timed(torch, stream, lambda: hx.lookup(tex, q, out=out, stream=stream), 50)
        res[fmt] = {"lookups_per_s": n / (ms / 1e3), "ms": ms, "pool_bytes": tex.pool_bytes}
        tex.close()
    return res


def precision_asset_bench(hx, torch, stream, rows: int = 115, nq: int = 1 << 22):
    """Reduced-precision texels where the filter is DRAM-bound: the asset
    mesh recipe at a quarter of its rows (115: about 130k halfedges, the
    asset's density of queries per texture), 64x64 RGBA textures with mip
    chains stored as FP32, FP16, E4M3 (per-texture scale 1) and RGBA8,
    4,194,304 queries with the workload's footprints, sorted
    (HTEX_LOOKUP_BIN).  Texel codes are random (a timing workload: each
    format's error against the FP64 oracle is measured on the cube)."""
    import htex_synth as syn
    fs, fv, V, _ = syn.cylinder(rows=rows)
    mesh = hx.Mesh(fs, fv, V)
    log2n = np.full(mesh.E, 6, np.int32)
    q = torch.from_numpy(hx.pack_queries(*syn.queries(mesh.H, nq, seed=5, footprint="loguniform"))).cuda()
    out = torch.empty((nq, 4), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(77)
    res = {"halfedges": mesh.H, "edges": mesh.E, "queries": nq}
    for fmt in ("f32", "f16", "e4m3", "u8"):
        total, _ = hx.Textures.layout(mesh, log2n, 4, fmt)
        if fmt == "f32":
            pool = rng.random(total // 4, dtype=np.float32).view(np.uint8)
        elif fmt == "f16":
            pool = rng.random(total // 2, dtype=np.float32).astype(np.float16).view(np.uint8)
        elif fmt == "e4m3":
            pool = rng.integers(0, 0x7f, total, dtype=np.uint8)      # finite non-negative codes
        else:
            pool = np.frombuffer(rng.bytes(total), np.uint8)
        tex = hx.Textures.upload_pool(mesh, log2n, pool, np.ones(mesh.E, np.float32), 4, fmt)
        del pool
        ms = timed(torch, stream, lambda: hx.lookup(tex, q, out=out, flags=hx.LOOKUP_BIN, stream=stream), 20)
        res[fmt] = {"lookups_per_s": nq / (ms / 1e3), "ms": ms, "pool_bytes": tex.pool_bytes,
                    "texel_bytes": 4 * {"f32": 4, "f16": 2, "e4m3": 1, "u8": 1}[fmt]}
        tex.close()
    return res


def aniso_bench(hx, torch, stream, mesh, tex, n=1 << 22, reps=10, warm=3, sorted_too=True):
    """Anisotropic lookups on the asset-scale textures: major axis
    log-uniform 2^-8..1 quad widths, anisotropy log-uniform 1..16, uniform
    direction, at most 16 probes.  The kernel is bound by instruction issue,
    not DRAM: its roofline entry gives the DRAM bytes per lookup and the
    issue activity from the committed ncu summary (while the kernel's
    sources are unchanged), the live time, and the DRAM rate they imply."""
    import htex_synth as syn
    h, u, v, _ = syn.queries(mesh.H, n, seed=31)
    rng = np.random.default_rng(32)
    major = np.exp2(rng.uniform(-8.0, 0.0, n))
    minor = major / np.exp(rng.uniform(0.0, np.log(16.0), n))
    th = rng.uniform(0, 2 * np.pi, n)
    c, s = np.cos(th), np.sin(th)
    d = [np.float32(x) for x in (major * c, major * s, -minor * s, minor * c)]
    px2, py2 = d[0] * d[0] + d[1] * d[1], d[2] * d[2] + d[3] * d[3]
    k = np.minimum(np.ceil(np.sqrt(np.maximum(px2, py2) / np.minimum(px2, py2))), 16)
    q = torch.from_numpy(hx.pack_queries_aniso(h, u, v, *d)).cuda()
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    for _ in range(warm):
        hx.lookup_aniso(tex, q, 16, out=out, stream=stream)
    ms = timed(torch, stream, lambda: hx.lookup_aniso(tex, q, 16, out=out, stream=stream), reps, warm=0)
    sorted_ms = (timed(torch, stream, lambda: hx.lookup_aniso(tex, q, 16, out=out, stream=stream,
                                                              flags=hx.LOOKUP_BIN), reps) if sorted_too else None)
    prof = profiled_values("lookup_aniso.md", ANISO_SOURCES)
    peak, _ = hbm_peak()
    roof = {"bound": "instruction issue", "unit": "GB/s", "peak": peak}
    if prof:
        b = prof["aniso_dram_bytes_per_lookup"]
        roof.update({"dram_bytes_per_lookup": b, "achieved": b * n / (ms / 1e3) / 1e9,
                     "frac": b * n / (ms / 1e3) / 1e9 / peak, "issue_active_pct": prof.get("aniso_issue_active_pct"),
                     "source": "profiles/lookup_aniso.md (ncu, quarter-size asset)"})
    return {"queries": n, "max_aniso": 16, "mean_probes": float(k.mean()), "ms": ms,
            "lookups_per_s": n / (ms / 1e3), "probes_per_s": float(k.sum()) / (ms / 1e3),
            "sorted_ms": sorted_ms, "sorted_lookups_per_s": n / (sorted_ms / 1e3) if sorted_ms else None,
            "roofline": roof}


def backward_roofline(taps, bwd_bytes, n, call_ms, peak):
    """The sorted adjoint against HBM: algorithmic bytes (query, gradient
    row, one C-float atomic add per tap) over the whole sorted call's time,
    and, while the committed ncu summary matches the kernel's sources, the
    DRAM bytes the kernel moves per query."""
    r = {"bound": "L2 atomics + hbm (latency-bound: see profiles/backward_differentiation.md)", "unit": "GB/s",
         "peak": peak, "mean_taps": taps, "algorithmic_bytes_per_query": bwd_bytes,
         "achieved": bwd_bytes * n / (call_ms / 1e3) / 1e9,
         "frac": bwd_bytes * n / (call_ms / 1e3) / 1e9 / peak,
         "atomic_adds_per_s": taps * n / (call_ms / 1e3),
         "note": "whole htex_lookup_backward call with HTEX_LOOKUP_BIN (range sort carrying the gradient rows, "
                 "then the warp-aggregated adjoint)"}
    prof = profiled_values("backward_differentiation.md", BACKWARD_SOURCES)
    if prof:
        b = prof["backward_dram_bytes_per_query"]
        r["dram"] = {"bytes_per_query": b, "achieved": b * n / (call_ms / 1e3) / 1e9,
                     "frac": b * n / (call_ms / 1e3) / 1e9 / peak}
    return r


def backward_bench(hx, torch, stream):
    """Config 4: closed sphere (about 104k halfedges), 32x32 RGB FP32 edge
    textures, 2M queries: forward and backward throughput (plain and
    sorted), and a 200-step Adam fit (fresh 2M device-drawn queries per
    step, drawn before the timed loop) from zero texels to a smooth target
    asset, with each stage of a step timed on its own."""
    import htex_synth as syn
    from paper_2207_05618_gb300 import fit
    fs, fv, V, _ = syn.uv_sphere()
    mesh = hx.Mesh(fs, fv, V)
    log2n = np.full(mesh.E, 5, np.int32)
    target = hx.Textures.upload(mesh, log2n, syn.texels_smooth(log2n, 3, seed=2), 3, "f32", hx.BUILD_MIPS)
    tex = hx.Textures.upload(mesh, log2n, np.zeros(mesh.E * 1024 * 3, np.float32), 3, "f32", hx.BUILD_MIPS)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4)
    n = 2_000_000
    q = device_queries(torch, mesh.H, n, gen)
    g = torch.randn((n, 3), device="cuda", generator=gen)
    grad = torch.zeros(tex.pool_elements, dtype=torch.float32, device="cuda")
    fwd_ms = timed(torch, stream, lambda: hx.lookup(target, q, stream=stream), 50)
    bwd_ms = timed(torch, stream, lambda: hx.lookup_backward(target, q, g, grad_texels=grad, stream=stream), 50)
    fwd_sorted_ms = timed(torch, stream, lambda: hx.lookup(target, q, flags=hx.LOOKUP_BIN, stream=stream), 50)
    bwd_sorted_ms = timed(torch, stream, lambda: hx.lookup_backward(target, q, g, grad_texels=grad,
                                                                    flags=hx.LOOKUP_BIN, stream=stream), 50)
    qh = q.cpu().numpy()
    taps = mean_taps(mesh.halfedges(), 5, (qh[:, 0], qh[:, 1].view(np.float32), qh[:, 2].view(np.float32),
                                           qh[:, 3].view(np.float32)))
    bwd_bytes = 16 + 12 + taps * 12          # query, upstream gradient row, one 12-byte atomic add per tap
    peak, _ = hbm_peak()

    # the fit: every step's queries and targets drawn before the timed loop
    steps = 200
    gen_ms = timed(torch, stream, lambda: device_queries(torch, mesh.H, n, gen), 10)
    pre = []
    for _ in range(steps):
        qq = device_queries(torch, mesh.H, n, gen)
        pre.append((qq, hx.lookup(target, qq)))
    m1 = torch.zeros(tex.pool_elements, dtype=torch.float32, device="cuda")
    m2 = torch.zeros_like(m1)
    qq, tt = pre[0]

    def loss_stage():
        d = hx.lookup(tex, qq, stream=stream) - tt
        return d.double().pow(2).sum() / d.numel()

    stages = {"query_generation_ms (outside the timed loop)": gen_ms,
              "lookup_and_loss_ms": timed(torch, stream, loss_stage, 20),
              "backward_sorted_ms": timed(torch, stream, lambda: hx.lookup_backward(
                  tex, qq, tt, grad_texels=grad, flags=hx.LOOKUP_BIN, stream=stream), 20),
              "adam_ms": timed(torch, stream, lambda: tex.adam_step(None, grad, m1, m2, 1, 0.0), 20)}
    # a short untimed fit first: the first step of the first fit in a process
    # stalled the host for about 0.5 s (a one-time cost, measured with
    # per-step events), which is not a cost of the step; every fit starts
    # from zero texels, so the timed fit is unaffected by it
    fit.fit(tex, lambda step: pre[step], steps=3, lr=0.05)
    r = fit.fit(tex, lambda step: pre[step], steps=steps, lr=0.05)
    target.close()
    tex.close()
    return {"halfedges": mesh.H, "edges": mesh.E, "queries": n,
            "forward_lookups_per_s": n / (fwd_ms / 1e3), "backward_queries_per_s": n / (bwd_ms / 1e3),
            "forward_sorted_lookups_per_s": n / (fwd_sorted_ms / 1e3),
            "backward_sorted_queries_per_s": n / (bwd_sorted_ms / 1e3),
            "backward_ms": bwd_ms, "backward_sorted_ms": bwd_sorted_ms,
            "roofline": backward_roofline(taps, bwd_bytes, n, bwd_sorted_ms, peak),
            "fit": {"steps": r.steps, "initial_loss": r.losses[0], "final_loss": r.losses[-1],
                    "final_over_initial": r.ratio, "ms_per_step": r.seconds * 1e3 / r.steps,
                    "stages": stages, "loss_every_20": r.losses[::20]}}


def cube_stream(hx, torch, stream, args):
    """Closed cube, 12 textures 16x16 RGBA FP32 + mips, 2^24 queries at
    level 0: 32 algorithmic bytes per lookup (query + output)."""
    import htex_synth as syn
    fs, fv, V, _ = syn.cube()
    mesh = hx.Mesh(fs, fv, V)
    log2n = np.full(mesh.E, 4, np.int32)
    tex = hx.Textures.upload(mesh, log2n, syn.texels_f32(log2n, 4, seed=1), 4, "f32", hx.BUILD_MIPS)
    res = {}
    for name, n in (("batched_2^24", 1 << 24), ("single_65536", 65536)):
        q = torch.from_numpy(hx.pack_queries(*syn.queries(mesh.H, n, seed=2))).cuda()
        out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        for _ in range(5):
            hx.lookup(tex, q, out=out, stream=stream)
        reps = 50
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            hx.lookup(tex, q, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"lookups_per_s": n / (ms / 1e3), "ms": ms, "gbs": 32.0 * n / (ms / 1e3) / 1e9}
    peak, _ = hbm_peak()
    res["batched_2^24"]["frac_of_hbm"] = res["batched_2^24"]["gbs"] / peak
    tex.close()
    return res


if __name__ == "__main__":
    main()
