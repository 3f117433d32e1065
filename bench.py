"""Benchmark: exact truss decomposition throughput on GB300.

Workload of one step (default): the full decomposition -- CSR build, support,
triangle lists, level-synchronous peel, per-row scatter -- of the Chung-Lu
graph with n = 2^24 vertices, power-law expected degrees of exponent 2.1,
mean degree 20, expected degrees capped at 2^16, seed 2 (167,772,160 distinct
undirected edges, 3.5e9 triangles), inputs resident in HBM.  ``--workload
mid`` times the R-MAT scale-20 graph instead.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload large|mid] [--mode single|batch|serve|top|core|budget]

Prints ONE JSON line (rank 0).  `value` is distinct edges decomposed per
second summed over ranks (each rank decomposes its own replica: one graph does
not shard).  `e2e` is the same metric through the C ABI with pinned host
buffers: moving the rows to the GPU and the outputs back is inside the timed
region (the library's kernels read and write pinned buffers in place over
the host link; the byte counts are those moved).  `roofline` reports
the dominant kernel's algorithmic bytes (the per-edge formulas that
truss_run_stats documents) over its CUDA-event duration against the measured
HBM copy bandwidth, with the kernel's bytes by its own per-unit figures
beside them.  `cpu_baseline` is the CPU oracle (single thread) on a bounded
prefix of the same rows, with the oracle's time on the whole graph beside it.
`--impl reference` times that oracle as the reference arm.

The single-mode line also carries `batch` (the 4,096-graph mixed batch in one
truss_decompose_batch call against a loop of per-graph truss_decompose calls
over the same steps) and `serve` (a Poisson stream of 200 R-MAT requests per
second for 60 s through the truss_serve_* server, each request generated on
the GPU shortly before its arrival; p50/p99 latency from the scheduled
arrival, achieved against offered edges/s), each with its own timing and
clocks; `--no-batch` / `--no-serve` leave them out, and `--mode batch|serve`
prints either alone.  Under torchrun each rank takes its own share of the
graphs (batch) or of the arrivals (serve); no collective touches the data
path.
"""
from __future__ import annotations

import argparse
import json
import os
import queue
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen  # noqa: E402

METRIC = "edges/sec full truss decomposition (bit-exact)"
UNIT = "edges/s"
WORKLOADS = {
    "large": ("large: Chung-Lu n=2^24, expected-degree exponent 2.1, mean degree 20, cap 2^16, "
              "seed 2; 167,772,160 distinct undirected edges; int32 ids, int64 CSR offsets"),
    "mid": ("mid: R-MAT scale 20, edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), seed 1; "
            "16,777,216 raw rows -> 15,702,720 distinct undirected edges; int32 ids, "
            "int64 CSR offsets"),
}
WORKLOAD = WORKLOADS["large"]
CPU_SAMPLE_ROWS = 8_000_000     # cpu_baseline: oracle on this prefix of the rows
REF_SAMPLE_ROWS = 2_000_000     # --impl reference: oracle per step on this prefix
L2_FLUSH_BYTES = 512 << 20
DIGESTS = os.path.join(ROOT, "tests", "golden", "digests.json")


def load_rows(workload: str, rows: int | None = None):
    """(n, src, dst) of a named workload, or only its first `rows` rows."""
    if workload == "large":
        return graphgen.large(rows=rows)
    if workload == "mid":
        n, s, d = graphgen.mid()
        if rows is not None:
            s, d = s[:rows].copy(), d[:rows].copy()
        return n, s, d
    raise ValueError(workload)


def full_graph_oracle(workload: str):
    """The oracle's recorded time on the whole graph (the run that wrote the
    stored digests; single thread, x86-64 host), or None."""
    try:
        with open(DIGESTS) as f:
            d = json.load(f).get(workload)
    except (OSError, ValueError):
        return None
    if not d or not d.get("oracle_seconds"):
        return None
    return {"seconds": d["oracle_seconds"], "value": d["m"] / d["oracle_seconds"], "unit": UNIT,
            "cores": 1, "host": "x86-64, one core (the run that wrote tests/golden/digests.json)"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def csrc_sha256() -> str:
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_1205_6693_gb300", "csrc", "*"))):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(os.path.basename(f).encode())
            with open(f, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


def traffic_for(stage: str, workload: str = "mid"):
    """DRAM bytes per launch of `stage`'s kernel(s) on `workload` from the
    committed ncu summary profiles/traffic_<workload>.txt, or None if there
    is none or the CUDA sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.txt")
    if not os.path.exists(path):
        return None
    sha, rows = None, {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == "csrc_sha256":
                sha = parts[1]
            elif len(parts) >= 4:  # a stage may run several kernels: add them up
                rows[parts[0]] = rows.get(parts[0], 0) + int(parts[2]) + int(parts[3])
    if sha != csrc_sha256():
        return None
    return rows.get(stage)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the GPU this rank uses: its local rank, unless TRUSS_BENCH_DEVICE names
    # one GPU for every rank (the multi-rank test on one GPU)
    local = int(os.environ.get("TRUSS_BENCH_DEVICE", local))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during timing."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_rate(workload: str, rows_prefix: int):
    """Oracle (single thread) on a prefix of the workload's rows."""
    import oracle
    n, s, d = load_rows(workload, rows_prefix)
    t0 = time.perf_counter()
    r = oracle.truss(n, s, d)
    dt = time.perf_counter() - t0
    return r.m, dt


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    import oracle
    wl = args.workload
    n, s, d = load_rows(wl, REF_SAMPLE_ROWS)
    for _ in range(args.warmup):
        oracle.truss(n, s, d)
    times, m = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.truss(n, s, d)
        times.append(time.perf_counter() - t0)
        m = r.m
    tot = sum(times)
    value = m * args.steps / tot
    sample = (f"first {REF_SAMPLE_ROWS:,} rows of the workload ({m:,} distinct edges) per step, "
              f"oracle = single-threaded Algorithm 2 in C; a prefix is sparser in triangles "
              f"than the whole graph, so this rate is above the oracle's whole-graph rate")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOADS[wl], "sample_rows": REF_SAMPLE_ROWS},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample, "full_graph": full_graph_oracle(wl)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _dist_init(ws, local):
    """Device and process group of this rank.  NCCL across GPUs by default;
    TRUSS_BENCH_BACKEND=gloo and TRUSS_BENCH_DEVICE=<index> run the ranks
    over gloo on one named GPU (the multi-rank test uses this: its ranks'
    kernels never wait on one another)."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        backend = os.environ.get("TRUSS_BENCH_BACKEND", "nccl")
        if backend == "nccl":
            dist.init_process_group("nccl", device_id=dev)
        else:
            dist.init_process_group(backend)
    return dev, dist


def _max_over_ranks(dist, dev, x: float) -> float:
    if dist is None:
        return x
    import torch
    on = dev if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=on)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def schedule_for(args, local, rows, graphs, call):
    """Schedule opts for this GPU and size bucket: from the autotuner's cache
    or the schedules shipped with the package, else tuned now (untimed,
    before the warm-up), else the defaults."""
    from paper_1205_6693_gb300 import autotune
    got, src = autotune.lookup_any(autotune.gpu_key(local), rows, graphs)
    if got is not None:
        return got, src
    if args.no_tune:
        return {}, "default"
    return autotune.tune_call(local, call, rows, graphs)["opts"], "tuned"


def _timed_steps(fn, steps, warmup, stream, flush, dev, dist=None):
    """W untimed calls, then K calls each bracketed by CUDA events on the
    calling stream, with an L2 flush (a 512 MB write) before each, outside
    the timed region.  Returns the per-step milliseconds."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    out = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        out.append(e0.elapsed_time(e1))
    if dist:
        dist.barrier()
    return out


def batch_section(args, ws, rank, local, dev, dist):
    """Batched form: the mixed 4,096-graph batch in one truss_decompose_batch
    call, against per-graph truss_decompose calls on the same stream and the
    same device buffers, over the same steps and warm-up."""
    import torch
    from paper_1205_6693_gb300 import truss as T
    from paper_1205_6693_gb300.shard import shard_range
    g0, g1 = shard_range(args.graphs, rank, ws)
    ns, off, src_np, dst_np = graphgen.batch(g1 - g0, first=g0)
    G, rows = len(ns), int(off[-1])
    src_h, dst_h = torch.from_numpy(src_np).pin_memory(), torch.from_numpy(dst_np).pin_memory()
    sup_h = torch.empty(rows, dtype=torch.int32).pin_memory()
    tr_h = torch.empty(rows, dtype=torch.int32).pin_memory()
    km_h = torch.empty(G, dtype=torch.int32).pin_memory()
    src = torch.from_numpy(src_np).to(dev)
    dst = torch.from_numpy(dst_np).to(dev)
    sup, tr = torch.empty_like(src), torch.empty_like(src)
    kmax = torch.empty(G, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    sched, sched_src = schedule_for(
        args, local, rows, G,
        lambda c: (c.decompose_batch(ns, off, src, dst, sup, tr, kmax), (sup, tr, kmax))[1])
    ctx = T.Context(local, profile=True, **sched)
    K, W = args.batch_steps, args.batch_warmup
    launches = []

    def batched():
        ctx.decompose_batch(ns, off, src, dst, sup, tr, kmax, stream=stream)
        launches.append(ctx.stats()["launches"])

    def loop():
        for g in range(G):
            a, b = int(off[g]), int(off[g + 1])
            ctx.decompose(int(ns[g]), src[a:b], dst[a:b], sup[a:b], tr[a:b], stream=stream)

    sampler = ClockSampler(local)
    sampler.start()
    ms = _timed_steps(batched, K, W, stream, flush, dev, dist)
    st = ctx.stats()
    loop_ms = _timed_steps(loop, K, W, stream, flush, dev, dist)
    clocks = sampler.stop()
    # end to end: host buffers through the C ABI (copies inside the timed region)
    e2e_ms = _timed_steps(
        lambda: ctx.decompose_batch(ns, off, src_h, dst_h, sup_h, tr_h, km_h, stream=stream),
        K, 1, stream, flush, dev, dist)
    ctx.close()
    tot = _max_over_ranks(dist, dev, sum(ms))
    loop_tot = _max_over_ranks(dist, dev, sum(loop_ms))
    e2e_tot = _max_over_ranks(dist, dev, sum(e2e_ms))
    value = args.graphs * K / (tot / 1e3)
    loop_value = args.graphs * K / (loop_tot / 1e3)
    return {"metric": "batched graphs/s (bit-exact truss decomposition)", "value": value,
            "unit": "graphs/s", "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": tot / K, "higher_is_better": True, "scaling": "weak",
            "config": {"workload": (f"{args.graphs} graphs: ER / R-MAT / ER+clique, edges "
                                    "log-uniform in [64, 65536], seed SplitMix64(0xB47C^g)"),
                       "rows": rows * ws, "edges_rank0": st["m"],
                       "triangles_rank0": st["triangles"],
                       "parallelism": f"graphs sharded over {ws} rank(s)",
                       "l2_flush": "512 MB write before every timed step",
                       "schedule": {"opts": sched, "source": sched_src}},
            "per_graph_loop": {"value": loop_value, "unit": "graphs/s",
                               "ms_per_step": loop_tot / K, "steps": K, "warmup": W},
            "speedup_vs_loop": value / loop_value,
            "e2e": {"value": args.graphs * K / (e2e_tot / 1e3), "unit": "graphs/s",
                    "h2d_bytes_per_step": 8 * rows * ws,
                    "d2h_bytes_per_step": (8 * rows + 4 * G) * ws},
            "gpu_launches": int(sum(launches[W:])), "clocks": clocks}


def run_batch(args, ws, rank, local):
    dev, dist = _dist_init(ws, local)
    line = batch_section(args, ws, rank, local, dev, dist)
    if rank == 0:
        line.update({"vs_baseline": None, "dtype": "int32", "data": "synthetic"})
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_top(args, ws, rank, local):
    """Top-t classes (Algorithm 7) of the mid graph: truss_top against a full
    truss_decompose of the same graph on the same stream."""
    import torch
    from paper_1205_6693_gb300 import truss as T
    dev, dist = _dist_init(ws, local)
    n, src_np, dst_np = graphgen.mid()
    src = torch.from_numpy(src_np).to(dev)
    dst = torch.from_numpy(dst_np).to(dev)
    out = torch.empty_like(src)
    sup = torch.empty_like(src)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ctx = T.Context(local, profile=True)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        tot = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            tot += e0.elapsed_time(e1)
        return _max_over_ranks(dist, dev, tot)

    ms = timed(lambda: ctx.top(n, src, dst, args.t, out, stream=stream))
    st = ctx.stats()
    full_ms = timed(lambda: ctx.decompose(n, src, dst, sup, out, stream=stream))
    ctx.close()
    if rank == 0:
        m = st["m"]
        line = {"metric": f"top-{args.t} truss classes (Algorithm 7), edges/s of the input graph",
                "value": ws * m * args.steps / (ms / 1e3), "unit": "edges/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32", "data": "synthetic",
                "config": {"workload": WORKLOADS["mid"], "t": args.t, "m": m, "kmax": st["kmax"],
                           "candidate_edges": st["candidates"], "rounds": st["rounds"],
                           "stage_ms": {"build_support_psi": round(st["ms_support"], 3),
                                        "candidate_rounds": round(st["ms_peel"], 3)},
                           "parallelism": f"replicas x{ws}", "l2_flush": True},
                "full_decomposition_ms": full_ms / args.steps,
                "speedup_vs_full": full_ms / ms}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_core(args, ws, rank, local):
    """Vertex core numbers (truss_core) of the mid graph."""
    import torch
    from paper_1205_6693_gb300 import truss as T
    dev, dist = _dist_init(ws, local)
    n, src_np, dst_np = graphgen.mid()
    src = torch.from_numpy(src_np).to(dev)
    dst = torch.from_numpy(dst_np).to(dev)
    core = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ctx = T.Context(local, profile=True)
    for _ in range(args.warmup):
        ctx.core(n, src, dst, core, stream=stream)
    torch.cuda.synchronize(dev)
    tot = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kc = ctx.core(n, src, dst, core, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        tot += e0.elapsed_time(e1)
    st = ctx.stats()
    ctx.close()
    ms = _max_over_ranks(dist, dev, tot)
    if rank == 0:
        line = {"metric": "edges/sec core decomposition (vertex core numbers, bit-exact)",
                "value": ws * st["m"] * args.steps / (ms / 1e3), "unit": "edges/s",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": WORKLOADS["mid"], "m": st["m"], "n": n, "max_core": kc,
                           "levels": st["levels"], "subrounds": st["subrounds"],
                           "stage_ms": {"build": round(st["ms_build"], 3),
                                        "peel": round(st["ms_peel"], 3)},
                           "parallelism": f"replicas x{ws}", "l2_flush": True}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_budget(args, ws, rank, local):
    """Bottom-up decomposition under a working-set budget (Section 5) of an
    R-MAT graph, against the in-memory decomposition of the same graph."""
    import torch
    from paper_1205_6693_gb300 import truss as T
    dev, dist = _dist_init(ws, local)
    sc = args.rmat_scale
    if sc == 20:
        n, src_np, dst_np = graphgen.mid()
        workload = WORKLOADS["mid"]
    else:
        src_np, dst_np = graphgen.rmat_raw(sc, 16 * 2 ** sc, seed=1)
        n = 2 ** sc
        workload = f"R-MAT scale {sc}, edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), seed 1"
    src = torch.from_numpy(src_np).to(dev)
    dst = torch.from_numpy(dst_np).to(dev)
    sup, tr = torch.empty_like(src), torch.empty_like(src)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    ctx = T.Context(local, profile=True)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        tot = 0.0
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            tot += e0.elapsed_time(e1)
        return _max_over_ranks(dist, dev, tot)

    ms = timed(lambda: ctx.decompose_budget(n, src, dst, args.budget, sup, tr, stream=stream))
    st = ctx.stats()
    full_ms = timed(lambda: ctx.decompose(n, src, dst, sup, tr, stream=stream))
    ctx.close()
    if rank == 0:
        m = st["m"]
        line = {"metric": "edges/sec truss decomposition under a working-set budget "
                          "(Section 5 bottom-up, bit-exact)",
                "value": ws * m * args.steps / (ms / 1e3), "unit": "edges/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32", "data": "synthetic",
                "config": {"workload": workload, "m": m, "kmax": st["kmax"],
                           "budget_edges": args.budget, "subgraphs": st["rounds"],
                           "largest_subgraph_edges": st["candidates"],
                           "parallelism": f"replicas x{ws}", "l2_flush": True},
                "in_memory_ms": full_ms / args.steps}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def serve_section(args, ws, rank, local, dev, dist):
    """Served form: a Poisson request stream replayed in real time through the
    server.  Each request's edge list is generated on the GPU (side stream)
    shortly before its scheduled arrival and released once its result is
    back, so a stream of any length runs within memory.  Latency runs from
    the scheduled arrival to the result in host memory."""
    import torch
    from paper_1205_6693_gb300 import truss as T
    count = max(1, int(round(args.rate * args.window)))
    t_arr, m_req = graphgen.serve_schedule(count * ws, rate=args.rate * ws)
    mine = list(range(rank, count * ws, ws))
    side = torch.cuda.Stream(dev)

    def gen(j):
        m = int(m_req[j])
        scale = graphgen.serve_scale(m)
        with torch.cuda.stream(side):
            s, d = graphgen.rmat_raw_cuda(scale, m, seed=graphgen.gg_seed(3, j), device=dev,
                                          cuda_stream=side.cuda_stream)
        side.synchronize()
        return 1 << scale, s, d

    opts = T.truss_serve_opts()
    opts.streams = args.serve_streams
    opts.max_queue = args.serve_queue
    ctx = T.truss_ctx_create(local)
    srv = T.truss_serve_start(ctx, opts)
    # warm-up: the first requests of the stream, outside the timed run
    for j in mine[: min(4, len(mine))]:
        n, s, d = gen(j)
        T.truss_serve_wait(srv, T.truss_serve_submit(srv, n, s, d))
    T.truss_serve_stop(srv)
    srv = T.truss_serve_start(ctx, opts)
    T.truss_ctx_destroy(ctx)
    if dist:
        dist.barrier()
    results = queue.Queue()
    t0 = time.perf_counter() + args.serve_lead
    late = [0.0]

    def client():
        try:
            for i, j in enumerate(mine):
                w = t0 + t_arr[j] - args.serve_lead - time.perf_counter()
                if w > 0:
                    time.sleep(w)
                n, s, d = gen(j)
                w = t0 + t_arr[j] - time.perf_counter()
                if w > 0:
                    time.sleep(w)
                delay = time.perf_counter() - (t0 + t_arr[j])
                late[0] = max(late[0], delay)
                try:
                    tk = T.truss_serve_submit(srv, n, s, d)
                except T.TrussError as e:
                    if e.code != T.TRUSS_EBUSY:
                        raise
                    tk = None
                results.put((tk, delay, int(m_req[j]), len(s), (s, d)))
        finally:
            results.put(None)

    sampler = ClockSampler(local)
    sampler.start()
    th = threading.Thread(target=client)
    th.start()
    lat, m_done, rows_done, rejected, failed = [], 0, 0, 0, 0
    t_last = t0
    while True:
        item = results.get()
        if item is None:
            break
        tk, delay, m, rws, bufs = item
        if tk is None:
            rejected += 1
            continue
        try:
            st = T.truss_serve_wait(srv, tk)
        except T.TrussError:
            failed += 1
            continue
        t_last = max(t_last, time.perf_counter())
        lat.append(st["total_ms"] + 1e3 * delay)
        m_done += st["m"]
        rows_done += rws
        del bufs
    th.join()
    wall = t_last - t0
    stats = T.truss_serve_stop(srv)
    clocks = sampler.stop()
    lat.sort()
    p = (lambda q: lat[min(len(lat) - 1, int(q * (len(lat) - 1) + 0.5))]) if lat else (lambda q: None)
    offered = float(sum(int(m_req[j]) for j in mine)) / args.window
    return {"metric": "served p99 latency (bit-exact truss decomposition)", "value": p(0.99),
            "unit": "ms", "n_gpus": ws, "steps": len(mine), "warmup": min(4, len(mine)),
            "higher_is_better": False, "scaling": "weak",
            "config": {"workload": (f"Poisson {args.rate:g} req/s for {args.window:g} s (seed 3), "
                                    "R-MAT (0.57,0.19,0.19,0.05) requests, raw samples "
                                    "log-uniform in [1e3, 5e7], generated on the GPU "
                                    f"{args.serve_lead:g} s before arrival"),
                       "requests": len(mine), "streams": args.serve_streams,
                       "max_queue": args.serve_queue},
            "p50_ms": p(0.50), "p99_ms": p(0.99), "mean_ms": sum(lat) / len(lat) if lat else None,
            "completed": len(lat), "rejected_at_submit": rejected, "failed": failed,
            "achieved_edges_per_s": m_done / wall if wall > 0 else None,
            "offered_samples_per_s": offered, "wall_s": wall,
            "submit_late_max_ms": 1e3 * late[0],
            "server": stats, "clocks": clocks,
            "e2e": {"value": p(0.99), "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": int(8 * rows_done / max(1, len(lat))),
                    "note": ("each latency includes the copy of the request's result to host "
                             "memory; inputs are generated on the device before arrival")}}


def run_serve(args, ws, rank, local):
    dev, dist = _dist_init(ws, local)
    line = serve_section(args, ws, rank, local, dev, dist)
    if rank == 0:
        line.update({"vs_baseline": None, "dtype": "int32", "data": "synthetic"})
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_single(args, ws, rank, local):
    import torch
    from paper_1205_6693_gb300 import truss as T
    dev, dist = _dist_init(ws, local)
    wl = args.workload
    if args.rmat_scale:
        sc = args.rmat_scale
        src_np, dst_np = graphgen.rmat_raw(sc, 16 * 2 ** sc, seed=1)
        n = 2 ** sc
        workload = (f"R-MAT scale {sc}, edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), "
                    f"seed 1 (profiling case)")
    else:
        n, src_np, dst_np = load_rows(wl)
        workload = WORKLOADS[wl]
    rows = len(src_np)
    # pinned host buffers of the e2e leg, allocated before any device work
    # (like a serving process that keeps its staging buffers): on this machine,
    # pinned memory allocated after the 200 GB workspace copied at a tenth
    # of the link's rate, torch's own copies included
    src_h = torch.from_numpy(src_np).pin_memory()
    dst_h = torch.from_numpy(dst_np).pin_memory()
    sup_h = torch.empty(rows, dtype=torch.int32).pin_memory()
    tr_h = torch.empty(rows, dtype=torch.int32).pin_memory()
    src = torch.from_numpy(src_np).to(dev)
    dst = torch.from_numpy(dst_np).to(dev)
    sup = torch.empty_like(src)
    tr = torch.empty_like(src)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # algorithmic bytes (separate, untimed call)
    cctx = T.Context(local, count_bytes=True)
    cctx.decompose(n, src, dst, sup, tr)
    counts = cctx.stats()
    cctx.close()

    sched, sched_src = schedule_for(
        args, local, rows, 1, lambda c: (c.decompose(n, src, dst, sup, tr), (sup, tr))[1])
    ctx = T.Context(local, profile=True, **sched)
    stage = {"support": [], "lists": [], "peel": [], "build": []}
    launches = []
    res = {}

    def step():
        res["kmax"] = ctx.decompose(n, src, dst, sup, tr, stream=stream)
        st = ctx.stats()
        res["st"] = st
        for k in stage:
            stage[k].append(st["ms_" + k])
        launches.append(st["launches"])

    sampler = ClockSampler(local)
    sampler.start()
    step_ms = _timed_steps(step, args.steps, max(args.warmup, 0), stream, flush, dev, dist)
    clocks = sampler.stop()
    for k in stage:
        stage[k] = stage[k][max(args.warmup, 0):]
    st, kmax = res["st"], res["kmax"]
    total_ms = _max_over_ranks(dist, dev, sum(step_ms))
    m = st["m"]
    value = ws * m * args.steps / (total_ms / 1e3)

    # end to end through the C ABI with the pinned host buffers
    e2e_stage = {"build": [], "support": [], "lists": [], "peel": [], "scatter": []}
    e2e_layout = []

    def e2e_step():
        ctx.decompose(n, src_h, dst_h, sup_h, tr_h, stream=stream)
        st2 = ctx.stats()
        for k in e2e_stage:
            e2e_stage[k].append(st2["ms_" + k])
        e2e_layout.append(st2["lists_layout"])

    e2e_ms = _timed_steps(e2e_step, args.steps, 1, stream, flush, dev, dist)
    e2e_value = ws * m * args.steps / (_max_over_ranks(dist, dev, sum(e2e_ms)) / 1e3)
    e2e_med = {k: round(statistics.median(v[1:]), 3) for k, v in e2e_stage.items()}
    ctx.close()
    del src, dst, sup, tr, src_h, dst_h, sup_h, tr_h
    torch.cuda.empty_cache()

    batch = None if args.no_batch else batch_section(args, ws, rank, local, dev, dist)
    torch.cuda.empty_cache()
    serve = None if args.no_serve else serve_section(args, ws, rank, local, dev, dist)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = peaks()
    med = {k: statistics.median(v) for k, v in stage.items()}
    byts = {"support": (counts["bytes_support"], counts["design_bytes_support"]),
            "lists": (counts["bytes_lists"], counts["bytes_lists"]),
            "peel": (counts["bytes_peel"], counts["design_bytes_peel"])}
    stages = {}
    for k, (b, bd) in byts.items():
        t = med[k] / 1e3
        stages[k] = {"ms": round(med[k], 3), "algorithmic_bytes": b,
                     "frac": (b / t / 1e9 / peak) if t > 0 else None,
                     "design_bytes": bd, "design_frac": (bd / t / 1e9 / peak) if t > 0 else None}
    dom = max(("support", "lists", "peel"), key=lambda k: med[k])
    dms = med[dom]
    dbytes, dbytes_design = byts[dom]
    achieved = dbytes / (dms / 1e3) / 1e9 if dms > 0 else 0.0
    kernel_name = {"support": "k_support_v",
                   "lists": "k_lists_from_records + k_lists_vw",
                   "peel": "k_peel (persistent, cooperative)"}[dom]
    traffic = None if args.rmat_scale else traffic_for(dom, wl)

    cpu = None
    if ws == 1 and not args.no_cpu_baseline and not args.rmat_scale:
        rows_s = CPU_SAMPLE_ROWS if wl == "large" else 4_000_000
        m_s, dt = oracle_rate(wl, rows_s)
        cpu = {"value": m_s / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": (f"prefix sample: the first {rows_s:,} rows of the workload "
                          f"({m_s:,} distinct edges), {dt:.1f} s single-threaded; a prefix is "
                          f"sparser in triangles than the whole graph, so this rate is above "
                          f"the oracle's whole-graph rate in full_graph"),
               "full_graph": full_graph_oracle(wl)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": workload, "m": m, "rows": rows, "triangles": st["triangles"],
                   "kmax": kmax, "parallelism": f"replicas x{ws}",
                   "l2_flush": "512 MB write before every timed step; inputs exceed L2",
                   "stage_ms_median": {k: round(v, 3) for k, v in med.items()},
                   "levels": st["levels"], "subrounds": st["subrounds"],
                   "lists_layout": st["lists_layout"],
                   "schedule": {"opts": sched, "source": sched_src}},
        "roofline": {"bound": "hbm", "kernel": kernel_name, "achieved": achieved, "peak": peak,
                     "peak_kind": f"{peak_kind} (HBM copy, burst)", "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes": dbytes,
                     "bytes_rule": ("per-edge formulas of truss_run_stats (bytes_support, "
                                    "bytes_peel); lists: the list passes' own figures"),
                     "design_bytes": dbytes_design,
                     "design_frac": dbytes_design / (dms / 1e3) / 1e9 / peak if dms > 0 else None,
                     "stages": stages,
                     "peel_counts": {k: counts[k] for k in (
                         "peel_sum_min_alive", "peel_sum_min_alive_start",
                         "peel_alive_levels", "peel_entries",
                         "peel_dead_entries", "peel_dead_earlier", "peel_decrements",
                         "peel_scanned")}},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * rows,
                "d2h_bytes_per_step": 8 * rows,
                "stage_ms_median": e2e_med, "lists_layout": e2e_layout[-1]},
        "gpu_launches": int(sum(launches[max(args.warmup, 0):])),
        "clocks": clocks,
        "batch": batch,
        "serve": serve,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rmat-scale", type=int, default=0,
                    help="single mode: time an R-MAT graph of this scale instead (profiling "
                         "cases)")
    ap.add_argument("--no-tune", action="store_true",
                    help="use cached, shipped or default schedules; never run the autotuner")
    ap.add_argument("--mode", default="single",
                    choices=["single", "batch", "serve", "top", "core", "budget"])
    ap.add_argument("--no-batch", action="store_true", help="single mode: leave out `batch`")
    ap.add_argument("--no-serve", action="store_true", help="single mode: leave out `serve`")
    ap.add_argument("--budget", type=int, default=4_000_000,
                    help="budget mode: edges per neighbourhood subgraph")
    ap.add_argument("--t", type=int, default=10, help="top mode: number of top classes")
    ap.add_argument("--graphs", type=int, default=4096, help="batch: graphs")
    ap.add_argument("--batch-steps", type=int, default=0,
                    help="batch: timed steps (0 = min(steps, 5))")
    ap.add_argument("--batch-warmup", type=int, default=3, help="batch: warm-up steps")
    ap.add_argument("--window", type=float, default=60.0, help="serve: arrival window (s)")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: requests per second")
    ap.add_argument("--serve-streams", type=int, default=4, help="serve: worker streams")
    ap.add_argument("--serve-queue", type=int, default=16,
                    help="serve: waiting requests before submit is refused")
    ap.add_argument("--serve-lead", type=float, default=1.0,
                    help="serve: seconds before its arrival a request is generated")
    args = ap.parse_args()
    if args.batch_steps <= 0:
        args.batch_steps = max(1, min(args.steps, 5))
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    return {"single": run_single, "batch": run_batch, "serve": run_serve, "top": run_top,
            "core": run_core, "budget": run_budget}[args.mode](args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
