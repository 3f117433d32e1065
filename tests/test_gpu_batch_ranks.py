"""The batch form sharded over two ranks (gloo, both on cuda:0): every graph
of each rank's shard matches the oracle, the shards cover the batch exactly
once, and bench.py's batch mode runs its sharded path to a JSON line."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, env=None, timeout=600):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_port()}", *args]
    e = dict(os.environ, **(env or {}))
    return subprocess.run(cmd, capture_output=True, text=True, timeout=timeout, cwd=ROOT, env=e)


def test_two_ranks_on_one_gpu_decompose_their_shards_exactly(tmp_path):
    graphs = 64
    out = str(tmp_path / "parts.npy")
    r = _torchrun([os.path.join(ROOT, "tests", "batch_rank_worker.py"), str(graphs), out])
    assert r.returncode == 0, r.stderr[-3000:]
    parts = np.load(out, allow_pickle=True)
    covered = []
    for g0, g1, off, sup, tr, kmax in parts:
        covered.extend(range(g0, g1))
        for i, g in enumerate(range(g0, g1)):
            n, s, d = graphgen.batch_graph(g)
            ref = oracle.truss(n, s, d)
            a, b = int(off[i]), int(off[i + 1])
            assert np.array_equal(sup[a:b], ref.support), g
            assert np.array_equal(tr[a:b], ref.truss), g
            assert int(kmax[i]) == ref.kmax, g
    assert covered == list(range(graphs))
    assert all(g1 > g0 for g0, g1, *_ in parts)


def test_bench_batch_mode_runs_sharded_over_two_ranks():
    r = _torchrun([os.path.join(ROOT, "bench.py"), "--mode", "batch", "--graphs", "64",
                   "--gpus", "2", "--steps", "1", "--warmup", "1", "--batch-warmup", "1",
                   "--no-tune"],
                  env={"TRUSS_BENCH_BACKEND": "gloo", "TRUSS_BENCH_DEVICE": "0"})
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1  # rank 0 alone prints
    line = json.loads(lines[0])
    assert line["n_gpus"] == 2 and line["value"] > 0
    assert line["config"]["parallelism"] == "graphs sharded over 2 rank(s)"
    assert line["per_graph_loop"]["steps"] == line["steps"] == 1
