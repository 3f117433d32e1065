"""Write tests/golden/digests.json: expected outputs of the full-size workloads.

Every value written here comes from the CPU oracle (oracle/, Algorithm 2) run
on the seeded inputs of graphgen; nothing is taken from the GPU library.  The
full-size runs take minutes (mid) to hours (large) single-threaded, so the GPU
parity tests compare against these stored results:

* SHA-256 of the per-row support and truss arrays (int32, little endian),
* m, triangle count, k_max and the size of every k-class,
* the support and truss of 4,096 sampled rows (seeded), for diagnostics.

Usage: python tests/golden/make_digests.py mid [large ...]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(HERE, "digests.json")
CONFIGS = {"tiny": graphgen.tiny, "mid": graphgen.mid, "large": graphgen.large}
SAMPLE = 4096


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


def sample_rows(rows: int, k: int = SAMPLE) -> np.ndarray:
    perm = graphgen.permutation(rows, seed=12345, stream=9) if rows <= 50_000_000 else None
    if perm is None:
        idx = np.array([graphgen.draw(12345, 9, i) % rows for i in range(k)], np.int64)
        return np.unique(idx)
    return np.sort(perm[: min(k, rows)]).astype(np.int64)


def run(name: str) -> dict:
    t0 = time.time()
    n, src, dst = CONFIGS[name]()
    t1 = time.time()
    r = oracle.truss(n, src, dst)
    t2 = time.time()
    _, _, r2e = oracle.edges(n, src, dst)
    phi_e = np.zeros(r.m, np.int32)
    ok = r2e >= 0
    phi_e[r2e[ok]] = r.truss[ok]
    classes = np.bincount(phi_e, minlength=3)
    idx = sample_rows(len(src))
    return {
        "n": int(n), "rows": int(len(src)), "m": int(r.m), "triangles": int(r.triangles),
        "kmax": int(r.kmax), "sha256_support": sha(r.support), "sha256_truss": sha(r.truss),
        "classes": {str(k): int(c) for k, c in enumerate(classes) if c > 0},
        "sample_rows": idx.tolist(), "sample_support": r.support[idx].tolist(),
        "sample_truss": r.truss[idx].tolist(),
        "oracle_seconds": round(t2 - t1, 1), "generate_seconds": round(t1 - t0, 1),
    }


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names:
        print(f"[digest] {name} ...", flush=True)
        data[name] = run(name)
        print(f"[digest] {name}: m={data[name]['m']} kmax={data[name]['kmax']} "
              f"oracle {data[name]['oracle_seconds']} s", flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["tiny", "mid"])
