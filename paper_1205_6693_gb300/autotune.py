"""Schedule autotuner for the truss library.

The schedule fields of ``truss_opts`` (support walk range size, hub staging
threshold, per-edge range cost, peel kernel variant, list layout) change how the work is
laid out on the GPU, never what is computed: every schedule returns the same
supports and truss numbers.  This module picks them per GPU and per input
size bucket by timing candidates through the C ABI (the library's own CUDA
event stage times, ``truss_opts.profile``) and keeps the winners in a JSON
cache::

    {"<gpu key>": {"<bucket>": {"opts": {...}, "ms": {...}, "tuned_on": {...}}}}

The gpu key names the device model, compute capability and SM count; the
bucket is the kind of call ("single" or "batch") with the input's row count
rounded to a power of two (and, for a batch, the graph count likewise).

Search: coordinate descent in stage order.  Support knobs are judged on the
support + list stage time, the peel variant on the peel stage time; each
candidate runs ``reps`` times and keeps its minimum, and a candidate replaces
the incumbent only when it is faster by ``min_gain``.  Each candidate's
outputs are compared with the first run's; a difference raises, since it
would mean a schedule changed the result.
"""
from __future__ import annotations

import json
import math
import os
import tempfile
import threading
from typing import Callable

# Candidate values per knob, in search order.  0 is the library default.
SPACE: dict[str, tuple[int, ...]] = {
    "support_range_work": (0, 4096, 8192, 32768, 65536),
    "support_stage_max": (0, 64, 128, 256),
    "support_pair_cost": (0, 16, 32, 128, 256),
    "peel_variant": (0, 1, 3, 4),
    "lists_in_place": (0, 1),
}
# Stage-time keys of truss_last_stats each knob is judged on.
OBJECTIVE: dict[str, tuple[str, ...]] = {
    "support_range_work": ("ms_support", "ms_lists"),
    "support_stage_max": ("ms_support", "ms_lists"),
    "support_pair_cost": ("ms_support", "ms_lists"),
    "peel_variant": ("ms_lists", "ms_peel"),  # variant 4 also changes the list pass
    "lists_in_place": ("ms_lists", "ms_peel"),
}

_lock = threading.Lock()


# Schedules tuned on GB300 and shipped with the package: consulted when the
# user's cache has no entry for the call's bucket.
SHIPPED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "schedules_gb300.json")


def cache_path() -> str:
    p = os.environ.get("TRUSS_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "gb300_truss", "schedules.json")


def gpu_key(device: int = 0) -> str:
    import torch
    p = torch.cuda.get_device_properties(device)
    return f"{p.name}|sm_{p.major}{p.minor}|{p.multi_processor_count}SM"


def _log2_bucket(x: int) -> int:
    return 0 if x <= 1 else int(round(math.log2(x)))


def bucket(rows: int, graphs: int = 1) -> str:
    """Size bucket of a call: rows (and graphs, for a batch) to the nearest
    power of two."""
    if graphs > 1:
        return f"batch:r{_log2_bucket(rows)}:g{_log2_bucket(graphs)}"
    return f"single:r{_log2_bucket(rows)}"


def _parse(b: str):
    parts = b.split(":")
    kind = parts[0]
    r = int(parts[1][1:])
    g = int(parts[2][1:]) if len(parts) > 2 else 0
    return kind, r, g


def load(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save(cache: dict, path: str | None = None) -> None:
    """Write the cache atomically (temporary file + rename)."""
    path = path or cache_path()
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(path)), suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(key: str, rows: int, graphs: int = 1, cache: dict | None = None,
           nearest: bool = True):
    """Tuned opts for (gpu key, bucket): the exact bucket if cached, else (if
    ``nearest``) the nearest cached bucket of the same kind by log-size
    distance, else None."""
    cache = load() if cache is None else cache
    entries = cache.get(key, {})
    b = bucket(rows, graphs)
    if b in entries:
        return dict(entries[b]["opts"])
    if not nearest:
        return None
    kind, r, g = _parse(b)
    best, bd = None, None
    for name, ent in entries.items():
        try:
            k2, r2, g2 = _parse(name)
        except (ValueError, IndexError):
            continue
        if k2 != kind:
            continue
        dist = abs(r2 - r) + abs(g2 - g)
        if bd is None or dist < bd:
            best, bd = ent, dist
    return dict(best["opts"]) if best else None


def lookup_any(key: str, rows: int, graphs: int = 1):
    """(opts, source) for an exact bucket match: the user's cache first
    ("cache"), then the schedules shipped with the package ("shipped"); else
    (None, None)."""
    got = lookup(key, rows, graphs, nearest=False)
    if got is not None:
        return got, "cache"
    got = lookup(key, rows, graphs, cache=load(SHIPPED), nearest=False)
    if got is not None:
        return got, "shipped"
    return None, None


def search(run: Callable[[dict], tuple[dict, object]], reps: int = 2, min_gain: float = 0.03,
           space: dict | None = None, same: Callable[[object, object], bool] | None = None,
           log: Callable[[str], None] | None = None):
    """Coordinate descent over ``space``.  ``run(opts)`` performs one call with
    those schedule opts and returns (stage times, outputs).  Returns
    (best opts, their stage times, number of calls)."""
    space = SPACE if space is None else space
    calls = 0
    first_out = None

    def measure(opts):
        nonlocal calls, first_out
        best = None
        for _ in range(reps):
            st, out = run(dict(opts))
            calls += 1
            if first_out is None:
                first_out = out
            elif same is not None and not same(first_out, out):
                raise RuntimeError(f"schedule {opts} changed the result")
            if best is None:
                best = dict(st)
            else:
                for k, v in st.items():
                    if isinstance(v, (int, float)):
                        best[k] = min(best[k], v)
        return best

    cur = {k: 0 for k in space}
    cur_ms = measure(cur)
    for knob, values in space.items():
        obj = OBJECTIVE.get(knob, ("ms_total",))
        score = lambda st: sum(st.get(k, 0.0) for k in obj)  # noqa: E731
        base = score(cur_ms)
        for v in values:
            if v == cur[knob]:
                continue
            trial = dict(cur)
            trial[knob] = v
            st = measure(trial)
            if log:
                log(f"  {knob}={v}: {score(st):.3f} ms (incumbent {base:.3f})")
            if score(st) < base * (1.0 - min_gain):
                cur, cur_ms, base = trial, st, score(st)
    return cur, cur_ms, calls


def tune_call(device: int, call: Callable[[object], object], rows: int, graphs: int = 1,
              reps: int = 2, space: dict | None = None, write: bool = True,
              log: Callable[[str], None] | None = None) -> dict:
    """Tune the schedule of ``call(ctx)`` (one truss_decompose or
    truss_decompose_batch on the given context) and store the winner in the
    cache.  ``call`` returns the output tensors, which must be equal under
    every schedule.  All candidates run on one warm context
    (truss_ctx_set_opts), so no candidate pays for workspace allocation."""
    import torch

    from . import truss as T

    ctx = T.Context(device, profile=True)
    try:
        def run(opts):
            ctx.set_opts(profile=True, **opts)
            out = call(ctx)
            torch.cuda.synchronize(device)
            return ctx.stats(), tuple(o.clone() for o in out)

        def same(a, b):
            return all(torch.equal(x, y) for x, y in zip(a, b))

        run({})  # warm-up: module load, workspace growth
        opts, ms, calls = search(run, reps=reps, space=space, same=same, log=log)
    finally:
        ctx.close()
    entry = {"opts": opts,
             "ms": {k: round(v, 4) for k, v in ms.items() if k.startswith("ms_")},
             "tuned_on": {"rows": int(rows), "graphs": int(graphs), "calls": calls}}
    if write:
        key = gpu_key(device)
        with _lock:
            cache = load()
            cache.setdefault(key, {})[bucket(rows, graphs)] = entry
            save(cache)
    return entry
