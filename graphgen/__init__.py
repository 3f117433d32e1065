"""Seeded synthetic graph inputs shared by the oracle side and the GPU side.

This package only generates edge lists (int32 ``src``/``dst`` rows over
vertex ids ``[0, n)``).  It contains none of the truss-decomposition
arithmetic and imports neither the oracle nor the CUDA library.  The C source
``gen.c`` is compiled on first use with gcc into ``libgraphgen.so`` beside it.

Workloads (each fully defined by its seed, sizes and sampling rule below):

* ``tiny()``  - Erdos-Renyi n=4,096, m=32,768 distinct pairs (seed 0) plus six
  planted cliques of sizes 8, 12, 16, 20, 24, 32 on disjoint vertex sets.
* ``mid()``   - R-MAT scale 20, 16 * 2^20 raw samples, (a,b,c,d) =
  (.57,.19,.19,.05), seed 1; duplicates and self-loops kept in the rows.
* ``large()`` - Chung-Lu, n = 2^24, expected-degree exponent 2.1, mean 20, cap
  2^16, seed 2; the first 167,772,160 distinct pairs.
* ``batch_graph(g)`` / ``batch(G)`` - the 4,096-graph mixed batch.
* ``serve_schedule(...)`` - Poisson arrivals and log-uniform request sizes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None
_CU_SRC = os.path.join(_HERE, "gen_cuda.cu")
_CU_LIB = os.path.join(_HERE, "libgraphgen_cuda.so")
_culib = None

RMAT_ABCD = (Fraction(57, 100), Fraction(19, 100), Fraction(19, 100), Fraction(5, 100))
TINY_CLIQUES = (8, 12, 16, 20, 24, 32)
BATCH_BASE_SEED = 0xB47C

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile gen.c into libgraphgen.so (no fused multiply-add, for
    bit-identical results across x86-64 and aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fno-fast-math",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def build_cuda(force: bool = False) -> str:
    """Compile gen_cuda.cu (GPU form of the R-MAT generator) for sm_103a."""
    if force or not os.path.exists(_CU_LIB) or os.path.getmtime(_CU_LIB) < os.path.getmtime(_CU_SRC):
        tmp = _CU_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["nvcc", "-O3", "-std=c++17", "-gencode",
                               "arch=compute_103a,code=sm_103a", "-Xcompiler", "-fPIC", "-shared",
                               "-o", tmp, _CU_SRC])
        os.replace(tmp, _CU_LIB)
    return _CU_LIB


def culib():
    global _culib
    if _culib is None:
        build_cuda()
        L = ctypes.CDLL(_CU_LIB)
        L.gg_rmat_raw_cuda.restype = ctypes.c_int
        L.gg_rmat_raw_cuda.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]
        _culib = L
    return _culib


def rmat_raw_cuda(scale: int, nsamples: int, seed: int, stream: int = 0, device=None,
                  cuda_stream=None):
    """As rmat_raw, generated on the GPU into new torch int32 tensors."""
    import torch
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    src = torch.empty(nsamples, dtype=torch.int32, device=dev)
    dst = torch.empty(nsamples, dtype=torch.int32, device=dev)
    t1, t2, t3 = rmat_thresholds()
    cs = cuda_stream if cuda_stream is not None else torch.cuda.current_stream(dev).cuda_stream
    if culib().gg_rmat_raw_cuda(scale, nsamples, t1, t2, t3, seed, stream, src.data_ptr(),
                                dst.data_ptr(), cs):
        raise RuntimeError("gg_rmat_raw_cuda failed")
    return src, dst


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.gg_draw.restype = ctypes.c_uint64
        L.gg_draw.argtypes = [ctypes.c_uint64] * 3
        L.gg_splitmix64.restype = ctypes.c_uint64
        L.gg_splitmix64.argtypes = [ctypes.c_uint64]
        L.gg_log_public.restype = ctypes.c_double
        L.gg_log_public.argtypes = [ctypes.c_double]
        L.gg_exp_public.restype = ctypes.c_double
        L.gg_exp_public.argtypes = [ctypes.c_double]
        L.gg_er.restype = ctypes.c_int64
        L.gg_er.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                            _i32p, _i32p, ctypes.c_int64]
        L.gg_rmat_raw.restype = None
        L.gg_rmat_raw.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, _i32p, _i32p]
        L.gg_rmat_distinct.restype = ctypes.c_int64
        L.gg_rmat_distinct.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_uint64, _i32p, _i32p, ctypes.c_int64]
        L.gg_permutation.restype = None
        L.gg_permutation.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, _i32p]
        L.gg_add_cliques.restype = ctypes.c_int64
        L.gg_add_cliques.argtypes = [ctypes.c_int64, _i32p, _i32p, _i32p, ctypes.c_int, _i32p]
        L.gg_chung_lu_weights.restype = ctypes.c_double
        L.gg_chung_lu_weights.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, _f64p]
        L.gg_alias_build.restype = ctypes.c_int
        L.gg_alias_build.argtypes = [ctypes.c_int64, _f64p, _u64p, _i32p]
        L.gg_chung_lu.restype = ctypes.c_int64
        L.gg_chung_lu.argtypes = [ctypes.c_int64, ctypes.c_int64, _u64p, _i32p, ctypes.c_uint64,
                                  ctypes.c_uint64, _i32p, _i32p, ctypes.c_int64]
        L.gg_chung_lu_sorted.restype = ctypes.c_int64
        L.gg_chung_lu_sorted.argtypes = [ctypes.c_int64, ctypes.c_int64, _u64p, _i32p,
                                         ctypes.c_uint64, ctypes.c_uint64, _i32p, _i32p]
        L.gg_batch_spec.restype = None
        L.gg_batch_spec.argtypes = [ctypes.c_int64, ctypes.c_uint64, _i32p, _i64p, _i64p, _u64p,
                                    _i32p]
        L.gg_serve_schedule.restype = None
        L.gg_serve_schedule.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_uint64, _f64p, _i64p]
        _lib = L
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def rmat_thresholds(abcd=RMAT_ABCD):
    """32-bit cumulative quadrant thresholds (a, a+b, a+b+c) * 2^32, rounded."""
    a, b, c, _ = abcd
    return (round(a * 2 ** 32), round((a + b) * 2 ** 32), round((a + b + c) * 2 ** 32))


def draw(seed: int, stream: int, ctr: int) -> int:
    return int(lib().gg_draw(seed, stream, ctr))


def er(n: int, m: int, seed: int, stream: int = 0, max_draws: int | None = None):
    """G(n, m): first m distinct non-loop pairs; returns (src, dst) int32."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    md = max_draws if max_draws is not None else 64 * m + 1024
    k = lib().gg_er(n, m, seed, stream, _p(src, _i32p), _p(dst, _i32p), md)
    if k < 0:
        raise MemoryError("gg_er")
    return src[:k].copy(), dst[:k].copy()


def rmat_raw(scale: int, nsamples: int, seed: int, stream: int = 0):
    t1, t2, t3 = rmat_thresholds()
    src = np.empty(nsamples, np.int32)
    dst = np.empty(nsamples, np.int32)
    lib().gg_rmat_raw(scale, nsamples, t1, t2, t3, seed, stream, _p(src, _i32p), _p(dst, _i32p))
    return src, dst


def rmat_distinct(scale: int, m: int, seed: int, stream: int = 0, max_draws: int | None = None):
    t1, t2, t3 = rmat_thresholds()
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    md = max_draws if max_draws is not None else 64 * m + 4096
    k = lib().gg_rmat_distinct(scale, m, t1, t2, t3, seed, stream, _p(src, _i32p),
                               _p(dst, _i32p), md)
    if k < 0:
        raise MemoryError("gg_rmat_distinct")
    return src[:k].copy(), dst[:k].copy()


def permutation(n: int, seed: int, stream: int) -> np.ndarray:
    out = np.empty(n, np.int32)
    lib().gg_permutation(n, seed, stream, _p(out, _i32p))
    return out


def add_cliques(src: np.ndarray, dst: np.ndarray, verts: np.ndarray, sizes):
    """Append clique edges on consecutive slices of ``verts``, skipping pairs
    already present.  Returns new (src, dst)."""
    sizes = np.asarray(sizes, np.int32)
    extra = int(sum(int(s) * (int(s) - 1) // 2 for s in sizes))
    m0 = len(src)
    s2 = np.empty(m0 + extra, np.int32)
    d2 = np.empty(m0 + extra, np.int32)
    s2[:m0] = src
    d2[:m0] = dst
    verts = np.ascontiguousarray(verts, np.int32)
    k = lib().gg_add_cliques(m0, _p(s2, _i32p), _p(d2, _i32p), _p(verts, _i32p), len(sizes),
                             _p(sizes, _i32p))
    if k < 0:
        raise MemoryError("gg_add_cliques")
    return s2[:k].copy(), d2[:k].copy()


def tiny():
    """ER n=4,096, m=32,768 (seed 0) plus cliques 8,12,16,20,24,32 placed on the
    first 112 entries of a seeded permutation.  Returns (n, src, dst)."""
    n = 4096
    src, dst = er(n, 32768, seed=0, stream=0)
    perm = permutation(n, seed=0, stream=1)
    src, dst = add_cliques(src, dst, perm[: sum(TINY_CLIQUES)], TINY_CLIQUES)
    return n, src, dst


def mid(nsamples: int = 16 * 2 ** 20):
    """R-MAT scale 20, edge factor 16: raw samples (duplicates, self-loops kept)."""
    src, dst = rmat_raw(20, nsamples, seed=1, stream=0)
    return 2 ** 20, src, dst


def chung_lu(n: int, m: int, mean: float, cap: float, gamma: float, seed: int, stream: int = 0,
             max_draws: int | None = None, sorted_dedup: bool = False):
    L = lib()
    w = np.empty(n, np.float64)
    L.gg_chung_lu_weights(n, mean, cap, gamma, _p(w, _f64p))
    thr = np.empty(n, np.uint64)
    alias = np.empty(n, np.int32)
    if L.gg_alias_build(n, _p(w, _f64p), _p(thr, _u64p), _p(alias, _i32p)):
        raise MemoryError("gg_alias_build")
    del w
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    md = max_draws if max_draws is not None else 4 * m + 4096
    if sorted_dedup:
        # same rows as the hash-set path (first m distinct pairs in sample
        # order), found by sorting: much faster for very large m
        k = L.gg_chung_lu_sorted(n, m, _p(thr, _u64p), _p(alias, _i32p), seed, stream,
                                 _p(src, _i32p), _p(dst, _i32p))
    else:
        k = L.gg_chung_lu(n, m, _p(thr, _u64p), _p(alias, _i32p), seed, stream, _p(src, _i32p),
                          _p(dst, _i32p), md)
    if k < 0:
        raise MemoryError("gg_chung_lu")
    if k < m:
        return src[:k].copy(), dst[:k].copy()
    return src, dst


def chung_lu_weights(n: int, mean: float, cap: float, gamma: float):
    w = np.empty(n, np.float64)
    c = lib().gg_chung_lu_weights(n, mean, cap, gamma, _p(w, _f64p))
    return c, w


def large(n: int = 2 ** 24, mean_deg: int = 20, cap: float = 2.0 ** 16, rows: int | None = None):
    """Chung-Lu, exponent 2.1, first n*mean/2 distinct pairs (seed 2).  With
    ``rows``, only the first ``rows`` of those rows (the rows are the distinct
    pairs in sample order, so a prefix needs only a shorter sampling run)."""
    m = n * mean_deg // 2
    if rows is not None:
        m = min(m, int(rows))
    src, dst = chung_lu(n, m, float(mean_deg), cap, 2.1, seed=2, sorted_dedup=True)
    return n, src, dst


def batch_spec(g: int, base: int = BATCH_BASE_SEED):
    t = ctypes.c_int32()
    n = ctypes.c_int64()
    m = ctypes.c_int64()
    sd = ctypes.c_uint64()
    cl = ctypes.c_int32()
    lib().gg_batch_spec(g, base, ctypes.byref(t), ctypes.byref(n), ctypes.byref(m),
                        ctypes.byref(sd), ctypes.byref(cl))
    return dict(type=t.value, n=n.value, m=m.value, seed=sd.value, clique=cl.value)


def batch_graph(g: int, base: int = BATCH_BASE_SEED):
    """Graph g of the mixed batch.  Returns (n, src, dst)."""
    sp = batch_spec(g, base)
    n, m, sd = sp["n"], sp["m"], sp["seed"]
    if sp["type"] == 1:
        scale = n.bit_length() - 1
        src, dst = rmat_distinct(scale, m, sd, 0)
    else:
        src, dst = er(n, min(m, n * (n - 1) // 2), sd, 0)
        if sp["type"] == 2:
            perm = permutation(n, sd, 1)
            src, dst = add_cliques(src, dst, perm[: sp["clique"]], [sp["clique"]])
    return n, src, dst


def batch(G: int = 4096, base: int = BATCH_BASE_SEED, first: int = 0):
    """Pack graphs first..first+G-1: returns (n[G] int64, row_off[G+1] int64,
    src, dst) with per-graph local ids."""
    ns = np.empty(G, np.int64)
    off = np.zeros(G + 1, np.int64)
    parts_s, parts_d = [], []
    for i in range(G):
        n, s, d = batch_graph(first + i, base)
        ns[i] = n
        off[i + 1] = off[i] + len(s)
        parts_s.append(s)
        parts_d.append(d)
    src = np.concatenate(parts_s) if parts_s else np.empty(0, np.int32)
    dst = np.concatenate(parts_d) if parts_d else np.empty(0, np.int32)
    return ns, off, src, dst


def serve_schedule(count: int, rate: float = 200.0, mlo: float = 1e3, mhi: float = 5e7,
                   seed: int = 3):
    """Arrival times (s) and edge targets of a Poisson request stream."""
    t = np.empty(count, np.float64)
    m = np.empty(count, np.int64)
    lib().gg_serve_schedule(count, rate, mlo, mhi, seed, _p(t, _f64p), _p(m, _i64p))
    return t, m


def serve_scale(m: int) -> int:
    """R-MAT scale of a served request with target m: ceil(log2(m/8)), >= 4."""
    scale = 4
    while (1 << scale) < (m + 7) // 8:
        scale += 1
    return scale


def serve_request(j: int, m: int, seed: int = 3):
    """R-MAT request j: scale ceil(log2(m/8)) (at least 4), first m distinct pairs."""
    scale = 4
    while (1 << scale) < (m + 7) // 8:
        scale += 1
    src, dst = rmat_distinct(scale, m, gg_seed(seed, j), 0)
    return 1 << scale, src, dst


def gg_seed(seed: int, j: int) -> int:
    return int(lib().gg_splitmix64((seed * 0x100000001) ^ j))
