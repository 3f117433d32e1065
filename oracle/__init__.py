"""CPU oracle for truss decomposition -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The GPU library never imports it and it never
imports the GPU library; the only thing the two sides share is the seeded
input generator package ``graphgen``.

* ``alg2.c``  -- Algorithm 2 of Wang & Cheng (Section 3.2) in plain C, single
  threaded, with step 2's supports from forward triangle listing.  Wrapped
  here by :func:`truss`; :func:`psi` is the upper bound of Procedure 6
  (Section 6.2) from its definition, and :func:`top` the top-t classes of
  Algorithm 7 (Section 6.3) read off the full decomposition; :func:`core`
  gives vertex core numbers by the bin-sorted degree array.
* ``checks.py`` -- independent checkers written from the definitions: edge
  subset brute force (Definition 2), the literal Algorithm 1 (Section 3.1),
  triple-enumeration support (Definition 1), core numbers, the upper bound
  psi of Procedure 6 (Section 6.2) and the truss invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "alg2.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile alg2.c with gcc into liboracle.so beside it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_truss.restype = ctypes.c_int
        L.oracle_truss.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _i32p, _i32p,
                                   _i32p, _i64p, _i64p]
        L.oracle_edges.restype = ctypes.c_int
        L.oracle_edges.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _i32p, _i32p,
                                   _i32p, _i64p]
        L.oracle_check_sample.restype = ctypes.c_int64
        L.oracle_check_sample.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _i32p,
                                          _i32p, ctypes.c_int64, _i64p, _i32p]
        L.oracle_psi.restype = ctypes.c_int
        L.oracle_psi.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _i32p, _i32p]
        L.oracle_core.restype = ctypes.c_int
        L.oracle_core.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _i32p, _i32p]
        L.oracle_check_valid.restype = ctypes.c_int64
        L.oracle_check_valid.argtypes = [ctypes.c_int64, ctypes.c_int64, _i32p, _i32p, _i32p,
                                         _i32p]
        _lib = L
    return _lib


def _c(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class OracleResult:
    __slots__ = ("support", "truss", "kmax", "m", "triangles")

    def __init__(self, support, truss, kmax, m, triangles):
        self.support, self.truss, self.kmax, self.m, self.triangles = (
            support, truss, kmax, m, triangles)


def truss(n: int, src, dst, with_truss: bool = True) -> OracleResult:
    """Per-row support and truss number of the simple graph the rows define
    (Algorithm 2).  Self-loop rows get -1; duplicate rows share values."""
    src, dst = _c(src), _c(dst)
    rows = len(src)
    sup = np.empty(max(rows, 1), np.int32)
    tr = np.empty(max(rows, 1), np.int32)
    kmax = ctypes.c_int32(0)
    m = ctypes.c_int64(0)
    tri = ctypes.c_int64(0)
    rc = _L().oracle_truss(n, rows, src.ctypes.data_as(_i32p), dst.ctypes.data_as(_i32p),
                           sup.ctypes.data_as(_i32p),
                           tr.ctypes.data_as(_i32p) if with_truss else None,
                           ctypes.byref(kmax), ctypes.byref(m), ctypes.byref(tri))
    if rc == -1:
        raise ValueError("vertex id out of range")
    if rc:
        raise MemoryError("oracle_truss")
    return OracleResult(sup[:rows], tr[:rows] if with_truss else None, kmax.value, m.value,
                        tri.value)


def psi(n: int, src, dst):
    """Per-row (support, psi) with psi(e) = min{sup(e), x_u, x_v} + 2 of
    Procedure 6 (Section 6.2), computed from the definition."""
    src, dst = _c(src), _c(dst)
    rows = len(src)
    sup = np.empty(max(rows, 1), np.int32)
    ps = np.empty(max(rows, 1), np.int32)
    rc = _L().oracle_psi(n, rows, src.ctypes.data_as(_i32p), dst.ctypes.data_as(_i32p),
                         sup.ctypes.data_as(_i32p), ps.ctypes.data_as(_i32p))
    if rc == -1:
        raise ValueError("vertex id out of range")
    if rc:
        raise MemoryError("oracle_psi")
    return sup[:rows], ps[:rows]


def top(n: int, src, dst, t: int):
    """The top-t k-classes by definition: per-row phi(e) where phi(e) >=
    k_max - t + 1, else 0 (self-loop rows -1), from the full decomposition
    (Algorithm 2).  Returns (per-row values, k_max)."""
    r = truss(n, src, dst)
    thr = max(r.kmax - t + 1, 2)
    out = np.where(r.truss >= thr, r.truss, 0).astype(np.int32)
    out[r.truss < 0] = -1
    return out, r.kmax


def core(n: int, src, dst):
    """Core number of every vertex id in [0, n) (0 for isolated vertices) and
    the largest, by the bin-sorted degree array (see alg2.c)."""
    src, dst = _c(src), _c(dst)
    out = np.zeros(max(n, 1), np.int32)
    k = ctypes.c_int32(0)
    rc = _L().oracle_core(n, len(src), src.ctypes.data_as(_i32p), dst.ctypes.data_as(_i32p),
                          out.ctypes.data_as(_i32p), ctypes.byref(k))
    if rc == -1:
        raise ValueError("vertex id out of range")
    if rc:
        raise MemoryError("oracle_core")
    return out[:n], k.value


def edges(n: int, src, dst):
    """Canonical edge list (eu < ev, lexicographic) and the row->edge map."""
    src, dst = _c(src), _c(dst)
    rows = len(src)
    eu = np.empty(max(rows, 1), np.int32)
    ev = np.empty(max(rows, 1), np.int32)
    r2e = np.empty(max(rows, 1), np.int32)
    m = ctypes.c_int64(0)
    rc = _L().oracle_edges(n, rows, src.ctypes.data_as(_i32p), dst.ctypes.data_as(_i32p),
                           eu.ctypes.data_as(_i32p), ev.ctypes.data_as(_i32p),
                           r2e.ctypes.data_as(_i32p), ctypes.byref(m))
    if rc:
        raise ValueError("oracle_edges failed")
    return eu[: m.value].copy(), ev[: m.value].copy(), r2e[:rows].copy()


def check_valid(n: int, src, dst, truss_rows, support_rows) -> int:
    """Number of edges violating validity (each edge of T_phi has >= phi-2
    triangles inside T_phi), 2 <= phi <= sup+2, or phi=2 <=> sup=0."""
    src, dst = _c(src), _c(dst)
    t, s = _c(truss_rows), _c(support_rows)
    return int(_L().oracle_check_valid(n, len(src), src.ctypes.data_as(_i32p),
                                       dst.ctypes.data_as(_i32p), t.ctypes.data_as(_i32p),
                                       s.ctypes.data_as(_i32p)))


def check_sample(n: int, src, dst, truss_rows, support_rows, sample_rows):
    """Per sampled row: exact support by neighbour-list intersection and local
    validity of the claimed truss number (see alg2.c).  Returns (violations,
    exact supports of the sampled rows)."""
    src, dst = _c(src), _c(dst)
    t, s = _c(truss_rows), _c(support_rows)
    smp = np.ascontiguousarray(sample_rows, dtype=np.int64)
    out = np.empty(max(len(smp), 1), np.int32)
    bad = _L().oracle_check_sample(n, len(src), src.ctypes.data_as(_i32p),
                                   dst.ctypes.data_as(_i32p), t.ctypes.data_as(_i32p),
                                   s.ctypes.data_as(_i32p), len(smp),
                                   smp.ctypes.data_as(_i64p), out.ctypes.data_as(_i32p))
    if bad < 0:
        raise ValueError("oracle_check_sample failed")
    return int(bad), out[:len(smp)]
