"""ctypes binding of ``include/truss.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
computation of its own: buffers (torch tensors, on the GPU or the CPU, or numpy
arrays) are passed to the CUDA library by pointer.  The library must be built
(``__graft_entry__.build()`` or ``python -m paper_1205_6693_gb300._build``);
if it is missing this module raises instead of computing anything elsewhere.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

TRUSS_OK = 0
TRUSS_EINVAL = -1
TRUSS_ENOMEM = -2
TRUSS_ECUDA = -3
TRUSS_ETIMEOUT = -4
TRUSS_EAGAIN = -5
TRUSS_EBUSY = -6
TRUSS_ESHUTDOWN = -7
TRUSS_ECHECK = -8

ERRORS = {TRUSS_EINVAL: "EINVAL", TRUSS_ENOMEM: "ENOMEM", TRUSS_ECUDA: "ECUDA",
          TRUSS_ETIMEOUT: "ETIMEOUT", TRUSS_EAGAIN: "EAGAIN", TRUSS_EBUSY: "EBUSY",
          TRUSS_ESHUTDOWN: "ESHUTDOWN", TRUSS_ECHECK: "ECHECK"}


class TrussError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib().truss_strerror(code).decode() if _LIB is not None else str(code)
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({msg})")


class truss_opts(ctypes.Structure):
    _fields_ = [("wait_limit_ns", ctypes.c_int64), ("profile", ctypes.c_int32),
                ("count_bytes", ctypes.c_int32), ("support_stage_max", ctypes.c_int32),
                ("peel_variant", ctypes.c_int32), ("support_range_work", ctypes.c_int32),
                ("support_pair_cost", ctypes.c_int32), ("lists_by_walk", ctypes.c_int32),
                ("lists_in_place", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class truss_run_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("rows", ctypes.c_int64), ("m", ctypes.c_int64),
                ("triangles", ctypes.c_int64), ("kmax", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("subrounds", ctypes.c_int32),
                ("graphs", ctypes.c_int32), ("ms_build", ctypes.c_float),
                ("ms_support", ctypes.c_float), ("ms_lists", ctypes.c_float),
                ("ms_peel", ctypes.c_float), ("ms_scatter", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("bytes_support", ctypes.c_double),
                ("bytes_lists", ctypes.c_double), ("bytes_peel", ctypes.c_double),
                ("launches", ctypes.c_int64), ("candidates", ctypes.c_int64),
                ("rounds", ctypes.c_int32), ("lists_layout", ctypes.c_int32),
                ("peel_entries", ctypes.c_int64), ("peel_decrements", ctypes.c_int64),
                ("peel_scanned", ctypes.c_int64), ("design_bytes_support", ctypes.c_double),
                ("design_bytes_peel", ctypes.c_double), ("peel_sum_min_alive", ctypes.c_int64),
                ("peel_sum_min_alive_start", ctypes.c_int64),
                ("peel_alive_levels", ctypes.c_int64), ("peel_dead_entries", ctypes.c_int64),
                ("peel_dead_earlier", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("workspace_peak", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class truss_serve_opts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("batch_rows", ctypes.c_int64),
                ("max_batch", ctypes.c_int32), ("max_queue", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 6)]


class truss_req_stats(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("triangles", ctypes.c_int64), ("kmax", ctypes.c_int32),
                ("batched", ctypes.c_int32), ("queue_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class truss_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("edges", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("wall_s", ctypes.c_double), ("edges_per_s", ctypes.c_double),
                ("launches", ctypes.c_int64), ("retried", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_LIB = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32

# Symbols declared in include/truss.h (checked by the CPU test suite).
EXPORTS = ("truss_strerror", "truss_ctx_create", "truss_ctx_set_opts", "truss_ctx_destroy",
           "truss_support",
           "truss_decompose", "truss_decompose_batch", "truss_upper_bound", "truss_top",
           "truss_core", "truss_decompose_budget",
           "truss_last_stats",
           "truss_serve_footprint", "truss_serve_start", "truss_serve_submit", "truss_serve_poll",
           "truss_serve_wait", "truss_serve_stop", "truss_support_noalloc")


def library_path() -> str:
    return _build.LIB


def _lib():
    global _LIB
    if _LIB is None:
        if _build.stale():
            try:
                _build.build()
            except Exception as e:  # noqa: BLE001 - re-raised with context
                raise RuntimeError(f"libtruss.so is missing or stale and could not be built: {e}")
        L = ctypes.CDLL(_build.LIB)
        L.truss_strerror.restype = ctypes.c_char_p
        L.truss_strerror.argtypes = [ctypes.c_int]
        L.truss_ctx_create.restype = ctypes.c_int
        L.truss_ctx_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int,
                                       ctypes.POINTER(truss_opts)]
        L.truss_ctx_destroy.restype = ctypes.c_int
        L.truss_ctx_destroy.argtypes = [_vp]
        L.truss_ctx_set_opts.restype = ctypes.c_int
        L.truss_ctx_set_opts.argtypes = [_vp, ctypes.POINTER(truss_opts)]
        L.truss_support.restype = ctypes.c_int
        L.truss_support.argtypes = [_vp, _i64, _i64, _vp, _vp, _vp, _vp]
        L.truss_decompose.restype = ctypes.c_int
        L.truss_decompose.argtypes = [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp]
        L.truss_decompose_batch.restype = ctypes.c_int
        L.truss_decompose_batch.argtypes = [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.truss_upper_bound.restype = ctypes.c_int
        L.truss_upper_bound.argtypes = [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp]
        L.truss_decompose_budget.restype = ctypes.c_int
        L.truss_decompose_budget.argtypes = [_vp, _i64, _i64, _vp, _vp, _i64, _vp, _vp, _vp, _vp]
        L.truss_core.restype = ctypes.c_int
        L.truss_core.argtypes = [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp]
        L.truss_top.restype = ctypes.c_int
        L.truss_top.argtypes = [_vp, _i64, _i64, _vp, _vp, _i32, _vp, _vp, _vp]
        L.truss_last_stats.restype = ctypes.c_int
        L.truss_last_stats.argtypes = [_vp, ctypes.POINTER(truss_run_stats)]
        L.truss_serve_footprint.restype = ctypes.c_int64
        L.truss_serve_footprint.argtypes = [_i64, _i64]
        L.truss_serve_start.restype = ctypes.c_int
        L.truss_serve_start.argtypes = [_vp, ctypes.POINTER(truss_serve_opts), ctypes.POINTER(_vp)]
        L.truss_serve_submit.restype = ctypes.c_int
        L.truss_serve_submit.argtypes = [_vp, _i64, _i64, _vp, _vp, ctypes.POINTER(ctypes.c_uint64)]
        L.truss_serve_poll.restype = ctypes.c_int
        L.truss_serve_poll.argtypes = [_vp, ctypes.c_uint64, _vp, _vp,
                                       ctypes.POINTER(truss_req_stats)]
        L.truss_serve_wait.restype = ctypes.c_int
        L.truss_serve_wait.argtypes = [_vp, ctypes.c_uint64, _i64, _vp, _vp,
                                       ctypes.POINTER(truss_req_stats)]
        L.truss_support_noalloc.restype = ctypes.c_int
        L.truss_support_noalloc.argtypes = [_i64, _i64, _vp, _vp, _vp, _vp]
        L.truss_serve_stop.restype = ctypes.c_int
        L.truss_serve_stop.argtypes = [_vp, ctypes.POINTER(truss_serve_stats)]
        _LIB = L
    return _LIB


def load():
    """Load (building if needed) the CUDA library; returns the ctypes handle."""
    return _lib()


# ------------------------------------------------------------ marshalling ---
def _ptr(x, dtype=np.int32):
    """Device or host address of a torch tensor / numpy array (or None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or not x.flags.c_contiguous:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype).name} array")
        return x.ctypes.data
    # torch tensor
    import torch
    want = {np.int32: torch.int32, np.int64: torch.int64}[dtype]
    if x.dtype != want or not x.is_contiguous():
        raise TypeError(f"expected a contiguous {want} tensor")
    return x.data_ptr()


def _stream(stream, *tensors):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    for t in tensors:
        if t is not None and not isinstance(t, np.ndarray) and t.is_cuda:
            import torch
            return torch.cuda.current_stream(t.device).cuda_stream
    return None


def _check(rc, where):
    if rc != TRUSS_OK:
        raise TrussError(rc, where)


def _len(x):
    return int(x.shape[0])


def _rows(where, src, dst, *outs):
    """Row count of src, after checking that dst and every per-row output
    given (None = not given) have as many entries: a shorter buffer would be
    read or written past its end by the library."""
    rows = _len(src)
    for name, x in (("dst", dst),) + tuple((f"output {i}", o) for i, o in enumerate(outs)):
        if x is not None and _len(x) != rows:
            raise TypeError(f"{where}: {name} has {_len(x)} entries, src has {rows}")
    return rows


def _at_least(where, name, x, count):
    if x is not None and _len(x) < count:
        raise TypeError(f"{where}: {name} has {_len(x)} entries, {count} needed")


# ----------------------------------------------------------- entry points ---
def truss_strerror(code: int) -> str:
    return _lib().truss_strerror(code).decode()


def truss_ctx_create(device: int = 0, opts: truss_opts | None = None):
    ctx = _vp()
    _check(_lib().truss_ctx_create(ctypes.byref(ctx), device,
                                   ctypes.byref(opts) if opts is not None else None),
           "truss_ctx_create")
    return ctx


def truss_ctx_set_opts(ctx, opts: truss_opts) -> None:
    _check(_lib().truss_ctx_set_opts(ctx, ctypes.byref(opts)), "truss_ctx_set_opts")


def truss_ctx_destroy(ctx) -> None:
    _check(_lib().truss_ctx_destroy(ctx), "truss_ctx_destroy")


def truss_support(ctx, n: int, src, dst, support_out, stream=None) -> None:
    rows = _rows("truss_support", src, dst, support_out)
    _check(_lib().truss_support(ctx, n, rows, _ptr(src), _ptr(dst), _ptr(support_out),
                                _stream(stream, src, support_out)), "truss_support")


def truss_decompose(ctx, n: int, src, dst, support_out, truss_out, kmax_out=None,
                    stream=None) -> int:
    """Returns k_max (also written to kmax_out when given)."""
    rows = _rows("truss_decompose", src, dst, support_out, truss_out)
    _at_least("truss_decompose", "kmax_out", kmax_out, 1)
    k = np.zeros(1, np.int32)
    kp = _ptr(kmax_out) if kmax_out is not None else k.ctypes.data
    _check(_lib().truss_decompose(ctx, n, rows, _ptr(src), _ptr(dst), _ptr(support_out),
                                  _ptr(truss_out), kp, _stream(stream, src, truss_out)),
           "truss_decompose")
    return int(k[0]) if kmax_out is None else -1


def truss_upper_bound(ctx, n: int, src, dst, support_out, psi_out, stream=None) -> None:
    rows = _rows("truss_upper_bound", src, dst, support_out, psi_out)
    _check(_lib().truss_upper_bound(ctx, n, rows, _ptr(src), _ptr(dst), _ptr(support_out),
                                    _ptr(psi_out), _stream(stream, src, psi_out)),
           "truss_upper_bound")


def truss_top(ctx, n: int, src, dst, t: int, truss_out, kmax_out=None, stream=None) -> int:
    """Returns k_max (also written to kmax_out when given)."""
    rows = _rows("truss_top", src, dst, truss_out)
    _at_least("truss_top", "kmax_out", kmax_out, 1)
    k = np.zeros(1, np.int32)
    kp = _ptr(kmax_out) if kmax_out is not None else k.ctypes.data
    _check(_lib().truss_top(ctx, n, rows, _ptr(src), _ptr(dst), int(t), _ptr(truss_out), kp,
                            _stream(stream, src, truss_out)), "truss_top")
    return int(k[0]) if kmax_out is None else -1


def truss_decompose_budget(ctx, n: int, src, dst, budget_edges: int, support_out, truss_out,
                           kmax_out=None, stream=None) -> int:
    """Returns k_max (also written to kmax_out when given)."""
    rows = _rows("truss_decompose_budget", src, dst, support_out, truss_out)
    _at_least("truss_decompose_budget", "kmax_out", kmax_out, 1)
    k = np.zeros(1, np.int32)
    kp = _ptr(kmax_out) if kmax_out is not None else k.ctypes.data
    _check(_lib().truss_decompose_budget(ctx, n, rows, _ptr(src), _ptr(dst), int(budget_edges),
                                         _ptr(support_out), _ptr(truss_out), kp,
                                         _stream(stream, src, truss_out)),
           "truss_decompose_budget")
    return int(k[0]) if kmax_out is None else -1


def truss_core(ctx, n: int, src, dst, core_out, kmax_out=None, stream=None) -> int:
    """Core number per vertex into core_out (n entries); returns the largest."""
    rows = _rows("truss_core", src, dst)
    _at_least("truss_core", "core_out", core_out, n)
    _at_least("truss_core", "kmax_out", kmax_out, 1)
    k = np.zeros(1, np.int32)
    kp = _ptr(kmax_out) if kmax_out is not None else k.ctypes.data
    _check(_lib().truss_core(ctx, n, rows, _ptr(src), _ptr(dst), _ptr(core_out), kp,
                             _stream(stream, src, core_out)), "truss_core")
    return int(k[0]) if kmax_out is None else -1


def truss_decompose_batch(ctx, n, row_off, src, dst, support_out, truss_out, kmax_out=None,
                          stream=None) -> None:
    """n and row_off are host int64 arrays (G and G+1 entries)."""
    n = np.ascontiguousarray(n, np.int64)
    row_off = np.ascontiguousarray(row_off, np.int64)
    G = len(n)
    if len(row_off) != G + 1:
        raise TypeError(f"truss_decompose_batch: row_off has {len(row_off)} entries, {G + 1} needed")
    rows = _rows("truss_decompose_batch", src, dst, support_out, truss_out)
    if G > 0 and int(row_off[G]) != rows:
        raise TypeError(f"truss_decompose_batch: row_off[G] = {int(row_off[G])}, src has {rows} rows")
    _at_least("truss_decompose_batch", "kmax_out", kmax_out, G)
    _check(_lib().truss_decompose_batch(ctx, G, n.ctypes.data, row_off.ctypes.data, _ptr(src),
                                        _ptr(dst), _ptr(support_out), _ptr(truss_out),
                                        _ptr(kmax_out), _stream(stream, src, truss_out)),
           "truss_decompose_batch")


def truss_last_stats(ctx) -> dict:
    st = truss_run_stats()
    _check(_lib().truss_last_stats(ctx, ctypes.byref(st)), "truss_last_stats")
    return st.as_dict()


def truss_support_noalloc(n: int, src, dst, support_out, stream=None) -> None:
    """Allocation-free support for small graphs (device-accessible buffers;
    see include/truss.h for the size limits and the shared-scratch rules)."""
    rows = _rows("truss_support_noalloc", src, dst, support_out)
    args = (n, rows, _ptr(src), _ptr(dst), _ptr(support_out), _stream(stream, src, support_out))
    if not isinstance(src, np.ndarray) and src.is_cuda:
        import torch
        # the library launches on the current device: make it the tensors' one
        with torch.cuda.device(src.device):
            rc = _lib().truss_support_noalloc(*args)
    else:
        rc = _lib().truss_support_noalloc(*args)
    _check(rc, "truss_support_noalloc")


# ---------------------------------------------------------------- serving ---
def truss_serve_footprint(n: int, rows: int) -> int:
    return int(_lib().truss_serve_footprint(n, rows))


def truss_serve_start(ctx, opts: truss_serve_opts | None = None):
    srv = _vp()
    _check(_lib().truss_serve_start(ctx, ctypes.byref(opts) if opts is not None else None,
                                    ctypes.byref(srv)), "truss_serve_start")
    return srv


def truss_serve_submit(srv, n: int, src, dst) -> int:
    """Queue a request; src/dst must stay alive until it completes."""
    t = ctypes.c_uint64(0)
    rows = _rows("truss_serve_submit", src, dst)
    _check(_lib().truss_serve_submit(srv, n, rows, _ptr(src), _ptr(dst), ctypes.byref(t)),
           "truss_serve_submit")
    return int(t.value)


def truss_serve_poll(srv, ticket: int, support_out=None, truss_out=None):
    """Returns the request's stats dict if done, None if still running."""
    st = truss_req_stats()
    rc = _lib().truss_serve_poll(srv, ticket, _ptr(support_out), _ptr(truss_out),
                                 ctypes.byref(st))
    if rc == TRUSS_EAGAIN:
        return None
    _check(rc, "truss_serve_poll")
    return st.as_dict()


def truss_serve_wait(srv, ticket: int, timeout_ns: int = -1, support_out=None, truss_out=None):
    """Blocks until done (or timeout: returns None)."""
    st = truss_req_stats()
    rc = _lib().truss_serve_wait(srv, ticket, timeout_ns, _ptr(support_out), _ptr(truss_out),
                                 ctypes.byref(st))
    if rc == TRUSS_EAGAIN:
        return None
    _check(rc, "truss_serve_wait")
    return st.as_dict()


def truss_serve_stop(srv) -> dict:
    st = truss_serve_stats()
    _check(_lib().truss_serve_stop(srv, ctypes.byref(st)), "truss_serve_stop")
    return st.as_dict()


class Context:
    """Owns a truss_ctx; the methods are the entry points above."""

    def __init__(self, device: int = 0, profile: bool = False, count_bytes: bool = False,
                 wait_limit_ns: int = 0, **kw):
        o = truss_opts()
        o.profile = int(profile)
        o.count_bytes = int(count_bytes)
        o.wait_limit_ns = int(wait_limit_ns)
        for k, v in kw.items():
            setattr(o, k, v)
        self.ctx = truss_ctx_create(device, o)

    def set_opts(self, profile: bool = False, count_bytes: bool = False, wait_limit_ns: int = 0,
                 **kw):
        """Replace every option of the context (unnamed ones return to 0)."""
        o = truss_opts()
        o.profile = int(profile)
        o.count_bytes = int(count_bytes)
        o.wait_limit_ns = int(wait_limit_ns)
        for k, v in kw.items():
            setattr(o, k, v)
        truss_ctx_set_opts(self.ctx, o)

    def close(self):
        if self.ctx is not None:
            truss_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def support(self, n, src, dst, support_out, stream=None):
        return truss_support(self.ctx, n, src, dst, support_out, stream)

    def decompose(self, n, src, dst, support_out, truss_out, kmax_out=None, stream=None):
        return truss_decompose(self.ctx, n, src, dst, support_out, truss_out, kmax_out, stream)

    def upper_bound(self, n, src, dst, support_out, psi_out, stream=None):
        return truss_upper_bound(self.ctx, n, src, dst, support_out, psi_out, stream)

    def decompose_budget(self, n, src, dst, budget_edges, support_out, truss_out, kmax_out=None,
                         stream=None):
        return truss_decompose_budget(self.ctx, n, src, dst, budget_edges, support_out,
                                      truss_out, kmax_out, stream)

    def core(self, n, src, dst, core_out, kmax_out=None, stream=None):
        return truss_core(self.ctx, n, src, dst, core_out, kmax_out, stream)

    def top(self, n, src, dst, t, truss_out, kmax_out=None, stream=None):
        return truss_top(self.ctx, n, src, dst, t, truss_out, kmax_out, stream)

    def decompose_batch(self, n, row_off, src, dst, support_out, truss_out, kmax_out=None,
                        stream=None):
        return truss_decompose_batch(self.ctx, n, row_off, src, dst, support_out, truss_out,
                                     kmax_out, stream)

    def stats(self):
        return truss_last_stats(self.ctx)
