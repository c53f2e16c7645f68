"""Thin Python binding of libsbp (the C ABI declared in include/sbp.h).

Argument marshalling only: every step of the SBP path runs in the CUDA
library.  Functions keep the C names (``sbp_load_graph``,
``sbp_build_blockmodel``, ``sbp_nodal_sweep``, ``sbp_merge_blocks``,
``sbp_partition``, ...) and take numpy arrays (host memory) or torch CUDA
tensors (device memory) where the C call takes a pointer.  PyTorch is used
for device memory and streams only.

The library must be built (``paper_2305_18663_gb300.build.build()``); there
is no fallback path: a missing or unloadable library raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from .build import LIB, build as _build

__all__ = [
    "SbpError", "Params", "SweepStats", "Trace", "load", "lib", "sbp_default_params", "sbp_last_error",
    "sbp_load_graph", "sbp_free_graph", "sbp_graph_info", "sbp_build_blockmodel", "sbp_set_assignment",
    "sbp_nodal_sweep", "sbp_nodal_decide", "sbp_commit", "sbp_merge_proposals", "sbp_merge_blocks",
    "sbp_compact", "sbp_partition", "sbp_get_assignment", "sbp_get_pending", "sbp_set_pending", "sbp_get_B", "sbp_get_dl",
    "sbp_get_blockmodel_dense", "sbp_get_degrees", "sbp_get_blockmodel_coo", "sbp_sync", "sbp_free_model", "sbp_philox_check",
    "sbp_dense_dl_noalloc", "sbp_kernel_launches", "sbp_dxlogx32_check", "sbp_bracket_check",
    "sbp_default_batch_options", "sbp_partition_batch",
    "BatchOptions", "BatchResult", "BatchStats", "partition_batch", "Server", "sbp_autotune_batch", "autotune_batch",
    "sbp_server_create", "sbp_server_submit", "sbp_server_poll", "sbp_server_wait", "sbp_server_stats",
    "sbp_server_destroy",
    "Graph", "Model", "deal_vertices",
]

ERRORS = {-1: "SBP_EINVAL", -2: "SBP_ENOMEM", -3: "SBP_EHASHFULL", -4: "SBP_EPROBE", -5: "SBP_ECUDA", -6: "SBP_ESTATE"}


class SbpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64),
        ("beta", C.c_double),
        ("merge_proposals", C.c_int32),
        ("max_sweeps", C.c_int32),
        ("reduction", C.c_double),
        ("t_pre", C.c_double),
        ("t_post", C.c_double),
        ("dense_max_B", C.c_int32),
        ("full_rebuild", C.c_int32),
        ("dl_fp32", C.c_int32),
        ("hybrid_h", C.c_int32),
        ("reserved", C.c_int32),
    ]

    @classmethod
    def default(cls, **kw) -> "Params":
        p = cls()
        lib().sbp_default_params(C.byref(p))
        for k, v in kw.items():
            setattr(p, k, v)
        return p


class SweepStats(C.Structure):
    _fields_ = [
        ("n_proposed", C.c_int64),
        ("n_moves", C.c_int64),
        ("n_accepted", C.c_int64),
        ("n_margin", C.c_int64),
        ("n_move_edges", C.c_int64),
        ("dl_before", C.c_double),
        ("dl_after", C.c_double),
        ("n_recheck", C.c_int64),
        ("n_entries", C.c_int64),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchOptions(C.Structure):
    _fields_ = [
        ("workers", C.c_int32),
        ("max_B", C.c_int32),
        ("dense_max_B", C.c_int32),
        ("ctas_per_sm", C.c_int32),
        ("max_n", C.c_int32),
        ("movers_per_warp", C.c_int32),
        ("mem_fraction", C.c_double),
    ]

    @classmethod
    def default(cls, **kw) -> "BatchOptions":
        o = cls()
        _check(lib().sbp_default_batch_options(C.byref(o)))
        for k, v in kw.items():
            setattr(o, k, v)
        return o


class BatchResult(C.Structure):
    _fields_ = [
        ("B", C.c_int32),
        ("reserved", C.c_int32),
        ("dl", C.c_double),
        ("n_sweeps", C.c_int64),
        ("t_submit", C.c_double),
        ("t_admit", C.c_double),
        ("t_done", C.c_double),
    ]


class BatchStats(C.Structure):
    _fields_ = [
        ("rounds", C.c_int64),
        ("s_per_graph", C.c_double),
        ("s_batched", C.c_double),
        ("phases_batched", C.c_int64),
        ("phases_per_graph", C.c_int64),
        ("s_merge", C.c_double),
        ("s_sweeps", C.c_double),
        ("merges_batched", C.c_int64),
        ("starts_batched", C.c_int64),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Trace(C.Structure):
    _fields_ = [("s", C.c_void_p), ("flags", C.c_void_p), ("dH", C.c_void_p), ("logA", C.c_void_p)]


_lib = None


def load(path: str | None = None):
    """Load libsbp.so (build it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if path == LIB:
        _build()
    if not os.path.exists(path):
        raise RuntimeError(f"libsbp not found at {path}")
    L = C.CDLL(path)
    vp, i32, i64, u64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    P = C.POINTER
    sig = {
        "sbp_last_error": (C.c_size_t, [C.c_char_p, C.c_size_t]),
        "sbp_default_params": (C.c_int, [P(Params)]),
        "sbp_load_graph": (C.c_int, [i64, i64, vp, vp, P(vp)]),
        "sbp_graph_info": (C.c_int, [vp, P(i64), P(i64)]),
        "sbp_free_graph": (None, [vp]),
        "sbp_build_blockmodel": (C.c_int, [vp, i32, vp, P(Params), vp, P(vp)]),
        "sbp_set_assignment": (C.c_int, [vp, i32, vp]),
        "sbp_nodal_sweep": (C.c_int, [vp, u64, i64, i64, P(SweepStats)]),
        "sbp_nodal_decide": (C.c_int, [vp, u64, i64, i64, P(Trace)]),
        "sbp_commit": (C.c_int, [vp, P(SweepStats)]),
        "sbp_merge_proposals": (C.c_int, [vp, u64, vp, vp]),
        "sbp_merge_blocks": (C.c_int, [vp, u64, i32, P(i32), P(i32)]),
        "sbp_compact": (C.c_int, [vp, P(i32)]),
        "sbp_partition": (C.c_int, [vp, P(Params), vp, vp, P(i32), P(f64), P(i64)]),
        "sbp_get_assignment": (C.c_int, [vp, vp]),
        "sbp_get_pending": (C.c_int, [vp, i64, i64, vp]),
        "sbp_set_pending": (C.c_int, [vp, i64, i64, vp]),
        "sbp_get_B": (C.c_int, [vp, P(i32)]),
        "sbp_get_dl": (C.c_int, [vp, vp]),
        "sbp_get_blockmodel_dense": (C.c_int, [vp, vp]),
        "sbp_get_degrees": (C.c_int, [vp, vp, vp]),
        "sbp_get_blockmodel_coo": (C.c_int, [vp, i64, vp, vp, P(i64)]),
        "sbp_sync": (C.c_int, [vp]),
        "sbp_free_model": (None, [vp]),
        "sbp_philox_check": (C.c_int, [u64, u64, u64, u64, u64, u64, i32, vp]),
        "sbp_dense_dl_noalloc": (C.c_int, [vp, i32, vp, vp, i64, i64, vp, vp]),
        "sbp_kernel_launches": (C.c_int, [P(u64)]),
        "sbp_bracket_check": (C.c_int, [vp, vp, i32, C.c_double, vp, P(i32)]),
        "sbp_default_batch_options": (C.c_int, [P(BatchOptions)]),
        "sbp_dxlogx32_check": (C.c_int, [vp, vp, i32, vp, vp]),
        "sbp_partition_batch": (C.c_int, [vp, i32, P(Params), P(BatchOptions), vp, P(BatchResult), P(BatchStats)]),
        "sbp_autotune_batch": (C.c_int, [vp, i32, P(Params), i32, i32, P(BatchOptions), P(f64), P(i32)]),
        "sbp_server_create": (C.c_int, [P(Params), P(BatchOptions), P(vp)]),
        "sbp_server_submit": (C.c_int, [vp, vp, vp, P(i64)]),
        "sbp_server_poll": (C.c_int, [vp, i64, P(i32)]),
        "sbp_server_wait": (C.c_int, [vp, i64, P(BatchResult)]),
        "sbp_server_stats": (C.c_int, [vp, P(BatchStats)]),
        "sbp_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def lib():
    return load()


def _check(rc: int) -> None:
    if rc != 0:
        buf = C.create_string_buffer(1024)
        lib().sbp_last_error(buf, 1024)
        raise SbpError(rc, buf.value.decode(errors="replace"))


def _ptr(x, dtype) -> int | None:
    """Pointer of a numpy array (host) or a torch tensor (host or device)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a contiguous {np.dtype(dtype)} array")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        import torch

        want = {np.int32: torch.int32, np.float64: torch.float64, np.int64: torch.int64, np.uint64: torch.uint64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


# ---------------------------------------------------------------------------
# functions with the C names

def sbp_default_params() -> Params:
    return Params.default()


def sbp_last_error() -> str:
    buf = C.create_string_buffer(1024)
    lib().sbp_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def sbp_load_graph(n: int, src, dst) -> int:
    m = int(src.shape[0])
    if int(dst.shape[0]) != m:
        raise ValueError("src and dst differ in length")
    h = C.c_void_p()
    _check(lib().sbp_load_graph(n, m, _ptr(src, np.int32), _ptr(dst, np.int32), C.byref(h)))
    return h.value


def sbp_graph_info(g: int) -> tuple[int, int]:
    n, m = C.c_int64(), C.c_int64()
    _check(lib().sbp_graph_info(g, C.byref(n), C.byref(m)))
    return n.value, m.value


def sbp_free_graph(g: int) -> None:
    lib().sbp_free_graph(g)


def sbp_build_blockmodel(g: int, B: int, b, params: Params | None = None, stream=None) -> int:
    h = C.c_void_p()
    _check(lib().sbp_build_blockmodel(g, B, _ptr(b, np.int32), C.byref(params) if params else None, _stream_ptr(stream), C.byref(h)))
    return h.value


def sbp_set_assignment(m: int, B: int, b) -> None:
    _check(lib().sbp_set_assignment(m, B, _ptr(b, np.int32)))


def sbp_nodal_sweep(m: int, sweep_id: int, v_begin: int, v_end: int, stats: bool = True) -> SweepStats | None:
    st = SweepStats() if stats else None
    _check(lib().sbp_nodal_sweep(m, sweep_id, v_begin, v_end, C.byref(st) if st is not None else None))
    return st


def sbp_nodal_decide(m: int, sweep_id: int, v_begin: int, v_end: int, s=None, flags=None, dH=None, logA=None) -> None:
    tr = Trace(_ptr(s, np.int32), _ptr(flags, np.int32), _ptr(dH, np.float64), _ptr(logA, np.float64))
    any_tr = any(x is not None for x in (s, flags, dH, logA))
    _check(lib().sbp_nodal_decide(m, sweep_id, v_begin, v_end, C.byref(tr) if any_tr else None))


def sbp_commit(m: int, stats: bool = True) -> SweepStats | None:
    st = SweepStats() if stats else None
    _check(lib().sbp_commit(m, C.byref(st) if st is not None else None))
    return st


def sbp_merge_proposals(m: int, round_id: int, best_s, best_dDL) -> None:
    _check(lib().sbp_merge_proposals(m, round_id, _ptr(best_s, np.int32), _ptr(best_dDL, np.float64)))


def sbp_merge_blocks(m: int, round_id: int, n_merges: int) -> tuple[int, int]:
    B, rounds = C.c_int32(), C.c_int32()
    _check(lib().sbp_merge_blocks(m, round_id, n_merges, C.byref(B), C.byref(rounds)))
    return B.value, rounds.value


def sbp_compact(m: int) -> int:
    B = C.c_int32()
    _check(lib().sbp_compact(m, C.byref(B)))
    return B.value


def sbp_partition(g: int, b_out, params: Params | None = None, stream=None) -> tuple[int, float, int]:
    B, dl, ns = C.c_int32(), C.c_double(), C.c_int64()
    _check(lib().sbp_partition(g, C.byref(params) if params else None, _stream_ptr(stream), _ptr(b_out, np.int32), C.byref(B), C.byref(dl), C.byref(ns)))
    return B.value, dl.value, ns.value


def sbp_default_batch_options() -> BatchOptions:
    return BatchOptions.default()


def sbp_partition_batch(graphs: list[int], b_outs, params: Params | None = None,
                        options: BatchOptions | None = None, stats: BatchStats | None = None) -> list[BatchResult]:
    """graphs: handles; b_outs: None or one int32 buffer per graph."""
    n = len(graphs)
    ga = (C.c_void_p * max(n, 1))(*graphs)
    res = (BatchResult * max(n, 1))()
    if b_outs is None:
        bp = None
    else:
        bp = (C.c_void_p * max(n, 1))(*[_ptr(b, np.int32) for b in b_outs])
    _check(lib().sbp_partition_batch(ga, n, C.byref(params) if params else None,
                                     C.byref(options) if options else None, bp, res,
                                     C.byref(stats) if stats is not None else None))
    return [res[i] for i in range(n)]


def sbp_get_assignment(m: int, b_out) -> None:
    _check(lib().sbp_get_assignment(m, _ptr(b_out, np.int32)))


def sbp_get_pending(m: int, v_begin: int, v_end: int, out) -> None:
    _check(lib().sbp_get_pending(m, v_begin, v_end, _ptr(out, np.int32)))


def sbp_set_pending(m: int, v_begin: int, v_end: int, labels) -> None:
    _check(lib().sbp_set_pending(m, v_begin, v_end, _ptr(labels, np.int32)))


def sbp_get_B(m: int) -> int:
    B = C.c_int32()
    _check(lib().sbp_get_B(m, C.byref(B)))
    return B.value


def sbp_get_dl(m: int) -> float:
    out = np.zeros(1, np.float64)
    _check(lib().sbp_get_dl(m, out.ctypes.data))
    return float(out[0])


def sbp_get_blockmodel_dense(m: int, M_out) -> None:
    _check(lib().sbp_get_blockmodel_dense(m, _ptr(M_out, np.int32)))


def sbp_get_degrees(m: int, dout, din) -> None:
    _check(lib().sbp_get_degrees(m, _ptr(dout, np.int32), _ptr(din, np.int32)))


def sbp_get_blockmodel_coo(m: int):
    nnz = C.c_int64()
    rc = lib().sbp_get_blockmodel_coo(m, 0, None, None, C.byref(nnz))
    n = nnz.value
    keys = np.zeros(max(n, 1), np.int64)
    cnt = np.zeros(max(n, 1), np.int32)
    _check(lib().sbp_get_blockmodel_coo(m, n, keys.ctypes.data, cnt.ctypes.data, C.byref(nnz)))
    return keys[:n], cnt[:n]


def sbp_sync(m: int) -> None:
    _check(lib().sbp_sync(m))


def sbp_free_model(m: int) -> None:
    lib().sbp_free_model(m)


def sbp_dense_dl_noalloc(M, B: int, dout, din, E: int, N: int, dl_out, stream=None) -> None:
    """DL of a dense blockmodel from caller-owned device buffers, without
    allocating device memory (see include/sbp.h)."""
    _check(lib().sbp_dense_dl_noalloc(_ptr(M, np.int32), B, _ptr(dout, np.int32), _ptr(din, np.int32), E, N,
                                      _ptr(dl_out, np.float64), _stream_ptr(stream)))


def sbp_dxlogx32_check(x, k):
    """(val, am): the FP32 term f(x+k) - f(x) of the precision form and its
    error magnitude, evaluated on the device."""
    x = np.ascontiguousarray(x, np.int32)
    k = np.ascontiguousarray(k, np.int32)
    val = np.zeros(x.size, np.float32)
    am = np.zeros(x.size, np.float32)
    _check(lib().sbp_dxlogx32_check(x.ctypes.data, k.ctypes.data, int(x.size), val.ctypes.data, am.ctypes.data))
    return val, am


def sbp_bracket_check(B, dl, reduction: float = 0.5):
    """(out, n_bad): the persistent kernel's bracket code, run on the host,
    against the host driver's bracket over the states (B[i], dl[i]) inserted
    in order; out has 12 entries per state (host: position B values, next
    phase exists, start, target; then the same from the kernel's code)."""
    B = np.ascontiguousarray(B, np.int32)
    dl = np.ascontiguousarray(dl, np.float64)
    out = np.zeros((B.size, 12), np.int32)
    bad = C.c_int32(0)
    _check(lib().sbp_bracket_check(B.ctypes.data, dl.ctypes.data, int(B.size), float(reduction), out.ctypes.data,
                                   C.byref(bad)))
    return out, int(bad.value)


def sbp_kernel_launches() -> int:
    """Kernel launches issued by the library so far in this process."""
    n = C.c_uint64(0)
    _check(lib().sbp_kernel_launches(C.byref(n)))
    return int(n.value)


def sbp_philox_check(ctr, key, count: int = 1) -> np.ndarray:
    out = np.zeros(4 * count, np.uint64)
    c = [int(x) for x in ctr]
    k = [int(x) for x in key]
    _check(lib().sbp_philox_check(c[0], c[1], c[2], c[3], k[0], k[1], count, out.ctypes.data))
    return out.reshape(count, 4)


# ---------------------------------------------------------------------------
# small owning wrappers

class Graph:
    """A device-resident graph (CSR of out-edges and of in-edges)."""

    def __init__(self, n: int, src, dst):
        self.n = int(n)
        self.m = int(src.shape[0])
        self.h = sbp_load_graph(self.n, src, dst)

    def close(self) -> None:
        if getattr(self, "h", None):
            sbp_free_graph(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def partition(self, params: Params | None = None, stream=None):
        b = np.zeros(self.n, np.int32)
        B, dl, ns = sbp_partition(self.h, b, params, stream)
        return b, B, dl, ns


def partition_batch(graphs: list["Graph"], params: Params | None = None, options: BatchOptions | None = None,
                    stats: BatchStats | None = None):
    """Partitions every graph (the batching form); returns per graph
    (b, B, dl, n_sweeps, t_admit, t_done)."""
    outs = [np.zeros(g.n, np.int32) for g in graphs]
    res = sbp_partition_batch([g.h for g in graphs], outs, params, options, stats)
    return [(outs[i], r.B, r.dl, r.n_sweeps, r.t_admit, r.t_done) for i, r in enumerate(res)]


def sbp_autotune_batch(graphs: list[int], params: Params | None = None, sample: int = 64,
                       start: BatchOptions | None = None) -> tuple[BatchOptions, float, int]:
    """graphs: handles.  Returns (best options, graphs/s on the sample, timed runs)."""
    n = len(graphs)
    ga = (C.c_void_p * max(n, 1))(*graphs)
    best = start if start is not None else BatchOptions.default()
    rate, trials = C.c_double(), C.c_int32()
    _check(lib().sbp_autotune_batch(ga, n, C.byref(params) if params else None, sample, 1 if start is not None else 0,
                                    C.byref(best), C.byref(rate), C.byref(trials)))
    return best, rate.value, trials.value


def autotune_batch(graphs: list["Graph"], params: Params | None = None, sample: int = 64,
                   start: BatchOptions | None = None) -> tuple[BatchOptions, float, int]:
    """Options of the batching form tuned on a sample of these graphs."""
    return sbp_autotune_batch([g.h for g in graphs], params, sample, start)


def sbp_server_create(params: Params | None = None, options: BatchOptions | None = None) -> int:
    h = C.c_void_p()
    _check(lib().sbp_server_create(C.byref(params) if params else None, C.byref(options) if options else None,
                                   C.byref(h)))
    return h.value


def sbp_server_submit(s: int, g: int, b_out) -> int:
    rid = C.c_int64()
    _check(lib().sbp_server_submit(s, g, _ptr(b_out, np.int32) if b_out is not None else None, C.byref(rid)))
    return rid.value


def sbp_server_poll(s: int, request: int) -> bool:
    d = C.c_int32()
    _check(lib().sbp_server_poll(s, request, C.byref(d)))
    return bool(d.value)


def sbp_server_wait(s: int, request: int) -> BatchResult:
    r = BatchResult()
    _check(lib().sbp_server_wait(s, request, C.byref(r)))
    return r


def sbp_server_stats(s: int) -> BatchStats:
    st = BatchStats()
    _check(lib().sbp_server_stats(s, C.byref(st)))
    return st


def sbp_server_destroy(s: int) -> None:
    lib().sbp_server_destroy(s)


class Server:
    """The serving form: submit graphs at any time, wait for their results.
    Keeps each submitted graph and its label buffer alive until done."""

    def __init__(self, params: Params | None = None, options: BatchOptions | None = None):
        self.h = sbp_server_create(params, options)
        self._keep: dict[int, tuple] = {}

    def submit(self, g: "Graph") -> int:
        b = np.zeros(g.n, np.int32)
        rid = sbp_server_submit(self.h, g.h, b)
        self._keep[rid] = (g, b)
        return rid

    def done(self, rid: int) -> bool:
        return sbp_server_poll(self.h, rid)

    def wait(self, rid: int):
        """(b, B, dl, n_sweeps, t_submit, t_admit, t_done)"""
        r = sbp_server_wait(self.h, rid)
        g, b = self._keep.pop(rid)
        return b, r.B, r.dl, r.n_sweeps, r.t_submit, r.t_admit, r.t_done

    def stats(self) -> BatchStats:
        return sbp_server_stats(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            sbp_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        self.close()


class Model:
    """A blockmodel (assignment, M, degrees, DL) resident on the device."""

    def __init__(self, g: Graph, B: int, b, params: Params | None = None, stream=None):
        self.g = g
        self.h = sbp_build_blockmodel(g.h, B, b, params, stream)

    def close(self) -> None:
        if getattr(self, "h", None):
            sbp_free_model(self.h)
            self.h = None

    def __del__(self):
        self.close()

    @property
    def B(self) -> int:
        return sbp_get_B(self.h)

    def assignment(self) -> np.ndarray:
        b = np.zeros(self.g.n, np.int32)
        sbp_get_assignment(self.h, b)
        return b

    def dense(self) -> np.ndarray:
        B = self.B
        M = np.zeros(B * B, np.int32)
        sbp_get_blockmodel_dense(self.h, M)
        return M.reshape(B, B)

    def coo(self):
        return sbp_get_blockmodel_coo(self.h)

    def degrees(self):
        B = self.B
        dout, din = np.zeros(B, np.int32), np.zeros(B, np.int32)
        sbp_get_degrees(self.h, dout, din)
        return dout, din

    def dl(self) -> float:
        return sbp_get_dl(self.h)

    def sweep(self, sweep_id: int, v_begin: int = 0, v_end: int | None = None, stats: bool = True):
        return sbp_nodal_sweep(self.h, sweep_id, v_begin, self.g.n if v_end is None else v_end, stats)


from .shard import deal_vertices  # noqa: E402  (Section III-B dealing)

