"""CPU oracle for the SBP hot path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
the two share no code.  ``build()`` compiles ``sbp_oracle.c`` with the host
C compiler into ``oracle/_build/``.

Parity status per step (details in ``sbp_oracle.c``): the blockmodel and
description length (Eq. 1-2), Philox, the nodal proposal / Delta DL /
Hastings and the acceptance draw, the merge Delta DL and the merge
application (with its further rounds), the MCMC stop rule and the phase
sequence of a full run are pinned by the tests; the driver's constants are
readings of the paper, not values it gives.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbp_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


class _Params(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64),
        ("beta", C.c_double),
        ("merge_proposals", C.c_int64),
        ("reduction", C.c_double),
        ("t_pre", C.c_double),
        ("t_post", C.c_double),
        ("max_sweeps", C.c_int64),
        ("hybrid_h", C.c_int64),
        ("dense_max_B", C.c_int64),
    ]


def lib():
    global _lib
    if _lib is not None:
        return _lib
    L = C.CDLL(build())
    vp, i64, u64, f64, ci = C.c_void_p, C.c_int64, C.c_uint64, C.c_double, C.c_int
    sig = {
        "og_philox4x64": (None, [u64p, u64p, u64p]),
        "og_graph_new": (vp, [i64, i64, i32p, i32p]),
        "og_graph_free": (None, [vp]),
        "og_graph_csr": (None, [vp, i64p, i32p, i64p, i32p]),
        "og_model_new": (vp, [vp, i64, i32p]),
        "og_model_free": (None, [vp]),
        "og_model_set_b": (ci, [vp, i64, i32p]),
        "og_model_nnz": (i64, [vp]),
        "og_model_B": (i64, [vp]),
        "og_model_get": (None, [vp, vp, vp, vp, vp, vp]),
        "og_model_L": (f64, [vp]),
        "og_model_dl": (f64, [vp]),
        "og_dl": (f64, [i64, i64, i64, f64]),
        "og_move_delta": (ci, [vp, i64, i64, C.POINTER(f64), C.POINTER(f64), C.POINTER(f64)]),
        "og_nodal_decide": (i64, [vp, u64, u64, f64, i64, i64, i32p, vp, vp, vp, vp, vp, ci]),
        "og_hybrid_decide": (i64, [vp, u64, u64, f64, i64, i32p, vp, vp, vp, vp, vp, ci]),
        "og_merge_delta": (f64, [vp, i64, i64]),
        "og_merge_key": (i64, [f64]),
        "og_merge_propose": (i64, [vp, u64, u64, i64, i64]),
        "og_merge_proposals": (None, [vp, u64, u64, i64, i32p, f64p, ci]),
        "og_merge_apply": (i64, [i64, i32p, f64p, i64, i32p, C.POINTER(i64)]),
        "og_compact": (i64, [i64, i64, i32p]),
        "og_bracket_new": (vp, []),
        "og_bracket_free": (None, [vp]),
        "og_bracket_insert": (None, [vp, i64, f64]),
        "og_bracket_next": (ci, [vp, f64, i64p, f64p, C.POINTER(ci), C.POINTER(i64)]),
        "og_partition": (ci, [vp, C.POINTER(_Params), i32p, C.POINTER(i64), C.POINTER(f64), C.POINTER(i64), ci, vp, i64,
                              C.POINTER(i64)]),
        "og_mcmc_phase": (i64, [vp, C.POINTER(_Params), u64, f64, ci, f64p]),
        "og_merge_phase": (i64, [vp, C.POINTER(_Params), u64, i64, ci, C.POINTER(i64)]),
        "og_max_threads": (ci, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def philox4x64(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint64)
    lib().og_philox4x64(np.ascontiguousarray(ctr, np.uint64), np.ascontiguousarray(key, np.uint64), out)
    return out


def dl(E: int, V: int, C_: int, L: float) -> float:
    return lib().og_dl(E, V, C_, L)


def merge_key(d: float) -> int:
    return lib().og_merge_key(d)


def max_threads() -> int:
    return lib().og_max_threads()


class Graph:
    """Directed graph in CSR (out) + CSC (in), neighbour lists ascending."""

    def __init__(self, n: int, src, dst):
        src = np.ascontiguousarray(src, np.int32)
        dst = np.ascontiguousarray(dst, np.int32)
        self.n, self.m = int(n), int(src.size)
        self._h = lib().og_graph_new(self.n, self.m, src, dst)
        if not self._h:
            raise ValueError("vertex id out of range")

    def csr(self):
        op = np.zeros(self.n + 1, np.int64)
        ip = np.zeros(self.n + 1, np.int64)
        oc = np.zeros(max(self.m, 1), np.int32)
        ic = np.zeros(max(self.m, 1), np.int32)
        lib().og_graph_csr(self._h, op, oc, ip, ic)
        return op, oc[: self.m], ip, ic[: self.m]

    def __del__(self):
        if getattr(self, "_h", None):
            lib().og_graph_free(self._h)
            self._h = None


@dataclass
class Decisions:
    b_new: np.ndarray
    s: np.ndarray
    flags: np.ndarray
    dH: np.ndarray
    logA: np.ndarray
    lnu: np.ndarray
    accepted: int


class Model:
    """Blockmodel of a graph under an assignment (Eq. 1-2 state)."""

    def __init__(self, g: Graph, B: int, b):
        self.g = g
        b = np.ascontiguousarray(b, np.int32)
        self._h = lib().og_model_new(g._h, int(B), b)
        if not self._h:
            raise ValueError("label out of range")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().og_model_free(self._h)
            self._h = None

    @property
    def B(self) -> int:
        return lib().og_model_B(self._h)

    def set_b(self, B: int, b) -> None:
        if lib().og_model_set_b(self._h, int(B), np.ascontiguousarray(b, np.int32)) != 0:
            raise ValueError("label out of range")

    def coo(self):
        nnz = lib().og_model_nnz(self._h)
        keys = np.zeros(max(nnz, 1), np.int64)
        cnt = np.zeros(max(nnz, 1), np.int64)
        lib().og_model_get(self._h, _ptr(keys), _ptr(cnt), None, None, None)
        return keys[:nnz], cnt[:nnz]

    def dense(self) -> np.ndarray:
        B = self.B
        keys, cnt = self.coo()
        M = np.zeros(B * B, np.int64)
        M[keys] = cnt
        return M.reshape(B, B)

    def degrees(self):
        B = self.B
        dout = np.zeros(B, np.int64)
        din = np.zeros(B, np.int64)
        lib().og_model_get(self._h, None, None, _ptr(dout), _ptr(din), None)
        return dout, din

    def assignment(self) -> np.ndarray:
        b = np.zeros(self.g.n, np.int32)
        lib().og_model_get(self._h, None, None, None, None, _ptr(b))
        return b

    def L(self) -> float:
        return lib().og_model_L(self._h)

    def dl(self) -> float:
        return lib().og_model_dl(self._h)

    def move_delta(self, v: int, s: int):
        dH, pf, pb = C.c_double(), C.c_double(), C.c_double()
        if lib().og_move_delta(self._h, v, s, C.byref(dH), C.byref(pf), C.byref(pb)) != 0:
            raise ValueError("bad move")
        return dH.value, pf.value, pb.value

    def nodal_decide(self, seed: int, sweep_id: int, beta: float, v_begin: int = 0, v_end: int | None = None, nthreads: int = 1) -> Decisions:
        n = self.g.n
        v_end = n if v_end is None else v_end
        b_new = self.assignment()
        s = np.zeros(n, np.int32)
        flags = np.zeros(n, np.int32)
        dH = np.zeros(n, np.float64)
        logA = np.zeros(n, np.float64)
        lnu = np.zeros(n, np.float64)
        acc = lib().og_nodal_decide(self._h, seed, sweep_id, beta, v_begin, v_end, b_new, _ptr(s), _ptr(flags), _ptr(dH), _ptr(logA), _ptr(lnu), nthreads)
        return Decisions(b_new, s, flags, dH, logA, lnu, int(acc))

    def hybrid_decide(self, seed: int, sweep_id: int, beta: float, h: int, nthreads: int = 1) -> Decisions:
        """Hybrid pass: the h highest-degree vertices sequentially (the model
        is updated by each accepted move), then the rest by asynchronous
        Gibbs against the resulting model.  The model keeps the state after
        the sequential part; commit b_new with set_b."""
        n = self.g.n
        b_new = self.assignment()
        s = np.zeros(n, np.int32)
        flags = np.zeros(n, np.int32)
        dH = np.zeros(n, np.float64)
        logA = np.zeros(n, np.float64)
        lnu = np.zeros(n, np.float64)
        acc = lib().og_hybrid_decide(self._h, seed, sweep_id, beta, h, b_new, _ptr(s), _ptr(flags), _ptr(dH), _ptr(logA),
                                     _ptr(lnu), nthreads)
        return Decisions(b_new, s, flags, dH, logA, lnu, int(acc))

    def mcmc_phase(self, p: "Params", sweep_id: int, t: float, nthreads: int = 1):
        """One MCMC phase (Alg. 2) from the current state, sweep ids from
        sweep_id on; the model ends in the phase's final state.  Returns
        (sweeps run, DL after 0..sweeps sweeps)."""
        hist = np.zeros(p.max_sweeps + 1, np.float64)
        ns = lib().og_mcmc_phase(self._h, C.byref(_cparams(p)), sweep_id, t, nthreads, hist)
        return int(ns), hist[: ns + 1]

    def merge_phase(self, p: "Params", round_id: int, n_merges: int, nthreads: int = 1):
        """One merge phase (Alg. 1) from the current state, round ids from
        round_id on.  Returns (B after, proposal rounds taken)."""
        rounds = C.c_int64()
        Bn = lib().og_merge_phase(self._h, C.byref(_cparams(p)), round_id, n_merges, nthreads, C.byref(rounds))
        return int(Bn), int(rounds.value)

    def merge_delta(self, r: int, s: int) -> float:
        return lib().og_merge_delta(self._h, r, s)

    def merge_propose(self, seed: int, round_id: int, r: int, i: int) -> int:
        return int(lib().og_merge_propose(self._h, seed, round_id, r, i))

    def merge_proposals(self, seed: int, round_id: int, x: int = 10, nthreads: int = 1):
        B = self.B
        bs = np.zeros(B, np.int32)
        bd = np.zeros(B, np.float64)
        lib().og_merge_proposals(self._h, seed, round_id, x, bs, bd, nthreads)
        return bs, bd


def merge_apply(B: int, best_s, best_dDL, n_merges: int):
    m = np.zeros(B, np.int32)
    Bn = C.c_int64()
    done = lib().og_merge_apply(B, np.ascontiguousarray(best_s, np.int32), np.ascontiguousarray(best_dDL, np.float64), n_merges, m, C.byref(Bn))
    return int(done), m, int(Bn.value)


def compact(B: int, b) -> tuple[int, np.ndarray]:
    b = np.ascontiguousarray(b, np.int32).copy()
    Bn = lib().og_compact(b.size, B, b)
    return int(Bn), b


class Bracket:
    """The golden-ratio bracket rule on its own (hi, mid, lo by C)."""

    def __init__(self):
        self._h = lib().og_bracket_new()

    def __del__(self):
        if getattr(self, "_h", None):
            lib().og_bracket_free(self._h)
            self._h = None

    def insert(self, B: int, dl: float) -> None:
        lib().og_bracket_insert(self._h, B, dl)

    def next(self, reduction: float = 0.5):
        Bs = np.zeros(3, np.int64)
        dls = np.zeros(3, np.float64)
        st, tg = C.c_int(), C.c_int64()
        more = lib().og_bracket_next(self._h, reduction, Bs, dls, C.byref(st), C.byref(tg))
        return bool(more), Bs, dls, int(st.value), int(tg.value)


@dataclass
class Params:
    seed: int = 0
    beta: float = 3.0
    merge_proposals: int = 10
    reduction: float = 0.5
    t_pre: float = 5e-4
    t_post: float = 1e-4
    max_sweeps: int = 100
    hybrid_h: int = 0
    dense_max_B: int = 4096


def _cparams(p: Params) -> _Params:
    return _Params(p.seed, p.beta, p.merge_proposals, p.reduction, p.t_pre, p.t_post, p.max_sweeps, p.hybrid_h,
                   p.dense_max_B)


def partition(g: Graph, p: Params = Params(), nthreads: int = 1, phase_log: bool = False):
    """Full run.  Returns (b, B, DL, sweeps), plus with phase_log a
    (phases, 7) array: start B, target B, B after the merges, MCMC
    threshold t, sweeps, compacted B and its DL."""
    cp = _cparams(p)
    b = np.zeros(g.n, np.int32)
    B, d, ns, nl = C.c_int64(), C.c_double(), C.c_int64(), C.c_int64()
    cap = 4096 if phase_log else 0
    log = np.zeros((max(cap, 1), 7), np.float64)
    if lib().og_partition(g._h, C.byref(cp), b, C.byref(B), C.byref(d), C.byref(ns), nthreads,
                          _ptr(log) if phase_log else None, cap, C.byref(nl)) != 0:
        raise RuntimeError("partition failed")
    out = (b, int(B.value), float(d.value), int(ns.value))
    if phase_log:
        return out + (log[: min(int(nl.value), cap)].copy(),)
    return out
