"""CPU oracle for higher-order (k,h)-truss decomposition -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  It is a plain, single-threaded C implementation of the paper's
definitions (Sec. 2, Def. 2-4) and of level-synchronous peeling (Sec. 3, Algorithm 1)
with every h-support recomputed from scratch after each removal round.  It shares no
code with the CUDA path.

Parity status of each function (what pins it, in ``tests/test_oracle_pins.py``):

* ``normalise``           -- pinned: set semantics checked against a Python set build.
* ``OracleGraph.h_support`` -- pinned: brute-force all-pairs distances (Floyd-Warshall)
  on small graphs, closed forms (K_n, star, path, cycle, K_{a,b}), h=1 triangle counts.
* ``OracleGraph.truss_decompose`` -- pinned: exhaustive Def. 4 brute force over edge
  subsets (m <= 12), closed forms, h=1 equals an independent classic truss peel,
  the literal one-edge-at-a-time Algorithm 1, monotonicity in h, t <= sup + 2,
  the paper's surviving worked-example value (minimum 2-support 2 -> 2-trussness 4).
* ``OracleGraph.certify`` -- pinned: accepts the oracle's own decompositions and rejects
  planted errors (t off by one, stamps swapped) on small graphs.
* ``certify_all`` (``htd_cert.c``, multithreaded) -- pinned: its h-supports in the growing
  subgraphs equal Floyd-Warshall's on every edge; it accepts every oracle decomposition
  and rejects every claim with a wrong trussness (``tests/test_cert_pins.py``).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "htd_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "htd_cert.c")]
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle_htd.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle_htd.so (portable flags)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-o", tmp,
                           *_SRCS])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i32, i64, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        lib.htdo_normalise.argtypes = [i32, p, p, i64, p, p]
        lib.htdo_normalise.restype = i64
        lib.htdo_graph_new.argtypes = [i32, i64, p, p]
        lib.htdo_graph_new.restype = p
        lib.htdo_graph_free.argtypes = [p]
        lib.htdo_graph_free.restype = None
        lib.htdo_edge_h_support.argtypes = [p, i32, p, i32, i64]
        lib.htdo_edge_h_support.restype = i32
        lib.htdo_h_support.argtypes = [p, i32, p, i32, p]
        lib.htdo_h_support.restype = None
        lib.htdo_truss_decompose.argtypes = [p, i32, p, p]
        lib.htdo_truss_decompose.restype = i64
        lib.htdo_truss_sequential.argtypes = [p, i32, p]
        lib.htdo_truss_sequential.restype = i32
        lib.htdo_certify.argtypes = [p, i32, p, p, p, i64, p]
        lib.htdo_certify.restype = i64
        lib.htdo_check_stamp_order.argtypes = [i64, p, p]
        lib.htdo_check_stamp_order.restype = i64
        lib.htdo_hindex.argtypes = [p, i32, i32, i32, p, p]
        lib.htdo_hindex.restype = i32
        lib.htdo_hindex_pruned.argtypes = [p, i32, i32, p, p, p]
        lib.htdo_hindex_pruned.restype = i32
        lib.htdo_certify_all.argtypes = [i32, i64, p, p, i32, p, p, i32, p, p, p, p]
        lib.htdo_certify_all.restype = i64
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def normalise(n: int, src, dst):
    """Canonical edge list (eu < ev, lexicographic, distinct, no loops) as int32 arrays."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    eu = np.empty(max(1, src.size), dtype=np.int32)
    ev = np.empty(max(1, src.size), dtype=np.int32)
    m = lib.htdo_normalise(int(n), _ptr(src), _ptr(dst), src.size, _ptr(eu), _ptr(ev))
    if m == -1:
        raise ValueError("vertex id outside [0, n) or negative n")
    if m < 0:
        raise MemoryError("oracle normalise: allocation failed")
    return eu[:m].copy(), ev[:m].copy()


class OracleGraph:
    """A normalised graph held by the C oracle."""

    def __init__(self, n: int, eu, ev):
        self._lib = _load()
        self.n = int(n)
        self.eu = np.ascontiguousarray(eu, dtype=np.int32)
        self.ev = np.ascontiguousarray(ev, dtype=np.int32)
        self.m = int(self.eu.size)
        self._g = self._lib.htdo_graph_new(self.n, self.m, _ptr(self.eu), _ptr(self.ev))
        if not self._g:
            raise MemoryError("oracle graph allocation failed")

    @classmethod
    def from_raw(cls, n: int, src, dst):
        eu, ev = normalise(n, src, dst)
        return cls(n, eu, ev)

    def __del__(self):
        g = getattr(self, "_g", None)
        if g:
            self._lib.htdo_graph_free(g)
            self._g = None

    def h_support(self, h: int, key=None, thr: int = 0) -> np.ndarray:
        """sup(e,h) for every edge of {key >= thr} (all edges if key is None), -1 elsewhere."""
        out = np.empty(max(1, self.m), dtype=np.int32)
        k = None if key is None else np.ascontiguousarray(key, dtype=np.int32)
        self._lib.htdo_h_support(self._g, int(h), _ptr(k), int(thr), _ptr(out))
        return out[: self.m]

    def edge_h_support(self, h: int, e: int, key=None, thr: int = 0) -> int:
        k = None if key is None else np.ascontiguousarray(key, dtype=np.int32)
        return int(self._lib.htdo_edge_h_support(self._g, int(h), _ptr(k), int(thr), int(e)))

    def truss_decompose(self, h: int):
        """(t, stamp, rounds): level-synchronous peel with full recomputation."""
        t = np.zeros(max(1, self.m), dtype=np.int32)
        st = np.zeros(max(1, self.m), dtype=np.int32)
        r = self._lib.htdo_truss_decompose(self._g, int(h), _ptr(t), _ptr(st))
        if r < 0:
            raise MemoryError("oracle decomposition: allocation failed")
        return t[: self.m], st[: self.m], int(r)

    def truss_sequential(self, h: int) -> np.ndarray:
        """Algorithm 1 literally, one edge at a time (tiny graphs only)."""
        t = np.zeros(max(1, self.m), dtype=np.int32)
        if self._lib.htdo_truss_sequential(self._g, int(h), _ptr(t)) != 0:
            raise MemoryError("oracle sequential peel: allocation failed")
        return t[: self.m]

    def hindex(self, h: int, asynchronous: bool = False, max_iter: int = -1):
        """The H-index iteration of Sec. 4 from H^(0) = sup(e,h).  Returns (H values after
        the last order computed, orders computed, converged).  Converged: t = H + 2."""
        hv = np.zeros(max(1, self.m), dtype=np.int32)
        it = ctypes.c_int32()
        rc = self._lib.htdo_hindex(self._g, int(h), int(bool(asynchronous)), int(max_iter),
                                   _ptr(hv), ctypes.byref(it))
        if rc < 0:
            raise MemoryError("oracle H-index iteration: allocation failed")
        return hv[: self.m], int(it.value), rc == 1

    def hindex_pruned(self, h: int, max_iter: int = -1):
        """Synchronous H-index iteration with the Lemma 4 pruning of Sec. 4.  Returns (H
        values, orders computed, converged, H^(n)(e) evaluations actually computed)."""
        hv = np.zeros(max(1, self.m), dtype=np.int32)
        it = ctypes.c_int32()
        ev = ctypes.c_int64()
        rc = self._lib.htdo_hindex_pruned(self._g, int(h), int(max_iter), _ptr(hv),
                                          ctypes.byref(it), ctypes.byref(ev))
        if rc < 0:
            raise MemoryError("oracle pruned H-index iteration: allocation failed")
        return hv[: self.m], int(it.value), rc == 1, int(ev.value)

    def certify(self, h: int, t, stamp, edges=None):
        """Peeling certificate: returns (stamp_order_violations, failing_edges, fail_codes).

        fail code 1 = validity fails (sup in {t >= t(e)} below t(e)-2), 2 = removability
        fails (sup in {stamp >= stamp(e)} above t(e)-2)."""
        t = np.ascontiguousarray(t, dtype=np.int32)
        stamp = np.ascontiguousarray(stamp, dtype=np.int32)
        order_bad = int(self._lib.htdo_check_stamp_order(self.m, _ptr(t), _ptr(stamp)))
        if edges is None:
            ed = None
            ne = self.m
        else:
            ed = np.ascontiguousarray(edges, dtype=np.int64)
            ne = ed.size
        fails = np.zeros(max(1, ne), dtype=np.int32)
        self._lib.htdo_certify(self._g, int(h), _ptr(t), _ptr(stamp), _ptr(ed), int(ne),
                               _ptr(fails))
        fails = fails[:ne]
        idx = np.nonzero(fails)[0]
        bad_edges = idx if ed is None else ed[idx]
        return order_bad, bad_edges, fails[idx]


def certify_all(n: int, eu, ev, h: int, t, stamp, threads: int | None = None,
                sups: bool = False):
    """All-edge peeling certificate of a claimed decomposition (``htd_cert.c``).

    Checks, on every edge, that stamps are ordered like t, validity (sup in {t >= t(e)}
    at least t(e)-2) and removability (sup in {stamp >= stamp(e)} at most t(e)-2); the
    three together prove t exact.  Returns (order_bad, failing_edges, fail_codes) and,
    with ``sups``, also (sup_rem, sup_val).  fail code bit 1 = validity, bit 2 =
    removability.  order_bad > 0 means nothing else was checked."""
    lib = _load()
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    t = np.ascontiguousarray(t, dtype=np.int32)
    stamp = np.ascontiguousarray(stamp, dtype=np.int32)
    m = eu.size
    if not (ev.size == t.size == stamp.size == m):
        raise ValueError("edge, t and stamp arrays differ in length")
    if threads is None:
        threads = os.cpu_count() or 1
    fail = np.zeros(max(1, m), dtype=np.int32)
    sr = np.full(max(1, m), -1, dtype=np.int32) if sups else None
    sv = np.full(max(1, m), -1, dtype=np.int32) if sups else None
    ob = ctypes.c_int64(0)
    rc = lib.htdo_certify_all(int(n), m, _ptr(eu), _ptr(ev), int(h), _ptr(t), _ptr(stamp),
                              int(threads), _ptr(fail), _ptr(sr), _ptr(sv), ctypes.byref(ob))
    if rc == -1:
        raise MemoryError("certificate: allocation failed")
    if rc == -2:
        raise ValueError("certificate: bad argument (h out of range or a stamp outside [0, m])")
    fail = fail[:m]
    idx = np.nonzero(fail)[0]
    out = (int(ob.value), idx, fail[idx])
    if sups:
        out = out + (sr[:m], sv[:m])
    return out
