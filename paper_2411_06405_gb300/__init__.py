"""Higher-order (k,h)-truss decomposition on GB300 (sm_103a): Python binding.

Thin marshalling over the C ABI of ``include/htruss.h``; every function keeps the C
entry point's name.  PyTorch provides device memory and the current CUDA stream; all
computation happens in the library's CUDA kernels.  There is no CPU fallback: importing
the binding succeeds without a GPU, but every call needs the built library and a device.

Method (Chen et al. 2024): h-support sup(e,h) = number of vertices within h hops of both
endpoints of e (Def. 2, Def. 3); t(e,h) = largest k such that e lies in the (k,h)-truss,
the maximal edge set whose every edge has h-support >= k-2 inside it (Def. 4), computed
by level-synchronous peeling (Sec. 3).
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (HTD_MAX_H, HTD_MAX_N, HTD_OPT_NO_GRAPH, HTD_OPT_REBUILD, HTD_OPT_TIMING,
                   HTD_OPT_TINY_LOSS_TABLE, HTD_OPT_PERSISTENT_ROUNDS, HTD_OPT_COMPACT_BALLS,
                   HTD_OPT_BATCH_BLOCKS, HtdError, HtdStats)

__all__ = [
    "HTD_MAX_H", "HTD_MAX_N", "HTD_OPT_NO_GRAPH", "HTD_OPT_REBUILD", "HTD_OPT_TIMING",
    "HTD_OPT_TINY_LOSS_TABLE", "HTD_OPT_PERSISTENT_ROUNDS", "HTD_OPT_COMPACT_BALLS",
    "HTD_OPT_BATCH_BLOCKS", "HtdError",
    "HtdStats",
    "Graph", "htd_build_csr", "htd_graph_info", "htd_edges", "htd_csr", "htd_h_support",
    "htd_truss_decompose", "htd_truss_decompose_host", "htd_h_support_static", "htd_graph_free",
    "htd_truss_decompose_batched", "BatchInput", "Server", "htd_footprint_estimate", "htd_hindex_decompose",
    "library_path",
]


def _torch():
    import torch

    return torch


def library_path() -> str:
    return _lib.LIB_PATH


def _stream_handle(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


class Graph:
    """Owns an ``htd_graph`` handle (CSR of the normalised graph on one device)."""

    def __init__(self, handle: ctypes.c_void_p, device):
        self._h = handle
        self.device = device
        n = ctypes.c_int32()
        m = ctypes.c_int64()
        _lib.check(_lib.load().htd_graph_info(self._h, ctypes.byref(n), ctypes.byref(m)),
                   "htd_graph_info")
        self.n = int(n.value)
        self.m = int(m.value)

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            _lib.load().htd_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def htd_build_csr(n: int, src, dst, stream=None) -> Graph:
    """Normalise an undirected edge list and build the graph on the current device.

    ``src``/``dst``: int32 torch tensors (CUDA or CPU) or numpy arrays of equal length."""
    torch = _torch()
    lib = _lib.load()
    if isinstance(src, np.ndarray):
        src = torch.from_numpy(np.ascontiguousarray(src, dtype=np.int32))
    if isinstance(dst, np.ndarray):
        dst = torch.from_numpy(np.ascontiguousarray(dst, dtype=np.int32))
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    src = src.to(torch.int32).contiguous()
    dst = dst.to(torch.int32).contiguous()
    on_dev = 1 if src.is_cuda else 0
    if src.is_cuda != dst.is_cuda:
        raise ValueError("src and dst must be on the same device")
    out = ctypes.c_void_p()
    st = lib.htd_build_csr(int(n), _ptr(src), _ptr(dst), int(src.numel()), on_dev,
                           _stream_handle(stream), ctypes.byref(out))
    _lib.check(st, "htd_build_csr")
    return Graph(out, torch.device("cuda", torch.cuda.current_device()))


def htd_graph_info(g: Graph):
    return g.n, g.m


def htd_edges(g: Graph, stream=None):
    """Canonical edges (eu < ev, lexicographic) as two int32 CUDA tensors of length m."""
    torch = _torch()
    eu = torch.empty(g.m, dtype=torch.int32, device=g.device)
    ev = torch.empty(g.m, dtype=torch.int32, device=g.device)
    _lib.check(_lib.load().htd_edges(g.handle, _ptr(eu), _ptr(ev), _stream_handle(stream)),
               "htd_edges")
    return eu, ev


def htd_csr(g: Graph, stream=None):
    """(row_ptr[n+1], col[2m], slot_eid[2m]) int32 CUDA tensors."""
    torch = _torch()
    row_ptr = torch.empty(g.n + 1, dtype=torch.int32, device=g.device)
    col = torch.empty(2 * g.m, dtype=torch.int32, device=g.device)
    slot_eid = torch.empty(2 * g.m, dtype=torch.int32, device=g.device)
    _lib.check(_lib.load().htd_csr(g.handle, _ptr(row_ptr), _ptr(col), _ptr(slot_eid),
                                   _stream_handle(stream)), "htd_csr")
    return row_ptr, col, slot_eid


def htd_h_support(g: Graph, h: int, out=None, stream=None):
    """sup(e,h) for every edge id, int32 CUDA tensor of length m."""
    torch = _torch()
    if out is None:
        out = torch.empty(g.m, dtype=torch.int32, device=g.device)
    _lib.check(_lib.load().htd_h_support(g.handle, int(h), _ptr(out), _stream_handle(stream)),
               "htd_h_support")
    return out


def htd_truss_decompose(g: Graph, h: int, stamps: bool = False, flags: int = 0, out=None,
                        stream=None):
    """t(e,h) for every edge id.  Returns (truss, stamp or None, stats dict)."""
    torch = _torch()
    if out is None:
        out = torch.empty(g.m, dtype=torch.int32, device=g.device)
    stamp = torch.empty(g.m, dtype=torch.int32, device=g.device) if stamps else None
    stats = HtdStats()
    st = _lib.load().htd_truss_decompose_ex(g.handle, int(h), int(flags), _ptr(out),
                                            _ptr(stamp) if stamp is not None else ctypes.c_void_p(0),
                                            ctypes.byref(stats), _stream_handle(stream))
    _lib.check(st, "htd_truss_decompose")
    return out, stamp, stats.as_dict()


def htd_truss_decompose_host(n: int, src, dst, h: int, out_eu=None, out_ev=None,
                             out_truss=None, stream=None):
    """End-to-end call on host buffers.  ``src``/``dst`` and the optional outputs are
    CPU int32 tensors (pinned memory is faster) or numpy arrays; the outputs need room
    for len(src) entries.  Returns (eu, ev, truss, stats) trimmed to the m edges."""
    torch = _torch()

    def host(a):
        if isinstance(a, np.ndarray):
            a = torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32))
        if a.is_cuda:
            raise ValueError("htd_truss_decompose_host takes host buffers")
        return a.to(torch.int32).contiguous()

    src, dst = host(src), host(dst)
    k = int(src.numel())
    out_eu = torch.empty(max(k, 1), dtype=torch.int32) if out_eu is None else out_eu
    out_ev = torch.empty(max(k, 1), dtype=torch.int32) if out_ev is None else out_ev
    out_truss = torch.empty(max(k, 1), dtype=torch.int32) if out_truss is None else out_truss
    m = ctypes.c_int64()
    stats = HtdStats()
    st = _lib.load().htd_truss_decompose_host(int(n), _ptr(src), _ptr(dst), k, int(h),
                                              ctypes.c_void_p(out_eu.data_ptr()),
                                              ctypes.c_void_p(out_ev.data_ptr()),
                                              ctypes.c_void_p(out_truss.data_ptr()),
                                              ctypes.byref(m), ctypes.byref(stats),
                                              _stream_handle(stream))
    _lib.check(st, "htd_truss_decompose_host")
    mm = int(m.value)
    return out_eu[:mm], out_ev[:mm], out_truss[:mm], stats.as_dict()


class BatchInput:
    """A batch of graphs concatenated once on the device (raw pairs with per-graph offsets),
    so that it can be decomposed repeatedly with its inputs resident."""

    def __init__(self, graphs, device=None):
        torch = _torch()
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        k = len(graphs)
        self.count = k
        self.n = np.zeros(max(k, 1), dtype=np.int32)
        self.h = np.zeros(max(k, 1), dtype=np.int32)
        self.off = np.zeros(k + 1, dtype=np.int64)
        srcs, dsts = [], []
        for i, (ng, s, d, hg) in enumerate(graphs):
            s = np.ascontiguousarray(s.cpu().numpy() if hasattr(s, "cpu") else s, dtype=np.int32).reshape(-1)
            d = np.ascontiguousarray(d.cpu().numpy() if hasattr(d, "cpu") else d, dtype=np.int32).reshape(-1)
            if s.shape != d.shape:
                raise ValueError(f"graph {i}: src and dst differ in length")
            self.n[i], self.h[i] = int(ng), int(hg)
            self.off[i + 1] = self.off[i] + s.size
            srcs.append(s)
            dsts.append(d)
        self.total = int(self.off[-1])
        cat = lambda xs: np.concatenate(xs) if xs else np.zeros(0, np.int32)
        self.src = torch.from_numpy(cat(srcs)).to(dev)
        self.dst = torch.from_numpy(cat(dsts)).to(dev)
        self.out = torch.empty(max(self.total, 1), dtype=torch.int32, device=dev)
        self.device = dev


def htd_truss_decompose_batched(graphs, flags: int = 0, max_union_vertices: int = 0,
                                device=None, stream=None):
    """Decomposes many graphs in one call.  ``graphs``: a BatchInput, or a sequence of
    (n, src, dst, h) with src/dst int32 tensors or numpy arrays of local ids in [0, n).
    Returns (list of int32 CUDA tensors, one per graph, t(e,h) over that graph's canonical
    edges; stats dict with the number of unions under "unions")."""
    b = graphs if isinstance(graphs, BatchInput) else BatchInput(graphs, device)
    k = b.count
    out_off = np.zeros(max(k, 1), dtype=np.int64)
    out_m = np.zeros(max(k, 1), dtype=np.int64)
    unions = ctypes.c_int32()
    stats = HtdStats()
    vp = lambda a: ctypes.c_void_p(a.ctypes.data)
    st = _lib.load().htd_truss_decompose_batched(
        k, vp(b.n), vp(b.h), vp(b.off), _ptr(b.src), _ptr(b.dst), int(flags),
        int(max_union_vertices), ctypes.c_void_p(b.out.data_ptr()), vp(out_off), vp(out_m),
        ctypes.byref(unions), ctypes.byref(stats), _stream_handle(stream))
    _lib.check(st, "htd_truss_decompose_batched")
    res = [b.out[int(out_off[i]):int(out_off[i]) + int(out_m[i])] for i in range(k)]
    sd = stats.as_dict()
    sd["unions"] = int(unions.value)
    return res, sd


def htd_h_support_static(n: int, row_ptr, col, eu, ev, h: int, out, stream=None):
    """Allocation-free h-support on caller-provided CUDA tensors (CSR + edges + output).
    Enqueues on the stream and returns without waiting."""
    _lib.check(_lib.load().htd_h_support_static(int(n), _ptr(row_ptr), _ptr(col), int(eu.numel()),
                                                _ptr(eu), _ptr(ev), int(h), _ptr(out),
                                                _stream_handle(stream)), "htd_h_support_static")
    return out


def htd_hindex_decompose(g: Graph, h: int, sweeps: int = 1, max_iter: int = -1, stream=None,
                         prune: bool = False):
    """The H-index iteration of Sec. 4 on the device.  sweeps = 1: synchronous orders
    (Algorithm 2); sweeps > 1: asynchronous updating by that many edge blocks per order;
    prune (sweeps = 1 only): the redundant-computation pruning of Lemma 4
    (htd_hindex_decompose_ex with HTD_HX_PRUNE).  Returns (truss = H + 2, H, stats dict) as
    int32 CUDA tensors of m entries."""
    torch = _torch()
    t = torch.empty(max(g.m, 1), dtype=torch.int32, device=g.device)
    hv = torch.empty(max(g.m, 1), dtype=torch.int32, device=g.device)
    st = _lib.HtdHindexStats()
    _lib.check(_lib.load().htd_hindex_decompose_ex(g.handle, int(h), int(sweeps), int(max_iter),
                                                   _lib.HTD_HX_PRUNE if prune else 0,
                                                   _ptr(t), _ptr(hv), ctypes.byref(st),
                                                   _stream_handle(stream)), "htd_hindex_decompose")
    return t[:g.m], hv[:g.m], st.as_dict()


class Server:
    """A served-decomposition loop (htd_server_*): requests are admitted by device memory as
    they arrive and run concurrently by worker threads; results come back on the host."""

    def __init__(self, workers: int = 4, budget_bytes: int = 0, flags: int = 0):
        h = ctypes.c_void_p()
        _lib.check(_lib.load().htd_server_create(int(workers), int(budget_bytes), int(flags),
                                                 ctypes.byref(h)), "htd_server_create")
        self._h = h

    def submit(self, n: int, src, dst, h: int) -> int:
        """Queues a decomposition of the raw pairs (numpy int32 arrays, copied); returns
        the request id."""
        src = np.ascontiguousarray(src, dtype=np.int32)
        dst = np.ascontiguousarray(dst, dtype=np.int32)
        if src.shape != dst.shape:
            raise ValueError("src and dst differ in length")
        rid = ctypes.c_int64()
        vp = lambda a: ctypes.c_void_p(a.ctypes.data) if a.size else None
        _lib.check(_lib.load().htd_server_submit(self._h, int(n), vp(src), vp(dst), src.size,
                                                 int(h), ctypes.byref(rid)), "htd_server_submit")
        return int(rid.value)

    def poll(self, rid: int) -> bool:
        done = ctypes.c_int32()
        _lib.check(_lib.load().htd_server_poll(self._h, int(rid), ctypes.byref(done)),
                   "htd_server_poll")
        return bool(done.value)

    def wait(self, rid: int, capacity: int):
        """Blocks until the request is done; returns (eu, ev, truss, info) as numpy arrays
        trimmed to the request's m edges (capacity >= m, e.g. its number of raw pairs)."""
        cap = max(1, int(capacity))
        eu = np.empty(cap, np.int32)
        ev = np.empty(cap, np.int32)
        t = np.empty(cap, np.int32)
        info = _lib.HtdRequestInfo()
        vp = lambda a: ctypes.c_void_p(a.ctypes.data)
        _lib.check(_lib.load().htd_server_wait(self._h, int(rid), vp(eu), vp(ev), vp(t), cap,
                                               ctypes.byref(info)), "htd_server_wait")
        m = int(info.m)
        return eu[:m], ev[:m], t[:m], info.as_dict()

    def info(self):
        st = _lib.HtdServerStats()
        _lib.check(_lib.load().htd_server_info(self._h, ctypes.byref(st)), "htd_server_info")
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.load().htd_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def htd_footprint_estimate(n: int, m_in: int, h: int, free_bytes: int) -> int:
    return int(_lib.load().htd_footprint_estimate(int(n), int(m_in), int(h), int(free_bytes)))


def htd_graph_free(g: Graph):
    g.free()
