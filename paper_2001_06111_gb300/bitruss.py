"""Thin ctypes binding of ``libbitruss.so`` (C ABI in include/bitruss.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Host inputs are numpy arrays; device inputs are CUDA torch tensors
(their pointers are passed with ``BT_DEVICE_PTRS``).  Torch is used only to
hold device memory and to name a stream.  If the library has not been built
(or a symbol is missing) loading fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbitruss.so")

BT_OK = 0
BT_ERR_ARG = 1
BT_ERR_RANGE = 2
BT_ERR_DUP = 3
BT_ERR_NOMEM = 4
BT_ERR_OVERFLOW = 5
BT_ERR_NOCONVERGE = 6
BT_ERR_CUDA = 7
BT_ERR_STATE = 8
BT_ERR_TOO_LARGE = 9
BT_ERR_CANCELLED = 10
BT_DEVICE_PTRS = 0x1
BT_TIE_LOWER_FIRST = 0x2
BT_PC_RECOUNT = 0x4  # bt_decompose_progressive: Alg. 7's candidate extraction

EXPORTED = ("bt_create", "bt_destroy", "bt_last_error", "bt_count_support", "bt_build_index",
            "bt_index_export", "bt_decompose", "bt_estimate_bytes", "bt_profile_enable",
            "bt_profile_read", "bt_count_support_static", "bt_decompose_batch",
            "bt_server_create", "bt_server_destroy", "bt_server_submit", "bt_server_poll",
            "bt_server_stats_read", "bt_decompose_progressive", "bt_hierarchy", "bt_k_bitruss",
            "bt_set_limits", "bt_count_support_part", "bt_server_cancel_queued")


class BitrussError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bitruss error {code}: {msg}")
        self.code = code


class IndexStats(ctypes.Structure):
    _fields_ = [("n_wedges", ctypes.c_uint64), ("n_bloom_wedges", ctypes.c_uint64),
                ("n_blooms", ctypes.c_uint64), ("n_butterflies", ctypes.c_uint64),
                ("index_bytes", ctypes.c_uint64)]


class BloomRec(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("first_pair", ctypes.c_uint32)]


class PeelStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_uint64), ("levels", ctypes.c_uint64),
                ("support_updates", ctypes.c_uint64), ("phi_max", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class Profile(ctypes.Structure):
    _fields_ = [("csr_ms", ctypes.c_float), ("count_ms", ctypes.c_float),
                ("emit_ms", ctypes.c_float), ("peel_ms", ctypes.c_float),
                ("total_ms", ctypes.c_float), ("reserved", ctypes.c_uint32),
                ("launches", ctypes.c_uint64), ("n_edges", ctypes.c_uint64),
                ("n_vertices", ctypes.c_uint64), ("n_wedges", ctypes.c_uint64),
                ("n_bloom_wedges", ctypes.c_uint64), ("n_blooms", ctypes.c_uint64),
                ("rounds", ctypes.c_uint64), ("levels", ctypes.c_uint64),
                ("support_updates", ctypes.c_uint64), ("pair_slots", ctypes.c_uint64),
                ("link_visits", ctypes.c_uint64), ("scanned", ctypes.c_uint64)]


class Graph(ctypes.Structure):
    _fields_ = [("edges", ctypes.c_void_p), ("m", ctypes.c_uint64), ("nU", ctypes.c_uint32),
                ("nL", ctypes.c_uint32), ("support_out", ctypes.c_void_p),
                ("phi_out", ctypes.c_void_p)]


class Limits(ctypes.Structure):
    _fields_ = [("peel_round_limit", ctypes.c_uint64), ("barrier_timeout_ns", ctypes.c_uint64),
                ("hold_barrier", ctypes.c_uint64), ("fail_alloc_at", ctypes.c_uint64),
                ("join_cap", ctypes.c_uint32), ("block_links", ctypes.c_uint32)]


class Tune(ctypes.Structure):
    _fields_ = [("max_edges_per_launch", ctypes.c_uint64), ("count_threads", ctypes.c_uint32),
                ("peel_item", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 2)]


class BatchStats(ctypes.Structure):
    _fields_ = [("graphs", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("edges", ctypes.c_uint64), ("wedges", ctypes.c_uint64),
                ("rounds", ctypes.c_uint64), ("levels", ctypes.c_uint64),
                ("support_updates", ctypes.c_uint64), ("count_threads", ctypes.c_uint32),
                ("peel_item", ctypes.c_uint32), ("tuned", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class PcStats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_uint64), ("rounds", ctypes.c_uint64),
                ("levels", ctypes.c_uint64), ("support_updates", ctypes.c_uint64),
                ("candidate_edges", ctypes.c_uint64), ("wedges", ctypes.c_uint64),
                ("k_max", ctypes.c_uint64), ("alpha", ctypes.c_uint64),
                ("index_bytes_max", ctypes.c_uint64), ("links", ctypes.c_uint64),
                ("dropped_edges", ctypes.c_uint64)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", ctypes.c_uint64), ("workers", ctypes.c_uint32),
                ("max_batch_graphs", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("large_edges", ctypes.c_uint32), ("large_batch", ctypes.c_uint32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("status", ctypes.c_int),
                ("queue_seconds", ctypes.c_double), ("latency_seconds", ctypes.c_double),
                ("admitted_bytes", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("queued", ctypes.c_uint64), ("max_batch_graphs", ctypes.c_uint64),
                ("in_flight_bytes", ctypes.c_uint64), ("peak_in_flight_bytes", ctypes.c_uint64),
                ("edges", ctypes.c_uint64), ("busy_seconds", ctypes.c_double)]


def _as_dict(s: ctypes.Structure) -> dict:
    out = {}
    for f, t in s._fields_:
        if f == "reserved":
            continue
        v = getattr(s, f)
        out[f] = float(v) if t in (ctypes.c_float, ctypes.c_double) else int(v)
    return out


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (build it first with ``paper_2001_06111_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"libbitruss.so not built at {path}; run paper_2001_06111_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name in EXPORTED:
            if not hasattr(lib, name):
                raise ImportError(f"libbitruss.so does not export {name}")
        P, U64, U32, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        lib.bt_create.argtypes = [ctypes.POINTER(P), I, P]
        lib.bt_destroy.argtypes = [P]
        lib.bt_last_error.argtypes = [P]
        lib.bt_last_error.restype = ctypes.c_char_p
        lib.bt_count_support.argtypes = [P, P, U64, U32, U32, P, U32]
        lib.bt_build_index.argtypes = [P, P, U64, U32, U32, ctypes.POINTER(IndexStats), U32]
        lib.bt_index_export.argtypes = [P, P, P, P]
        lib.bt_decompose.argtypes = [P, P, U64, U32, U32, P, P, ctypes.POINTER(PeelStats), U32]
        lib.bt_count_support_static.argtypes = [P, U64, U32, U32, P, U32, P]
        lib.bt_hierarchy.argtypes = [P, P, U64, P, P, U32]
        lib.bt_k_bitruss.argtypes = [P, P, U64, U32, P, ctypes.POINTER(U64), U32]
        lib.bt_decompose_batch.argtypes = [P, ctypes.POINTER(Graph), U32, ctypes.POINTER(Tune),
                                           ctypes.POINTER(BatchStats), U32]
        lib.bt_server_create.argtypes = [ctypes.POINTER(P), I, ctypes.POINTER(ServerConfig)]
        lib.bt_server_destroy.argtypes = [P]
        lib.bt_server_submit.argtypes = [P, ctypes.POINTER(Graph), ctypes.POINTER(U64)]
        lib.bt_server_poll.argtypes = [P, U64, I, ctypes.POINTER(RequestInfo)]
        lib.bt_server_stats_read.argtypes = [P, ctypes.POINTER(ServerStats)]
        lib.bt_server_cancel_queued.argtypes = [P, ctypes.POINTER(U64)]
        lib.bt_decompose_progressive.argtypes = [P, P, U64, U32, U32, ctypes.c_double, P, P,
                                                 ctypes.POINTER(PcStats), U32]
        lib.bt_profile_enable.argtypes = [P, I]
        lib.bt_set_limits.argtypes = [P, ctypes.POINTER(Limits)]
        lib.bt_count_support_part.argtypes = [P, P, U64, U32, U32, U32, U32, P, ctypes.POINTER(U32),
                                              ctypes.POINTER(U32), U32]
        lib.bt_profile_read.argtypes = [P, ctypes.POINTER(Profile)]
        lib.bt_estimate_bytes.argtypes = [P, U64, U32, U32, U32, ctypes.POINTER(U64),
                                          ctypes.POINTER(U64)]
        for name in EXPORTED:
            if name != "bt_last_error":
                getattr(lib, name).restype = I
        _lib = lib
        return lib


class Handle:
    """Owns a ``bt_handle*`` (device, stream and device-resident index)."""

    def __init__(self, ptr: int, device: int):
        self.ptr = ptr
        self.device = device

    def close(self):
        if self.ptr:
            load().bt_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check(h, rc: int):
    if rc != BT_OK:
        msg = load().bt_last_error(h.ptr if h is not None else None)
        raise BitrussError(rc, msg.decode() if msg else "")


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _edges_arg(edges):
    """(pointer, m, flags, keepalive) for a numpy (host) or torch (device) edge list."""
    if _is_torch(edges):
        if not edges.is_cuda:
            edges = edges.numpy()
        else:
            import torch
            assert edges.dtype == torch.int32 and edges.is_contiguous() and edges.dim() == 2
            return edges.data_ptr(), int(edges.shape[0]), BT_DEVICE_PTRS, edges
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    return e.ctypes.data, int(e.shape[0]), 0, e


def _out(like_device, m, dtype_np, torch_dtype, given):
    if given is not None:
        ptr = given.data_ptr() if _is_torch(given) else given.ctypes.data
        return given, ptr
    if like_device is not None:
        import torch
        t = torch.empty(m, dtype=torch_dtype, device=like_device.device)
        return t, t.data_ptr()
    a = np.empty(m, dtype=dtype_np)
    return a, a.ctypes.data


def bt_create(device: int = 0, stream=None) -> Handle:
    lib = load()
    p = ctypes.c_void_p()
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    rc = lib.bt_create(ctypes.byref(p), device, s)
    if rc != BT_OK:
        raise BitrussError(rc, f"bt_create(device={device}) failed")
    return Handle(p.value, device)


def bt_count_support(h: Handle, edges, nU: int, nL: int, support_out=None, flags: int = 0):
    ptr, m, f, keep = _edges_arg(edges)
    import_dev = keep if f & BT_DEVICE_PTRS else None
    sup, sptr = _out(import_dev, m, np.uint64, _torch_dtype("uint64"), support_out)
    _check(h, load().bt_count_support(h.ptr, ptr, m, nU, nL, sptr, flags | f))
    return sup


def bt_count_support_part(h: Handle, edges, nU: int, nL: int, part: int, nparts: int, support_out=None,
                          flags: int = 0):
    """One part of a counting shard: the supports contributed by the
    butterflies anchored in part `part` of `nparts` wedge-balanced priority-rank
    ranges.  Returns (support u64[m], rank_lo, rank_hi); the parts of a graph
    add up to bt_count_support's result."""
    ptr, m, f, keep = _edges_arg(edges)
    dev = keep if f & BT_DEVICE_PTRS else None
    sup, sptr = _out(dev, m, np.uint64, _torch_dtype("uint64"), support_out)
    lo, hi = ctypes.c_uint32(), ctypes.c_uint32()
    _check(h, load().bt_count_support_part(h.ptr, ptr, m, nU, nL, part, nparts, sptr, ctypes.byref(lo),
                                           ctypes.byref(hi), flags | f))
    return sup, int(lo.value), int(hi.value)


def _phi_arg(phi):
    """(pointer, m, flags, keepalive) for a u32 phi array: numpy (host) or CUDA torch tensor (device)."""
    if _is_torch(phi):
        import torch
        assert phi.dtype == _torch_dtype("uint32") and phi.is_contiguous() and phi.dim() == 1
        return (phi.data_ptr() if phi.numel() else None), phi.numel(), (BT_DEVICE_PTRS if phi.is_cuda else 0), phi
    a = np.ascontiguousarray(phi, dtype=np.uint32)
    return (a.ctypes.data if a.size else None), a.size, 0, a


def bt_hierarchy(h: Handle, phi, want_phi: bool = True):
    """Edges by bitruss number, largest first (ties in input order): every
    k-bitruss H_k is a prefix.  Returns (order u32[m], phi_sorted u32[m] or None)."""
    ptr, m, f, keep = _phi_arg(phi)
    dev = keep if f & BT_DEVICE_PTRS else None
    order, optr = _out(dev, m, np.uint32, _torch_dtype("uint32"), None)
    ps, pptr = (None, None)
    if want_phi:
        ps, pptr = _out(dev, m, np.uint32, _torch_dtype("uint32"), None)
    _check(h, load().bt_hierarchy(h.ptr, ptr, m, optr, pptr, f))
    return order, ps


def bt_k_bitruss(h: Handle, phi, k: int):
    """Indices (ascending) of the edges of the k-bitruss H_k, i.e. phi >= k."""
    ptr, m, f, keep = _phi_arg(phi)
    dev = keep if f & BT_DEVICE_PTRS else None
    out, optr = _out(dev, m, np.uint32, _torch_dtype("uint32"), None)
    n = ctypes.c_uint64(0)
    _check(h, load().bt_k_bitruss(h.ptr, ptr, m, k, optr, ctypes.byref(n), f))
    return out[: n.value]


def bt_build_index(h: Handle, edges, nU: int, nL: int, flags: int = 0) -> dict:
    ptr, m, f, keep = _edges_arg(edges)
    st = IndexStats()
    _check(h, load().bt_build_index(h.ptr, ptr, m, nU, nL, ctypes.byref(st), flags | f))
    return _as_dict(st)


def bt_index_export(h: Handle, stats: dict, m: int):
    """Return (bloom k u32[nb], bloom first pair u32[nb], pairs u32[w2,2], links per edge u32[m])."""
    nb, w2 = stats["n_blooms"], stats["n_bloom_wedges"]
    blooms = (BloomRec * max(nb, 1))()
    pairs = np.empty((max(w2, 1), 2), dtype=np.uint32)
    deg = np.empty(max(m, 1), dtype=np.uint32)
    _check(h, load().bt_index_export(h.ptr, ctypes.addressof(blooms), pairs.ctypes.data,
                                     deg.ctypes.data))
    k = np.array([blooms[i].k for i in range(nb)], dtype=np.uint32)
    first = np.array([blooms[i].first_pair for i in range(nb)], dtype=np.uint32)
    return k, first, pairs[:w2], deg[:m]


def bt_decompose(h: Handle, edges, nU: int, nL: int, support_out=None, phi_out=None,
                 flags: int = 0, want_support: bool = True):
    """Return (support u64[m] or None, phi u32[m], stats dict)."""
    ptr, m, f, keep = _edges_arg(edges)
    dev = keep if f & BT_DEVICE_PTRS else None
    sup, sptr = (None, None)
    if want_support or support_out is not None:
        sup, sptr = _out(dev, m, np.uint64, _torch_dtype("uint64"), support_out)
    phi, pptr = _out(dev, m, np.uint32, _torch_dtype("uint32"), phi_out)
    st = PeelStats()
    _check(h, load().bt_decompose(h.ptr, ptr, m, nU, nL, sptr, pptr, ctypes.byref(st), flags | f))
    return sup, phi, _as_dict(st)


def bt_count_support_static(d_edges, nU: int, nL: int, d_support_out, flags: int = 0,
                            stream=None) -> None:
    """Allocation-free support count on device buffers (CUDA torch tensors):
    scratch comes from a fixed array inside the library, for callers that
    cannot allocate device memory.  Raises BitrussError on failure."""
    import torch
    if not (isinstance(d_edges, torch.Tensor) and d_edges.is_cuda and d_edges.dtype == torch.int32
            and d_edges.dim() == 2 and d_edges.shape[1] == 2 and d_edges.is_contiguous()):
        raise ValueError("d_edges must be a contiguous CUDA int32 tensor of shape (m, 2)")
    m = int(d_edges.shape[0])
    if not (isinstance(d_support_out, torch.Tensor) and d_support_out.is_cuda
            and d_support_out.element_size() == 8 and d_support_out.is_contiguous()
            and d_support_out.numel() >= m and d_support_out.device == d_edges.device):
        raise ValueError("d_support_out must be a contiguous 64-bit CUDA tensor with at least m "
                         "entries on the device of d_edges")
    with torch.cuda.device(d_edges.device):
        if stream is None:
            stream = torch.cuda.current_stream()
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        rc = load().bt_count_support_static(d_edges.data_ptr(), m, nU, nL, d_support_out.data_ptr(),
                                            flags, s)
    if rc != BT_OK:
        raise BitrussError(rc, "bt_count_support_static failed")


def bt_decompose_batch(h: Handle, graphs, flags: int = 0, max_edges_per_launch: int = 0,
                       want_support: bool = True, count_threads: int = 0, peel_item: int = 0):
    """Decompose a list of graphs, each given as (edges, nU, nL) with numpy
    (host) or CUDA torch (device) edge lists; returns ([(support, phi)], stats)."""
    n = len(graphs)
    arr = (Graph * max(n, 1))()
    keep, outs = [], []
    dev_flag = 0
    for i, (edges, nU, nL) in enumerate(graphs):
        ptr, m, f, k = _edges_arg(edges)
        dev_flag |= f
        keep.append(k)
        dev = k if f & BT_DEVICE_PTRS else None
        sup, sptr = (None, None)
        if want_support:
            sup, sptr = _out(dev, m, np.uint64, _torch_dtype("uint64"), None)
        phi, pptr = _out(dev, m, np.uint32, _torch_dtype("uint32"), None)
        arr[i] = Graph(ptr, m, nU, nL, sptr, pptr)
        outs.append((sup, phi))
    tune = Tune(max_edges_per_launch, count_threads, peel_item)
    st = BatchStats()
    _check(h, load().bt_decompose_batch(h.ptr, arr, n, ctypes.byref(tune), ctypes.byref(st),
                                        flags | dev_flag))
    return outs, _as_dict(st)


class Server:
    """Continuous-batching request loop (bt_server_*).  Host buffers only; the
    request keeps its edge array and outputs alive until it completes."""

    def __init__(self, device: int = 0, memory_budget_bytes: int = 0, workers: int = 0,
                 max_batch_graphs: int = 0, flags: int = 0, large_edges: int = 0, large_batch: int = 0):
        lib = load()
        cfg = ServerConfig(memory_budget_bytes, workers, max_batch_graphs, flags, large_edges, large_batch)
        p = ctypes.c_void_p()
        rc = lib.bt_server_create(ctypes.byref(p), device, ctypes.byref(cfg))
        if rc != BT_OK:
            raise BitrussError(rc, "bt_server_create failed")
        self.ptr = p.value
        self._live = {}

    def submit(self, edges, nU: int, nL: int, want_support: bool = False) -> int:
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        m = e.shape[0]
        sup = np.empty(m, dtype=np.uint64) if want_support else None
        phi = np.empty(m, dtype=np.uint32)
        g = Graph(e.ctypes.data, m, nU, nL, sup.ctypes.data if sup is not None else None,
                  phi.ctypes.data)
        rid = ctypes.c_uint64()
        rc = load().bt_server_submit(self.ptr, ctypes.byref(g), ctypes.byref(rid))
        if rc != BT_OK:
            raise BitrussError(rc, "bt_server_submit failed")
        self._live[rid.value] = (e, sup, phi)
        return rid.value

    def poll(self, rid: int, wait: bool = False):
        """Return (info dict, (support, phi) or None while pending)."""
        info = RequestInfo()
        rc = load().bt_server_poll(self.ptr, rid, 1 if wait else 0, ctypes.byref(info))
        if rc != BT_OK:
            raise BitrussError(rc, "bt_server_poll failed")
        d = _as_dict(info)
        if d["done"]:
            _, sup, phi = self._live.pop(rid)
            return d, (sup, phi)
        return d, None

    def cancel_queued(self) -> int:
        """Cancel every request still waiting in the queue; returns how many."""
        n = ctypes.c_uint64()
        rc = load().bt_server_cancel_queued(self.ptr, ctypes.byref(n))
        if rc != BT_OK:
            raise BitrussError(rc, "bt_server_cancel_queued failed")
        return int(n.value)

    def stats(self) -> dict:
        st = ServerStats()
        load().bt_server_stats_read(self.ptr, ctypes.byref(st))
        return _as_dict(st)

    def close(self):
        if self.ptr:
            load().bt_server_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def bt_set_limits(h: Handle, peel_round_limit: int = 0, barrier_timeout_ns: int = 0,
                  hold_barrier: int = 0, fail_alloc_at: int = 0, join_cap: int = 0,
                  block_links: int = 0) -> None:
    """Diagnostic limits and host-side fault injection for later calls on h
    (all zero: the defaults).  See bt_set_limits in include/bitruss.h."""
    lim = Limits(peel_round_limit, barrier_timeout_ns, hold_barrier, fail_alloc_at, join_cap, block_links)
    _check(h, load().bt_set_limits(h.ptr, ctypes.byref(lim)))


def bt_profile_enable(h: Handle, on: bool = True):
    _check(h, load().bt_profile_enable(h.ptr, 1 if on else 0))


def bt_profile_read(h: Handle) -> dict:
    p = Profile()
    _check(h, load().bt_profile_read(h.ptr, ctypes.byref(p)))
    return _as_dict(p)


def bt_decompose_progressive(h: Handle, edges, nU: int, nL: int, tau: float = 0.1,
                             support_out=None, phi_out=None, flags: int = 0, want_support: bool = True):
    """Progressive compression (BiT-PC); returns (support or None, phi, stats).
    flags may add BT_PC_RECOUNT (Alg. 7's extraction: supports recounted on
    each candidate subgraph, candidates below eps dropped before indexing)."""
    ptr, m, f, keep = _edges_arg(edges)
    dev = keep if f & BT_DEVICE_PTRS else None
    sup, sptr = (None, None)
    if want_support or support_out is not None:
        sup, sptr = _out(dev, m, np.uint64, _torch_dtype("uint64"), support_out)
    phi, pptr = _out(dev, m, np.uint32, _torch_dtype("uint32"), phi_out)
    st = PcStats()
    _check(h, load().bt_decompose_progressive(h.ptr, ptr, m, nU, nL, tau, sptr, pptr,
                                              ctypes.byref(st), flags | f))
    return sup, phi, _as_dict(st)


def bt_estimate_bytes(edges, nU: int, nL: int, flags: int = 0):
    """Return (device bytes needed, priority-obeyed wedges) for a host edge list."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    b = ctypes.c_uint64()
    w = ctypes.c_uint64()
    rc = load().bt_estimate_bytes(e.ctypes.data, e.shape[0], nU, nL, flags, ctypes.byref(b),
                                  ctypes.byref(w))
    if rc != BT_OK:
        raise BitrussError(rc, "bt_estimate_bytes failed")
    return int(b.value), int(w.value)


def _torch_dtype(name):
    try:
        import torch
    except ImportError:  # host-only use
        return None
    return {"uint64": getattr(torch, "uint64", torch.int64),
            "uint32": getattr(torch, "uint32", torch.int32)}[name]
