"""CPU oracle for bitruss decomposition -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  It shares no
code with the CUDA library and the CUDA library never calls it.

The arithmetic lives in ``oracle.c`` (plain C, OpenMP over edges for the
read-only support count, single-threaded peeling):

* ``support``          -- butterfly support of every edge by direct
  enumeration (Defs. 2-3, Section II).
* ``bitruss``          -- initial supports and bitruss numbers by the
  one-edge-at-a-time bottom-up peeling of Alg. 1 (BiT-BS, Section III).
* ``support_sampled``  -- supports of selected edges only.
* ``support_anchored`` -- supports from the butterflies whose anchor (the
  vertex of highest priority, Def. 7) has a priority rank in a given range;
  by Lemma 3 the ranges of a partition sum to the supports.
* ``local_check``      -- per selected edge, the count of butterflies whose
  other edges all have phi >= phi(e), and the local h-value (the fixpoint
  property every correct phi satisfies; follows from Defs. 4-5).
* ``k_bitruss``        -- the k-bitruss H_k straight from Def. 4: delete every
  edge with fewer than k butterflies in the remaining graph until none is
  left (Python loop over ``support``).
* ``hierarchy``        -- edges ordered by bitruss number, largest first, ties
  in input order (numpy stable sort), so each H_k is a prefix.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_ERR = {-1: "allocation failed", -2: "vertex or edge id out of range", -3: "duplicate edge"}


def build() -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` beside it (gcc, OpenMP)."""
    if os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            U64 = ctypes.c_uint64
            U32 = ctypes.c_uint32
            lib.oracle_support.argtypes = [P, U64, U32, U32, P]
            lib.oracle_support_sampled.argtypes = [P, U64, U32, U32, P, U64, P]
            lib.oracle_bitruss.argtypes = [P, U64, U32, U32, P, P]
            lib.oracle_local_check.argtypes = [P, U64, U32, U32, P, P, U64, P, P]
            lib.oracle_support_anchored.argtypes = [P, U64, U32, U32, ctypes.c_int, U64, U64, P]
            lib.oracle_threads.restype = ctypes.c_int
            for f in (lib.oracle_support, lib.oracle_support_sampled, lib.oracle_bitruss,
                      lib.oracle_local_check, lib.oracle_support_anchored):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _edges(edges) -> np.ndarray:
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    return e


def _check(rc: int):
    if rc != 0:
        raise ValueError(f"oracle: {_ERR.get(rc, rc)}")


def threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().oracle_threads())


def support(edges, nU: int, nL: int) -> np.ndarray:
    e = _edges(edges)
    out = np.empty(e.shape[0], dtype=np.uint64)
    _check(_load().oracle_support(e.ctypes.data, e.shape[0], nU, nL, out.ctypes.data))
    return out


def support_sampled(edges, nU: int, nL: int, which) -> np.ndarray:
    e = _edges(edges)
    w = np.ascontiguousarray(np.asarray(which, dtype=np.uint64))
    out = np.empty(w.shape[0], dtype=np.uint64)
    _check(_load().oracle_support_sampled(e.ctypes.data, e.shape[0], nU, nL, w.ctypes.data,
                                          w.shape[0], out.ctypes.data))
    return out


def support_anchored(edges, nU: int, nL: int, rank_lo: int, rank_hi: int,
                     lower_first: bool = False) -> np.ndarray:
    """Supports counting only butterflies anchored at priority ranks in
    [rank_lo, rank_hi): the anchor is the butterfly's vertex of highest
    priority (Def. 7, degree then global id; global ids as in Section II, or
    the Fig. 6 reading with lower_first).  Rank 0 is the lowest priority."""
    e = _edges(edges)
    out = np.empty(e.shape[0], dtype=np.uint64)
    _check(_load().oracle_support_anchored(e.ctypes.data, e.shape[0], nU, nL, 1 if lower_first else 0,
                                           rank_lo, rank_hi, out.ctypes.data))
    return out


def bitruss(edges, nU: int, nL: int):
    """Return (support u64[m], phi u64[m]) by Alg. 1 peeling."""
    e = _edges(edges)
    sup = np.empty(e.shape[0], dtype=np.uint64)
    phi = np.empty(e.shape[0], dtype=np.uint64)
    _check(_load().oracle_bitruss(e.ctypes.data, e.shape[0], nU, nL, sup.ctypes.data,
                                  phi.ctypes.data))
    return sup, phi


def local_check(edges, nU: int, nL: int, phi, which):
    """Return (count_at_phi u64[q], h u64[q]) for the queried edges."""
    e = _edges(edges)
    p = np.ascontiguousarray(np.asarray(phi, dtype=np.uint32))
    w = np.ascontiguousarray(np.asarray(which, dtype=np.uint64))
    cnt = np.empty(w.shape[0], dtype=np.uint64)
    h = np.empty(w.shape[0], dtype=np.uint64)
    _check(_load().oracle_local_check(e.ctypes.data, e.shape[0], nU, nL, p.ctypes.data,
                                      w.ctypes.data, w.shape[0], cnt.ctypes.data, h.ctypes.data))
    return cnt, h


def k_bitruss(edges, nU: int, nL: int, k: int) -> np.ndarray:
    """Bool mask of the edges of the k-bitruss H_k (Def. 4, Section II): the
    maximal subgraph in which every edge lies in >= k of its butterflies.
    Deleting all edges below k and recounting until nothing changes reaches it
    (a deleted edge is in no subgraph with the property, as deletions only
    lower supports)."""
    e = _edges(edges)
    keep = np.ones(e.shape[0], dtype=bool)
    while True:
        idx = np.flatnonzero(keep)
        if idx.size == 0:
            return keep
        s = support(e[idx], nU, nL)
        low = s < np.uint64(k)
        if not low.any():
            return keep
        keep[idx[low]] = False


def hierarchy(phi) -> np.ndarray:
    """Edge ids by bitruss number, largest first, equal phi in ascending id.
    With H_k = {e : phi_e >= k} (Defs. 4-5; the k-bitrusses are nested) every
    H_k is the prefix of length |{e : phi_e >= k}|."""
    p = np.asarray(phi).astype(np.int64)
    return np.argsort(-p, kind="stable").astype(np.uint32)
