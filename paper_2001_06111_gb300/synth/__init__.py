"""Seeded synthetic bipartite workloads (input generation only).

The generator is written in C (``chunglu.c``) and holds none of the bitruss
method's arithmetic; the CPU oracle harness and the GPU harness both draw
their inputs from it.  The workloads stand in for the skewed real-world
KONECT graphs of the paper's Table 3 (Section VI), which are not available:

* ``small``   -- |U|=2,000, |L|=1,500, m=20,000, exponents 2.2 / 2.5, seed 1
* ``medium``  -- |U|=200,000, |L|=80,000, m=2,000,000, exponents 2.1 / 2.4,
  degree cap 20,000, seed 2
* ``large``   -- |U|=2,000,000, |L|=500,000, m=30,000,000, exponents 2.0 / 2.3,
  200 planted bicliques with sides uniform in [50,300] at density 0.9 placed
  first, then Chung-Lu edges until 30,000,000 distinct edges in total, seed 3
* ``batch(i)`` -- graph i of a 4,096-graph batch: m log-uniform in
  [100, 200,000], |U|=ceil(m/8), |L|=ceil(m/12), exponents uniform in
  [2.0, 2.6], seed SplitMix64(4*2^32 + i)

Edge lists are int32 arrays of shape (m, 2): column 0 is the upper vertex in
[0, |U|), column 1 the lower vertex in [0, |L|).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chunglu.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build() -> str:
    """Compile the generator into ``libsynth.so`` beside its source."""
    if os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_chunglu.restype = ctypes.c_int
            lib.synth_chunglu.argtypes = [
                ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                ctypes.c_uint64, ctypes.c_void_p]
            lib.synth_splitmix.restype = ctypes.c_uint64
            lib.synth_splitmix.argtypes = [ctypes.c_uint64]
            lib.synth_unit_from.restype = ctypes.c_double
            lib.synth_unit_from.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
            _lib = lib
    return _lib


@dataclass
class Graph:
    edges: np.ndarray  # int32 (m, 2)
    nU: int
    nL: int
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.edges.shape[0])


def chunglu(nU: int, nL: int, m: int, gammaU: float, gammaL: float, seed: int, cap: int = 0,
            nplant: int = 0, plant_lo: int = 0, plant_hi: int = 0, plant_p: float = 0.0,
            name: str = "") -> Graph:
    lib = _load()
    out = np.empty((m, 2), dtype=np.int32)
    rc = lib.synth_chunglu(nU, nL, m, gammaU, gammaL, cap, nplant, plant_lo, plant_hi, plant_p,
                           seed & (2**64 - 1), out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"synth_chunglu failed with code {rc} for {name or (nU, nL, m)}")
    return Graph(out, nU, nL, name)


def small() -> Graph:
    return chunglu(2000, 1500, 20000, 2.2, 2.5, seed=1, name="chunglu-2k-1.5k-20k")


def medium() -> Graph:
    return chunglu(200000, 80000, 2000000, 2.1, 2.4, seed=2, cap=20000,
                   name="chunglu-200k-80k-2M-cap20k")


def large() -> Graph:
    return chunglu(2000000, 500000, 30000000, 2.0, 2.3, seed=3, nplant=200, plant_lo=50,
                   plant_hi=300, plant_p=0.9, name="chunglu-2M-500k-30M-planted200")


def splitmix(x: int) -> int:
    return int(_load().synth_splitmix(x & (2**64 - 1)))


def batch_params(i: int, lo: int = 100, hi: int = 200000):
    """Size and exponents of graph i of the batched workload."""
    seed = splitmix(4 * 2**32 + i)
    lib = _load()
    x0 = lib.synth_unit_from(seed, 0)
    x1 = lib.synth_unit_from(seed, 1)
    x2 = lib.synth_unit_from(seed, 2)
    m = int(round(math.exp(math.log(lo) + x0 * (math.log(hi) - math.log(lo)))))
    m = max(lo, min(hi, m))
    nU = (m + 7) // 8
    nL = (m + 11) // 12
    return dict(m=m, nU=nU, nL=nL, gammaU=2.0 + 0.6 * x1, gammaL=2.0 + 0.6 * x2, seed=seed)


def batch_graph(i: int, lo: int = 100, hi: int = 200000) -> Graph:
    p = batch_params(i, lo, hi)
    return chunglu(p["nU"], p["nL"], p["m"], p["gammaU"], p["gammaL"], seed=p["seed"] ^ 0x5DEECE66D,
                   name=f"batch-{i}")


def random_tiny(seed: int, nU: int, nL: int, m: int) -> Graph:
    """Uniform random simple bipartite graph (numpy PCG64), for small parity cases."""
    rng = np.random.default_rng(seed)
    m = min(m, nU * nL)
    keys = rng.choice(nU * nL, size=m, replace=False)
    edges = np.stack([keys // nL, keys % nL], axis=1).astype(np.int32)
    return Graph(edges, nU, nL, f"uniform-{seed}")


def vertex_sample(g: Graph, frac: float, seed: int) -> Graph:
    """Vertex-induced subgraph on a seeded random fraction of both layers
    (the sampling used for the paper's scalability study, Section VI)."""
    rng = np.random.default_rng(seed)
    ku = rng.random(g.nU) < frac
    kl = rng.random(g.nL) < frac
    keep = ku[g.edges[:, 0]] & kl[g.edges[:, 1]]
    e = g.edges[keep]
    mu = np.cumsum(ku) - 1
    ml = np.cumsum(kl) - 1
    e2 = np.stack([mu[e[:, 0]], ml[e[:, 1]]], axis=1).astype(np.int32)
    return Graph(e2, int(ku.sum()), int(kl.sum()), f"{g.name}-sample{frac}")
