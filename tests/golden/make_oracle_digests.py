"""Writes ``oracle_digests.json``: SHA-256 digests of the CPU oracle's exact
supports (uint64) and bitruss numbers (uint32) on workloads too large for the
oracle to run inside the GPU test suite.

Only the oracle (``oracle.bitruss``: direct butterfly enumeration and the
one-edge-at-a-time peeling of Alg. 1) and the seeded input generator are
called; nothing here touches the CUDA library.  The GPU tests recompute the
same digests from the library's outputs and compare them, which is an
element-by-element comparison of every edge.

Entries:

* ``medium``        -- the 2,000,000-edge Chung-Lu workload at full size;
* ``large-sample``  -- a seeded vertex-induced sample of the 30,000,000-edge
  planted workload (the sampling of Section VI's scalability study), the
  largest the oracle finishes in about half an hour on 8 cores.  The full
  30M-edge graph is beyond the oracle (its peeling grows about as m^2.1).

Run (CPU only, tens of minutes):
    python tests/golden/make_oracle_digests.py [medium] [large-sample]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2001_06111_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "oracle_digests.json")

# vertex fraction and seed of the 30M-edge workload's sample
LARGE_SAMPLE = dict(frac=0.21, seed=5)


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def workload(name: str) -> synth.Graph:
    if name == "medium":
        return synth.medium()
    if name == "large-sample":
        return synth.vertex_sample(synth.large(), LARGE_SAMPLE["frac"], LARGE_SAMPLE["seed"])
    raise ValueError(name)


def digest_entry(name: str) -> dict:
    g = workload(name)
    t0 = time.time()
    sup, phi = oracle.bitruss(g.edges, g.nU, g.nL)
    dt = time.time() - t0
    assert int(phi.max(initial=0)) < 2**32
    phi32 = phi.astype(np.uint32)
    vals, cnts = np.unique(phi32, return_counts=True)
    return {
        "nU": g.nU, "nL": g.nL, "m": g.m,
        "edges_sha256": sha(g.edges.astype(np.int32)),
        "support_sha256": sha(sup.astype(np.uint64)),
        "phi_sha256": sha(phi32),
        "support_sum": int(sup.sum()),
        "phi_max": int(phi32.max(initial=0)),
        "phi_hist": [[int(v), int(c)] for v, c in zip(vals, cnts)],
        "oracle_seconds": round(dt, 1), "oracle_threads": oracle.threads(),
        **({"sample": LARGE_SAMPLE} if name == "large-sample" else {}),
    }


def main(argv):
    names = argv or ["medium", "large-sample"]
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names:
        data[name] = digest_entry(name)
        print(name, data[name]["m"], "edges,", data[name]["oracle_seconds"], "s", flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])
