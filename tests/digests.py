"""Comparison of GPU outputs with the CPU oracle's stored digests (SHA-256 of
the oracle's full support and bitruss-number arrays, written offline by
tests/golden/make_oracle_digests.py, which calls only the oracle and the input
generator)."""
import hashlib
import json
import os

import numpy as np


def oracle_digest(name):
    """The CPU oracle's digests of a workload too large to rerun here, written
    by tests/golden/make_oracle_digests.py (oracle and input generator only)."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_digests.json")) as f:
        return json.load(f)[name]


def assert_matches_digest(g, sup, phi, ref):
    """Every edge's support and bitruss number equal the oracle's: the SHA-256
    of the full uint64 / uint32 arrays in input order must match."""
    assert (g.nU, g.nL, g.m) == (ref["nU"], ref["nL"], ref["m"])
    # the generator must have produced the very graph the oracle decomposed
    assert hashlib.sha256(g.edges.astype(np.int32).tobytes()).hexdigest() == ref["edges_sha256"]
    assert int(sup.sum()) == ref["support_sum"]
    vals, cnts = np.unique(phi, return_counts=True)
    got_hist = [[int(v), int(c)] for v, c in zip(vals, cnts)]
    assert got_hist == ref["phi_hist"], "phi histogram differs from the oracle's"
    assert hashlib.sha256(np.ascontiguousarray(sup, dtype=np.uint64).tobytes()).hexdigest() == \
        ref["support_sha256"]
    assert hashlib.sha256(np.ascontiguousarray(phi, dtype=np.uint32).tobytes()).hexdigest() == \
        ref["phi_sha256"]
