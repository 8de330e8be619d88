"""Independent reference computations used to pin the oracle.

Each routine here is a different route to the same definitions (Section II,
Defs. 2-5) than the oracle's direct enumeration and Alg. 1 peeling, so a
mistake in either shows up as a disagreement:

* ``support_bruteforce``   -- every 2x2 vertex quadruple checked for all four
  edges (Def. 2), counted per edge.
* ``support_matrix``       -- closed form on the biadjacency matrix A:
  support(u,v) = (A A^T A)[u,v] - d(u) - d(v) + 1 (walks u-x-w-v with w != u
  and x != v).
* ``butterflies_total``    -- sum over upper pairs of C(|N(u1) ∩ N(u2)|, 2).
* ``phi_subsets``          -- bitruss numbers from Defs. 4-5 by enumerating
  every edge subset (tiny graphs): the k-bitruss is the union of all subsets
  in which every edge lies in >= k butterflies of the subset.
* ``phi_fixpoint``         -- for each k, the k-bitruss as the limit of
  repeatedly discarding edges with < k butterflies inside the current set,
  butterflies recounted from scratch with the matrix closed form.
"""
from __future__ import annotations

import itertools
from math import comb

import numpy as np


def read_golden(path):
    nU = nL = None
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if nU is None:
                nU, nL = int(parts[0]), int(parts[1])
                continue
            rows.append(parts)
    return nU, nL, rows


def biadjacency(edges, nU, nL):
    A = np.zeros((nU, nL), dtype=np.int64)
    e = np.asarray(edges).reshape(-1, 2)
    A[e[:, 0], e[:, 1]] = 1
    return A


def support_bruteforce(edges, nU, nL):
    e = np.asarray(edges).reshape(-1, 2)
    A = biadjacency(e, nU, nL)
    cnt = np.zeros((nU, nL), dtype=np.int64)
    for u1, u2 in itertools.combinations(range(nU), 2):
        for v1, v2 in itertools.combinations(range(nL), 2):
            if A[u1, v1] and A[u1, v2] and A[u2, v1] and A[u2, v2]:
                cnt[u1, v1] += 1
                cnt[u1, v2] += 1
                cnt[u2, v1] += 1
                cnt[u2, v2] += 1
    return cnt[e[:, 0], e[:, 1]].astype(np.uint64)


def support_matrix(edges, nU, nL):
    e = np.asarray(edges).reshape(-1, 2)
    A = biadjacency(e, nU, nL)
    P = A @ A.T @ A
    du = A.sum(1)
    dl = A.sum(0)
    s = P[e[:, 0], e[:, 1]] - du[e[:, 0]] - dl[e[:, 1]] + 1
    return s.astype(np.uint64)


def butterflies_total(edges, nU, nL):
    A = biadjacency(edges, nU, nL)
    C = A @ A.T
    iu = np.triu_indices(nU, 1)
    c = C[iu]
    return int((c * (c - 1) // 2).sum())


def _butterflies_in(edges_sub, nU, nL):
    """support of each edge inside the subgraph formed by edges_sub"""
    if len(edges_sub) == 0:
        return np.zeros(0, dtype=np.int64)
    return support_matrix(edges_sub, nU, nL).astype(np.int64)


def phi_subsets(edges, nU, nL):
    e = np.asarray(edges).reshape(-1, 2)
    m = e.shape[0]
    assert m <= 16, "subset enumeration is for tiny graphs"
    # butterflies as 4-edge index sets
    idx = {(int(a), int(b)): i for i, (a, b) in enumerate(e)}
    bfs = []
    for u1, u2 in itertools.combinations(range(nU), 2):
        for v1, v2 in itertools.combinations(range(nL), 2):
            q = [(u1, v1), (u1, v2), (u2, v1), (u2, v2)]
            if all(x in idx for x in q):
                bfs.append([idx[x] for x in q])
    kmax = len(bfs)
    phi = np.zeros(m, dtype=np.int64)
    for k in range(1, kmax + 1):
        union = 0
        for mask in range(1, 1 << m):
            cnt = [0] * m
            for b in bfs:
                if all(mask >> i & 1 for i in b):
                    for i in b:
                        cnt[i] += 1
            if all(cnt[i] >= k for i in range(m) if mask >> i & 1):
                union |= mask
        for i in range(m):
            if union >> i & 1:
                phi[i] = k
    return phi.astype(np.uint64)


def phi_fixpoint(edges, nU, nL):
    e = np.asarray(edges).reshape(-1, 2)
    m = e.shape[0]
    phi = np.zeros(m, dtype=np.int64)
    alive_k = np.ones(m, dtype=bool)
    k = 1
    while alive_k.any():
        cur = alive_k.copy()
        while True:
            sub = np.nonzero(cur)[0]
            s = _butterflies_in(e[sub], nU, nL)
            drop = sub[s < k]
            if drop.size == 0:
                break
            cur[drop] = False
        phi[cur] = k
        # the (k+1)-bitruss lies inside the k-bitruss
        alive_k = cur
        k += 1
    return phi.astype(np.uint64)


def biclique(a, b, u0=0, v0=0):
    return np.array([(u0 + i, v0 + j) for i in range(a) for j in range(b)], dtype=np.int32)


def fig2a_graph():
    """The 4002-vertex graph of Fig. 2(a) (Section I): u0 ~ {v0, v1};
    u1 ~ v0..v1000; v1 ~ u0..u1000; u2 ~ v1001..v2000; v2 ~ u1001..u2000.
    It has exactly one butterfly, [u0, v0, u1, v1]."""
    s = set()
    s.update({(0, 0), (0, 1)})
    s.update((1, j) for j in range(0, 1001))
    s.update((i, 1) for i in range(0, 1001))
    s.update((2, j) for j in range(1001, 2001))
    s.update((i, 2) for i in range(1001, 2001))
    e = np.array(sorted(s), dtype=np.int32)
    return e, 2001, 2001


def comb2(k):
    return comb(int(k), 2)
