"""Pins for the CPU oracle (no GPU): worked examples, closed forms, brute
force on tiny graphs and invariants, so that a plausible mistake anywhere in
the oracle (a dropped butterfly, a wrong decrement, a wrong peel order) fails
at least one of them."""
import os

import numpy as np
import pytest

import oracle
from paper_2001_06111_gb300 import synth
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_example_support_and_phi():
    nU, nL, rows = pins.read_golden(os.path.join(GOLDEN, "paper_example_g.txt"))
    edges = np.array([(int(r[1]), int(r[2])) for r in rows], dtype=np.int32)
    sup_ref = np.array([int(r[3]) for r in rows], dtype=np.uint64)
    phi_ref = np.array([int(r[4]) for r in rows], dtype=np.uint64)
    sup, phi = oracle.bitruss(edges, nU, nL)
    assert sup.tolist() == sup_ref.tolist()
    assert phi.tolist() == phi_ref.tolist()
    # four butterflies in G (Section IV-A: the 3-bloom H2 holds 3, plus [u2,v1,u3,v2])
    assert int(sup.sum()) == 4 * 4
    assert oracle.support(edges, nU, nL).tolist() == sup_ref.tolist()


@pytest.mark.parametrize("a,b", [(2, 2), (2, 5), (3, 3), (4, 7), (6, 5), (2, 1001)])
def test_biclique_closed_form(a, b):
    # A k-bloom holds C(k,2) butterflies and each edge lies in k-1 of them
    # (Lemmas 1-2); for K_{a,b} every edge is in (a-1)(b-1) butterflies and the
    # whole graph is its own (a-1)(b-1)-bitruss.  (2,1001) is Fig. 3(a).
    e = pins.biclique(a, b)
    sup, phi = oracle.bitruss(e, a, b)
    k = (a - 1) * (b - 1)
    assert (sup == k).all() and (phi == k).all()


def test_fig2a_single_butterfly():
    e, nU, nL = pins.fig2a_graph()
    assert e.shape[0] == 4002
    sup, phi = oracle.bitruss(e, nU, nL)
    bf = {(0, 0), (0, 1), (1, 0), (1, 1)}
    want = np.array([1 if (int(a), int(b)) in bf else 0 for a, b in e], dtype=np.uint64)
    assert sup.tolist() == want.tolist()
    assert phi.tolist() == want.tolist()


def test_disjoint_union_of_bicliques():
    parts = [(2, 3, 0, 0), (3, 4, 2, 3), (5, 2, 5, 7)]
    e = np.concatenate([pins.biclique(a, b, u0, v0) for a, b, u0, v0 in parts])
    sup, phi = oracle.bitruss(e, 10, 9)
    want = np.concatenate([np.full(a * b, (a - 1) * (b - 1)) for a, b, _, _ in parts])
    assert sup.tolist() == want.tolist() and phi.tolist() == want.tolist()


def test_empty_and_edgeless_cases():
    sup, phi = oracle.bitruss(np.zeros((0, 2), np.int32), 3, 3)
    assert sup.size == 0 and phi.size == 0
    star = np.array([(0, j) for j in range(6)], dtype=np.int32)  # no butterfly
    sup, phi = oracle.bitruss(star, 1, 6)
    assert (sup == 0).all() and (phi == 0).all()


def test_input_errors():
    with pytest.raises(ValueError, match="duplicate"):
        oracle.bitruss(np.array([(0, 0), (0, 0)], np.int32), 1, 1)
    with pytest.raises(ValueError, match="range"):
        oracle.support(np.array([(0, 3)], np.int32), 1, 2)


@pytest.mark.parametrize("seed", range(12))
def test_tiny_random_vs_subset_enumeration(seed):
    rng = np.random.default_rng(1000 + seed)
    nU, nL = int(rng.integers(2, 5)), int(rng.integers(2, 5))
    m = int(rng.integers(4, min(nU * nL, 13) + 1))
    g = synth.random_tiny(seed, nU, nL, m)
    sup, phi = oracle.bitruss(g.edges, nU, nL)
    assert sup.tolist() == pins.support_bruteforce(g.edges, nU, nL).tolist()
    assert phi.tolist() == pins.phi_subsets(g.edges, nU, nL).tolist()


@pytest.mark.parametrize("seed,nU,nL,m", [(1, 12, 10, 70), (2, 20, 8, 90), (3, 9, 30, 120),
                                          (4, 40, 40, 300), (5, 25, 60, 500)])
def test_small_random_vs_fixpoint(seed, nU, nL, m):
    g = synth.random_tiny(seed, nU, nL, m)
    sup, phi = oracle.bitruss(g.edges, nU, nL)
    assert sup.tolist() == pins.support_matrix(g.edges, nU, nL).tolist()
    assert phi.tolist() == pins.phi_fixpoint(g.edges, nU, nL).tolist()


def test_skewed_graph_vs_fixpoint():
    # a small Chung-Lu graph with hubs: deep peeling levels on few edges
    g = synth.chunglu(60, 50, 600, 2.1, 2.3, seed=11)
    sup, phi = oracle.bitruss(g.edges, g.nU, g.nL)
    assert sup.tolist() == pins.support_matrix(g.edges, g.nU, g.nL).tolist()
    assert phi.tolist() == pins.phi_fixpoint(g.edges, g.nU, g.nL).tolist()


def test_invariants_on_small_workload():
    g = synth.small()
    sup, phi = oracle.bitruss(g.edges, g.nU, g.nL)
    # sum of supports = 4 x butterflies (Lemma 8 proof)
    assert int(sup.sum()) == 4 * pins.butterflies_total(g.edges, g.nU, g.nL)
    # closed form per edge
    assert sup.tolist() == pins.support_matrix(g.edges, g.nU, g.nL).tolist()
    # phi <= support; support <= (d(u)-1)(d(v)-1) (Lemma 8)
    assert (phi <= sup).all()
    du = np.bincount(g.edges[:, 0], minlength=g.nU)
    dl = np.bincount(g.edges[:, 1], minlength=g.nL)
    assert (sup <= (du[g.edges[:, 0]] - 1) * (dl[g.edges[:, 1]] - 1)).all()
    # certificate and local fixpoint on every edge
    cnt, h = oracle.local_check(g.edges, g.nU, g.nL, phi, np.arange(g.m))
    assert (cnt >= phi).all()
    assert (h == phi).all()
    # phi_max <= k_max (largest k with >= k edges of support >= k, Section V-C)
    s = np.sort(sup)[::-1]
    kmax = int(np.max(np.minimum(s, np.arange(1, s.size + 1))))
    assert int(phi.max()) <= kmax


def test_relabel_and_layer_swap_invariance():
    g = synth.chunglu(300, 200, 3000, 2.2, 2.4, seed=5)
    sup, phi = oracle.bitruss(g.edges, g.nU, g.nL)
    rng = np.random.default_rng(9)
    pu, pl, pe = rng.permutation(g.nU), rng.permutation(g.nL), rng.permutation(g.m)
    e2 = np.stack([pu[g.edges[pe, 0]], pl[g.edges[pe, 1]]], 1).astype(np.int32)
    sup2, phi2 = oracle.bitruss(e2, g.nU, g.nL)
    assert sup2.tolist() == sup[pe].tolist() and phi2.tolist() == phi[pe].tolist()
    e3 = np.ascontiguousarray(g.edges[:, ::-1])
    sup3, phi3 = oracle.bitruss(e3, g.nL, g.nU)
    assert sup3.tolist() == sup.tolist() and phi3.tolist() == phi.tolist()


def test_sampled_support_matches_full():
    g = synth.small()
    full = oracle.support(g.edges, g.nU, g.nL)
    which = np.arange(0, g.m, 97, dtype=np.uint64)
    assert oracle.support_sampled(g.edges, g.nU, g.nL, which).tolist() == full[which].tolist()


def test_local_check_detects_planted_mistakes():
    # A planted off-by-one in phi (on the CPU) must break the fixpoint check
    g = synth.chunglu(300, 200, 3000, 2.2, 2.4, seed=5)
    _, phi = oracle.bitruss(g.edges, g.nU, g.nL)
    rng = np.random.default_rng(3)
    cand = np.nonzero(phi > 0)[0]
    for e in rng.choice(cand, 20, replace=False):
        for delta in (-1, 1):
            bad = phi.copy()
            bad[e] = bad[e] + delta if delta > 0 else bad[e] - 1
            cnt, h = oracle.local_check(g.edges, g.nU, g.nL, bad, np.array([e]))
            assert not (h[0] == bad[e] and cnt[0] >= bad[e])


# ---------------------------------------------------------------- hierarchy
def test_paper_example_k_bitrusses():
    # Section I and Example 1 (Section II): H_2 is the six blue edges
    # e0..e5, H_1 adds the three yellow edges e6..e8, the gray e9, e10 lie only
    # in H_0 = G.
    nU, nL, rows = pins.read_golden(os.path.join(GOLDEN, "paper_example_g.txt"))
    edges = np.array([(int(r[1]), int(r[2])) for r in rows], dtype=np.int32)
    assert np.flatnonzero(oracle.k_bitruss(edges, nU, nL, 0)).tolist() == list(range(11))
    assert np.flatnonzero(oracle.k_bitruss(edges, nU, nL, 1)).tolist() == list(range(9))
    assert np.flatnonzero(oracle.k_bitruss(edges, nU, nL, 2)).tolist() == list(range(6))
    assert not oracle.k_bitruss(edges, nU, nL, 3).any()
    # e0..e5 all have phi 2, e6..e8 phi 1: in ascending input order per level
    assert oracle.hierarchy([2, 2, 2, 2, 2, 2, 1, 1, 1, 0, 0]).tolist() == list(range(11))


@pytest.mark.parametrize("a,b", [(2, 2), (3, 4), (5, 3)])
def test_k_bitruss_of_biclique(a, b):
    # every edge of K_{a,b} is in (a-1)(b-1) butterflies (Lemmas 1-2)
    e = pins.biclique(a, b)
    t = (a - 1) * (b - 1)
    for k in (0, 1, t, t + 1):
        assert oracle.k_bitruss(e, a, b, k).all() == (k <= t)
        assert oracle.k_bitruss(e, a, b, k).any() == (k <= t)


def test_k_bitruss_of_disjoint_bicliques():
    # K_{2,3} (2 butterflies an edge) beside K_{3,3} (4 an edge): H_3 and H_4
    # are the K_{3,3} alone
    e = np.concatenate([pins.biclique(2, 3, 0, 0), pins.biclique(3, 3, 2, 3)])
    for k, want in ((2, np.ones(15, bool)), (3, np.r_[np.zeros(6, bool), np.ones(9, bool)]),
                    (4, np.r_[np.zeros(6, bool), np.ones(9, bool)]), (5, np.zeros(15, bool))):
        assert oracle.k_bitruss(e, 5, 6, k).tolist() == want.tolist()


@pytest.mark.parametrize("seed", range(6))
def test_k_bitruss_matches_phi(seed):
    # Def. 5: phi_e is the largest k whose k-bitruss holds e, so H_k computed by
    # deletion (Def. 4) and the edges with phi >= k from Alg. 1 peeling agree
    g = synth.random_tiny(50 + seed, 14, 12, 80)
    _, phi = oracle.bitruss(g.edges, 14, 12)
    for k in range(int(phi.max()) + 2):
        assert oracle.k_bitruss(g.edges, 14, 12, k).tolist() == (phi >= k).tolist()


def test_hierarchy_order_by_brute_force():
    rng = np.random.default_rng(7)
    phi = rng.integers(0, 6, size=300)
    order = oracle.hierarchy(phi)
    assert order.tolist() == sorted(range(300), key=lambda e: (-int(phi[e]), e))
    for k in range(8):
        n = int((phi >= k).sum())
        assert sorted(order[:n].tolist()) == np.flatnonzero(phi >= k).tolist()


def test_anchored_support_paper_example():
    # per-anchor contributions derived by hand from Lemma 3 and Def. 7 on G
    # (tests/golden/paper_example_anchored.txt), under both id readings
    nU, nL, rows = pins.read_golden(os.path.join(GOLDEN, "paper_example_anchored.txt"))
    edges = np.array([(int(r[1]), int(r[2])) for r in rows], dtype=np.int32)
    col = lambda j: [int(r[j]) for r in rows]  # noqa: E731
    assert oracle.support_anchored(edges, nU, nL, 8, 9).tolist() == col(3)
    assert oracle.support_anchored(edges, nU, nL, 7, 8).tolist() == col(4)
    assert oracle.support_anchored(edges, nU, nL, 0, 7).tolist() == [0] * len(rows)
    assert oracle.support_anchored(edges, nU, nL, 8, 9, lower_first=True).tolist() == col(5)
    assert oracle.support_anchored(edges, nU, nL, 0, 8, lower_first=True).tolist() == [0] * len(rows)


@pytest.mark.parametrize("a,b", [(2, 3), (3, 5), (4, 9)])
def test_anchored_support_biclique_closed_form(a, b):
    # K_{a,b}, a < b: upper vertices have degree b > a, so the anchor of a
    # butterfly {u_j, u_i} x {v_x, v_y} (j < i) is u_i (ties broken by the
    # larger id).  Anchor u_i holds i * C(b, 2) butterflies: its own edges lie
    # in i (b - 1) of them, each edge of a lower upper vertex u_j in b - 1.
    # Ranks: the b lower vertices first (degree a), then u_0 .. u_{a-1}, so
    # u_i has rank b + i.
    e = pins.biclique(a, b)
    for i in range(a):
        got = oracle.support_anchored(e, a, b, b + i, b + i + 1)
        want = np.array([i * (b - 1) if int(u) == i else (b - 1 if int(u) < i else 0) for u, _ in e])
        assert got.tolist() == want.tolist()
    assert (oracle.support_anchored(e, a, b, 0, b) == 0).all()


@pytest.mark.parametrize("seed", range(4))
def test_anchored_support_partitions_sum_to_support(seed):
    # Lemma 3: every butterfly has exactly one anchor, so the supports of the
    # ranges of any partition of the ranks add up to the supports
    g = synth.chunglu(120, 90, 900, 2.1, 2.4, seed=300 + seed)
    n = g.nU + g.nL
    rng = np.random.default_rng(seed)
    cuts = np.sort(rng.choice(np.arange(1, n), size=5, replace=False))
    bounds = [0, *cuts.tolist(), n]
    for lower_first in (False, True):
        parts = [oracle.support_anchored(g.edges, g.nU, g.nL, lo, hi, lower_first)
                 for lo, hi in zip(bounds[:-1], bounds[1:])]
        np.testing.assert_array_equal(np.sum(parts, axis=0), oracle.support(g.edges, g.nU, g.nL))
