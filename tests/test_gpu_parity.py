"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle,
bit for bit on supports (uint64) and bitruss numbers (uint32), plus BE-Index
structure checks (Section IV-A: Lemmas 1-4, 7; Fig. 6)."""
import os
from math import comb

import numpy as np
import pytest

import oracle
from paper_2001_06111_gb300 import bitruss as bt
from paper_2001_06111_gb300 import build, synth
from tests import pins
from tests.digests import assert_matches_digest, oracle_digest

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def h():
    build.build()
    handle = bt.bt_create(0)
    yield handle
    handle.close()


def decompose(h, edges, nU, nL, flags=0):
    sup, phi, st = bt.bt_decompose(h, edges, nU, nL, flags=flags)
    return sup, phi, st


def assert_parity(h, g_edges, nU, nL, flags=0):
    sup_ref, phi_ref = oracle.bitruss(g_edges, nU, nL)
    sup, phi, st = decompose(h, g_edges, nU, nL, flags)
    assert sup.dtype == np.uint64 and phi.dtype == np.uint32
    np.testing.assert_array_equal(sup, sup_ref)
    np.testing.assert_array_equal(phi.astype(np.uint64), phi_ref)
    cnt = bt.bt_count_support(h, g_edges, nU, nL, flags=flags)
    np.testing.assert_array_equal(cnt, sup_ref)
    return st


def test_paper_example(h):
    nU, nL, rows = pins.read_golden(os.path.join(GOLDEN, "paper_example_g.txt"))
    edges = np.array([(int(r[1]), int(r[2])) for r in rows], dtype=np.int32)
    sup_ref = np.array([int(r[3]) for r in rows], dtype=np.uint64)
    phi_ref = np.array([int(r[4]) for r in rows], dtype=np.uint32)
    for flags in (0, bt.BT_TIE_LOWER_FIRST):
        sup, phi, st = decompose(h, edges, nU, nL, flags)
        np.testing.assert_array_equal(sup, sup_ref)
        np.testing.assert_array_equal(phi, phi_ref)
    # batches: the two support-0 edges at k=0, then as in the BU++ example
    # (Section V-B) e6..e8 at k=1 and the six blue edges (three twin pairs of
    # B0) at k=2 -> three levels of one round each
    assert st["rounds"] == 3 and st["levels"] == 3 and st["phi_max"] == 2
    # support updates of the BU++ example under the Fig. 6 index (the last
    # flags above): the round at MBS = 1 kills the pairs (e5, e6) and (e7, e8)
    # of B1; e5 is outside the batch and loses k_B - 1 = 1 butterfly, the
    # twins e7, e8 are both in it, and B1 keeps no live pair.  The round at
    # MBS = 2 takes all three twin pairs of B0 with both members in the
    # batch, so no support changes: exactly one update in all.
    assert st["support_updates"] == 1


def test_paper_example_index_fig6(h):
    """Fig. 6 under the lower-layer-above reading: B0 is a 3-bloom (v1, v0
    dominant, wedges through u0, u1, u2), B1 the 2-bloom [u2, v1, u3, v2];
    twin(B0, e0) = e1; 10 links."""
    nU, nL, rows = pins.read_golden(os.path.join(GOLDEN, "paper_example_index.txt"))
    edges = np.array([(int(r[1]), int(r[2])) for r in rows if r[0].startswith("e")], dtype=np.int32)
    st = bt.bt_build_index(h, edges, nU, nL, bt.BT_TIE_LOWER_FIRST)
    k, first, pairs, deg = bt.bt_index_export(h, st, len(edges))
    assert sorted(k.tolist()) == [2, 3]
    assert st["n_bloom_wedges"] == 5 and st["n_butterflies"] == 4
    b0 = int(np.nonzero(k == 3)[0][0])
    p0 = pairs[first[b0]:first[b0] + 3]
    twins = {frozenset(map(int, p)) for p in p0}
    assert twins == {frozenset({0, 1}), frozenset({2, 3}), frozenset({4, 5})}
    b1 = int(np.nonzero(k == 2)[0][0])
    p1 = pairs[first[b1]:first[b1] + 2]
    assert {frozenset(map(int, p)) for p in p1} == {frozenset({5, 6}), frozenset({7, 8})}
    # links per edge: e5 is in both blooms, the gray edges in none
    assert deg.tolist() == [1, 1, 1, 1, 1, 2, 1, 1, 1, 0, 0]
    # default reading (upper ids above lower ids): four 2-blooms, 16 links
    st2 = bt.bt_build_index(h, edges, nU, nL, 0)
    k2, _, _, _ = bt.bt_index_export(h, st2, len(edges))
    assert sorted(k2.tolist()) == [2, 2, 2, 2] and st2["n_bloom_wedges"] == 8


def check_index_invariants(h, edges, nU, nL, sup, flags=0):
    st = bt.bt_build_index(h, edges, nU, nL, flags)
    k, first, pairs, deg = bt.bt_index_export(h, st, len(edges))
    # Lemma 7: a k-bloom is k priority-obeyed wedges (pairs); the layout keeps
    # each bloom's pairs contiguous and in bloom order (the peel relies on it)
    sizes = np.diff(np.append(first.astype(np.int64), st["n_bloom_wedges"]))
    np.testing.assert_array_equal(sizes, k.astype(np.int64))
    order = np.argsort(first)
    assert (np.sort(sizes[order]) >= 2).all() if len(k) else True
    assert int(k.astype(np.int64).sum()) == st["n_bloom_wedges"]
    # Lemmas 1, 3: blooms hold every butterfly exactly once
    bf = sum(comb(int(x), 2) for x in k)
    assert bf == st["n_butterflies"] == int(sup.sum()) // 4
    # Lemma 2 + Lemma 3: support(e) = sum over its blooms of (k_B - 1)
    bloom_of_pair = np.repeat(np.arange(len(k))[order], sizes[order]) if len(k) else np.zeros(0, int)
    acc = np.zeros(len(edges), dtype=np.int64)
    kk = k.astype(np.int64)
    np.add.at(acc, pairs[:, 0].astype(np.int64), kk[bloom_of_pair] - 1)
    np.add.at(acc, pairs[:, 1].astype(np.int64), kk[bloom_of_pair] - 1)
    np.testing.assert_array_equal(acc.astype(np.uint64), sup)
    # twins share their middle vertex (Def. 9): (u,v) and (v,w) meet in v
    a, b = edges[pairs[:, 0]], edges[pairs[:, 1]]
    assert ((a[:, 0] == b[:, 0]) ^ (a[:, 1] == b[:, 1])).all()
    # links per edge
    cnt = np.bincount(pairs.reshape(-1).astype(np.int64), minlength=len(edges))
    np.testing.assert_array_equal(cnt, deg)
    return st


@pytest.mark.parametrize("seed", range(40))
def test_random_small_graphs(h, seed):
    rng = np.random.default_rng(seed)
    nU, nL = int(rng.integers(1, 30)), int(rng.integers(1, 30))
    m = int(rng.integers(1, nU * nL + 1))
    g = synth.random_tiny(seed, nU, nL, m)
    assert_parity(h, g.edges, nU, nL)


@pytest.mark.parametrize("seed", range(6))
def test_chunglu_graphs_and_index(h, seed):
    g = synth.chunglu(400 + 100 * seed, 300, 4000 + 500 * seed, 2.1 + 0.1 * seed, 2.3, seed=100 + seed)
    assert_parity(h, g.edges, g.nU, g.nL)
    sup = oracle.support(g.edges, g.nU, g.nL)
    check_index_invariants(h, g.edges, g.nU, g.nL, sup)
    check_index_invariants(h, g.edges, g.nU, g.nL, sup, bt.BT_TIE_LOWER_FIRST)


def test_small_workload_parity(h):
    g = synth.small()
    st = assert_parity(h, g.edges, g.nU, g.nL)
    assert st["rounds"] >= st["levels"] >= 1


def test_small_workload_tie_reading_and_relabel(h):
    g = synth.small()
    s0, p0, _ = decompose(h, g.edges, g.nU, g.nL)
    s1, p1, _ = decompose(h, g.edges, g.nU, g.nL, bt.BT_TIE_LOWER_FIRST)
    np.testing.assert_array_equal(s0, s1)
    np.testing.assert_array_equal(p0, p1)
    sw = np.ascontiguousarray(g.edges[:, ::-1])
    s2, p2, _ = decompose(h, sw, g.nL, g.nU)
    np.testing.assert_array_equal(p0, p2)


@pytest.mark.parametrize("a,b", [(2, 2), (3, 7), (2, 1001), (40, 50), (1, 9)])
def test_bicliques(h, a, b):
    e = pins.biclique(a, b)
    sup, phi, _ = decompose(h, e, a, b)
    k = (a - 1) * (b - 1)
    assert (sup == k).all() and (phi == k).all()


def test_fig2a_graph(h):
    e, nU, nL = pins.fig2a_graph()
    assert_parity(h, e, nU, nL)


def test_heavy_vertex_over_many_chunks(h):
    # one upper vertex adjacent to every lower vertex plus a sparse rest:
    # its wedge walk spans many 512-vertex chunks
    rng = np.random.default_rng(7)
    nU, nL = 300, 3000
    hub = [(0, v) for v in range(nL)]
    rest = set()
    while len(rest) < 6000:
        u, v = int(rng.integers(1, nU)), int(rng.integers(0, nL))
        rest.add((u, v))
    e = np.array(hub + sorted(rest), dtype=np.int32)
    assert_parity(h, e, nU, nL)


def test_start_vertex_with_2_16_lower_neighbours(h):
    # a start vertex with at least 2^16 lower-ranked neighbours: its counter
    # words cannot also count readers, so the count kernel clears them in a
    # third walk and emit's place walk runs over the same 66k-arc vertex;
    # three more upper vertices share 200 random neighbours each with it
    rng = np.random.default_rng(11)
    nU, nL = 4, 66000
    rows = [(0, v) for v in range(nL)]
    for w in range(1, nU):
        rows += [(w, int(v)) for v in rng.choice(nL, 200, replace=False)]
    e = np.array(rows, dtype=np.int32)
    for flags in (0, bt.BT_TIE_LOWER_FIRST):
        st = assert_parity(h, e, nU, nL, flags)
        assert st["phi_max"] >= 100


def test_isolated_vertices_and_single_edge(h):
    assert_parity(h, np.array([[3, 4]], np.int32), 10, 12)
    e = pins.biclique(3, 3, 5, 7)
    assert_parity(h, e, 20, 20)


def test_empty_graph(h):
    sup, phi, st = decompose(h, np.zeros((0, 2), np.int32), 5, 5)
    assert sup.size == 0 and phi.size == 0


def test_input_errors(h):
    with pytest.raises(bt.BitrussError) as ei:
        decompose(h, np.array([[0, 1], [0, 1]], np.int32), 2, 2)
    assert ei.value.code == bt.BT_ERR_DUP
    with pytest.raises(bt.BitrussError) as ei:
        decompose(h, np.array([[0, 1], [2, 1]], np.int32), 2, 2)
    assert ei.value.code == bt.BT_ERR_RANGE
    with pytest.raises(bt.BitrussError) as ei:
        bt.bt_count_support(h, np.array([[0, -1]], np.int32), 2, 2)
    assert ei.value.code == bt.BT_ERR_RANGE
    with pytest.raises(bt.BitrussError) as ei:
        bt.bt_decompose(h, np.array([[0, 0]], np.int32), 1, 1, flags=0x80)
    assert ei.value.code == bt.BT_ERR_ARG
    # the handle stays usable after errors
    assert_parity(h, pins.biclique(3, 4), 3, 4)


def test_device_pointer_path(h):
    torch = pytest.importorskip("torch")
    g = synth.small()
    d = torch.from_numpy(g.edges).cuda()
    sup_d, phi_d, _ = bt.bt_decompose(h, d, g.nU, g.nL)
    sup_h, phi_h, _ = decompose(h, g.edges, g.nU, g.nL)
    np.testing.assert_array_equal(sup_d.cpu().numpy().view(np.uint64), sup_h)
    np.testing.assert_array_equal(phi_d.cpu().numpy().view(np.uint32), phi_h)


def test_medium_workload_full_size_exact(h):
    """The 2M-edge workload at full size, in the configuration the benchmark
    times: every support and bitruss number equals the CPU oracle's (digests
    of the oracle's full arrays, computed offline)."""
    g = synth.medium()
    sup, phi, st = decompose(h, g.edges, g.nU, g.nL)
    assert_matches_digest(g, sup, phi, oracle_digest("medium"))


def test_medium_workload_full_size(h):
    """The 2M-edge workload at full size: supports of sampled edges
    recomputed one by one by the oracle, bitruss numbers checked by the local
    fixpoint property on sampled edges, and global invariants on all edges."""
    g = synth.medium()
    sup, phi, st = decompose(h, g.edges, g.nU, g.nL)
    rng = np.random.default_rng(12)
    which = rng.choice(g.m, 400, replace=False).astype(np.uint64)
    # include the highest-support edges (hub edges) in the sample
    which = np.unique(np.concatenate([which, np.argsort(sup)[-40:].astype(np.uint64)]))
    np.testing.assert_array_equal(sup[which], oracle.support_sampled(g.edges, g.nU, g.nL, which))
    assert (phi.astype(np.uint64) <= sup).all()
    stats = bt.bt_build_index(h, g.edges, g.nU, g.nL)
    assert stats["n_butterflies"] * 4 == int(sup.sum())
    cnt, hv = oracle.local_check(g.edges, g.nU, g.nL, phi, which)
    assert (cnt >= phi[which]).all()
    np.testing.assert_array_equal(hv, phi[which].astype(np.uint64))


def test_medium_vertex_sample_exact(h):
    """Full bit-exact parity on a 20% vertex-induced sample of the 2M-edge
    workload (the sampling of the paper's scalability study, Section VI)."""
    g = synth.vertex_sample(synth.medium(), 0.2, 7)
    assert_parity(h, g.edges, g.nU, g.nL)


@pytest.mark.parametrize("join_cap,block_links", [(1, 2), (3, 16), (8, 64), (640, 2)])
def test_overflow_paths_exact(h, join_cap, block_links):
    """The paths large graphs take, forced on small ones (bt_set_limits): a
    block that lists more joining edges than its cap lets the others queue
    their own links, and link lists longer than the block stage takes become
    incidence items.  Results stay bit-exact against the oracle."""
    graphs = [synth.small(), synth.chunglu(600, 400, 6000, 2.2, 2.4, seed=42),
              synth.Graph(pins.biclique(40, 50), 40, 50)]
    try:
        bt.bt_set_limits(h, join_cap=join_cap, block_links=block_links)
        for g in graphs:
            assert_parity(h, g.edges, g.nU, g.nL)
        # the batch peel takes the same paths
        outs, _ = bt.bt_decompose_batch(h, [(g.edges, g.nU, g.nL) for g in graphs])
        for (sup, phi), g in zip(outs, graphs):
            sr, pr = oracle.bitruss(g.edges, g.nU, g.nL)
            np.testing.assert_array_equal(sup, sr)
            np.testing.assert_array_equal(phi.astype(np.uint64), pr)
    finally:
        bt.bt_set_limits(h)
