"""Progressive compression (BiT-PC, Alg. 6-7): bit-identical to the CPU
oracle and to the plain batch peel for every tau, including the degenerate
steps tau = 1 (one candidate pass per eps in {k_max, 0}) and small tau."""
import os

import numpy as np
import pytest

import oracle
from paper_2001_06111_gb300 import bitruss as bt
from paper_2001_06111_gb300 import build, synth
from tests import pins

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TAUS = (0.02, 0.1, 0.5, 1.0)


@pytest.fixture(scope="module")
def h():
    build.build()
    handle = bt.bt_create(0)
    yield handle
    handle.close()


@pytest.mark.parametrize("tau", TAUS)
def test_pc_paper_example(h, tau):
    nU, nL, rows = pins.read_golden(os.path.join(GOLDEN, "paper_example_g.txt"))
    edges = np.array([(int(r[1]), int(r[2])) for r in rows], dtype=np.int32)
    sup, phi, st = bt.bt_decompose_progressive(h, edges, nU, nL, tau)
    assert sup.tolist() == [int(r[3]) for r in rows]
    assert phi.tolist() == [int(r[4]) for r in rows]
    # supports 3,2,2,2,2,2,1,1,1,0,0: k_max = 2 (at least 2 edges with support >= 2)
    assert st["k_max"] == 2


@pytest.mark.parametrize("seed", range(16))
def test_pc_random_small_graphs(h, seed):
    rng = np.random.default_rng(300 + seed)
    nU, nL = int(rng.integers(2, 30)), int(rng.integers(2, 30))
    g = synth.random_tiny(300 + seed, nU, nL, int(rng.integers(1, nU * nL + 1)))
    sr, pr = oracle.bitruss(g.edges, nU, nL)
    for tau in TAUS:
        sup, phi, _ = bt.bt_decompose_progressive(h, g.edges, nU, nL, tau)
        np.testing.assert_array_equal(sup, sr)
        np.testing.assert_array_equal(phi.astype(np.uint64), pr)


@pytest.mark.parametrize("seed", range(4))
def test_pc_skewed_graphs_vs_oracle(h, seed):
    g = synth.chunglu(500, 300, 5000 + 1000 * seed, 2.0 + 0.15 * seed, 2.3, seed=700 + seed)
    sr, pr = oracle.bitruss(g.edges, g.nU, g.nL)
    for tau in TAUS:
        sup, phi, st = bt.bt_decompose_progressive(h, g.edges, g.nU, g.nL, tau,
                                                   flags=bt.BT_TIE_LOWER_FIRST if seed % 2 else 0)
        np.testing.assert_array_equal(phi.astype(np.uint64), pr)
        assert st["passes"] >= 1


def test_pc_small_workload_and_planted_bicliques(h):
    g = synth.small()
    sr, pr = oracle.bitruss(g.edges, g.nU, g.nL)
    _, phi, _ = bt.bt_decompose_progressive(h, g.edges, g.nU, g.nL, 0.05)
    np.testing.assert_array_equal(phi.astype(np.uint64), pr)
    # dense planted blocks: phi levels far above the rest
    p = synth.chunglu(3000, 2000, 40000, 2.1, 2.3, seed=8, nplant=6, plant_lo=20, plant_hi=40,
                      plant_p=0.9)
    sr, pr = oracle.bitruss(p.edges, p.nU, p.nL)
    _, phi, _ = bt.bt_decompose_progressive(h, p.edges, p.nU, p.nL, 0.02)
    np.testing.assert_array_equal(phi.astype(np.uint64), pr)


def test_pc_medium_equals_batch_peel(h):
    g = synth.medium()
    s0, p0, st0 = bt.bt_decompose(h, g.edges, g.nU, g.nL)
    s1, p1, st1 = bt.bt_decompose_progressive(h, g.edges, g.nU, g.nL, 0.1)
    np.testing.assert_array_equal(s0, s1)
    np.testing.assert_array_equal(p0, p1)


def test_pc_rejects_bad_tau(h):
    e = pins.biclique(3, 3)
    for tau in (0.0, -1.0, 1.5):
        with pytest.raises(bt.BitrussError) as ei:
            bt.bt_decompose_progressive(h, e, 3, 3, tau)
        assert ei.value.code == bt.BT_ERR_ARG


@pytest.mark.parametrize("tau", (0.5, 1.0))
def test_pc_links_of_compressed_indexes(h, tau):
    # Paper example G: the first pass (eps = k_max = 2) holds the six edges of
    # support >= 2, K_{3,2} on {u0,u1,u2} x {v0,v1}, one 3-bloom anchored at v1
    # (highest degree, then id), 3 pairs -> 6 links.  Later passes link only the
    # unassigned edges: e6..e8 each lie in one butterfly, i.e. one link to a
    # 2-bloom (support = sum of k_B - 1 over the links, Lemma 3), and e9, e10
    # in none: 9 links over all passes for both tau.
    nU, nL, rows = pins.read_golden(os.path.join(GOLDEN, "paper_example_g.txt"))
    edges = np.array([(int(r[1]), int(r[2])) for r in rows], dtype=np.int32)
    _, _, st = bt.bt_decompose_progressive(h, edges, nU, nL, tau)
    assert st["links"] == 9
    assert st["index_bytes_max"] > 0
    full = bt.bt_build_index(h, edges, nU, nL)
    assert st["index_bytes_max"] <= full["index_bytes"] + 8 * 12  # same graph, fewer links


def test_pc_compressed_index_smaller_on_medium(h):
    # the last pass indexes the whole graph but links only unassigned edges
    g = synth.medium()
    full = bt.bt_build_index(h, g.edges, g.nU, g.nL)
    _, _, st = bt.bt_decompose_progressive(h, g.edges, g.nU, g.nL, 0.1)
    assert 0 < st["index_bytes_max"] < full["index_bytes"]


# Alg. 7's own extraction (BT_PC_RECOUNT): supports recounted on each candidate
# subgraph and candidates below eps dropped before the compressed index.


@pytest.mark.parametrize("tau", TAUS)
def test_pc_recount_paper_example(h, tau):
    nU, nL, rows = pins.read_golden(os.path.join(GOLDEN, "paper_example_g.txt"))
    edges = np.array([(int(r[1]), int(r[2])) for r in rows], dtype=np.int32)
    sup, phi, st = bt.bt_decompose_progressive(h, edges, nU, nL, tau, flags=bt.BT_PC_RECOUNT)
    assert sup.tolist() == [int(r[3]) for r in rows]
    assert phi.tolist() == [int(r[4]) for r in rows]
    assert st["k_max"] == 2


@pytest.mark.parametrize("seed", range(16))
def test_pc_recount_random_small_graphs(h, seed):
    rng = np.random.default_rng(500 + seed)
    nU, nL = int(rng.integers(2, 30)), int(rng.integers(2, 30))
    g = synth.random_tiny(500 + seed, nU, nL, int(rng.integers(1, nU * nL + 1)))
    sr, pr = oracle.bitruss(g.edges, nU, nL)
    for tau in TAUS:
        sup, phi, _ = bt.bt_decompose_progressive(h, g.edges, nU, nL, tau, flags=bt.BT_PC_RECOUNT)
        np.testing.assert_array_equal(sup, sr)
        np.testing.assert_array_equal(phi.astype(np.uint64), pr)


@pytest.mark.parametrize("seed", range(3))
def test_pc_recount_skewed_graphs(h, seed):
    g = synth.chunglu(1500, 1000, 15000, 2.1, 2.4, seed=700 + seed)
    sr, pr = oracle.bitruss(g.edges, g.nU, g.nL)
    dropped = 0
    for tau in (0.02, 0.1):
        sup, phi, st = bt.bt_decompose_progressive(h, g.edges, g.nU, g.nL, tau, flags=bt.BT_PC_RECOUNT)
        np.testing.assert_array_equal(sup, sr)
        np.testing.assert_array_equal(phi.astype(np.uint64), pr)
        dropped += st["dropped_edges"]
        # the recount only removes candidates: a pass indexes at most what it extracted
        assert st["candidate_edges"] <= st["passes"] * g.m
    assert dropped > 0  # skewed supports: some candidates fall below eps on G_{>=eps}


def test_pc_recount_medium_sample_equals_batch_peel(h):
    g = synth.vertex_sample(synth.medium(), 0.2, 7)
    _, phi_bu, _ = bt.bt_decompose(h, g.edges, g.nU, g.nL)
    for tau in (0.02, 0.1):
        _, phi, _ = bt.bt_decompose_progressive(h, g.edges, g.nU, g.nL, tau, flags=bt.BT_PC_RECOUNT)
        np.testing.assert_array_equal(phi, phi_bu)
