"""Batched decomposition (bt_decompose_batch): every graph's result must be
bit-identical to its own decomposition, alone, and to the CPU oracle."""
import os

import numpy as np
import pytest

import oracle
from paper_2001_06111_gb300 import bitruss as bt
from paper_2001_06111_gb300 import build, synth
from tests import pins

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def h():
    build.build()
    handle = bt.bt_create(0)
    yield handle
    handle.close()


def mixed_graphs():
    nU, nL, rows = pins.read_golden(os.path.join(GOLDEN, "paper_example_g.txt"))
    ex = np.array([(int(r[1]), int(r[2])) for r in rows], dtype=np.int32)
    gs = [(ex, nU, nL), (np.zeros((0, 2), np.int32), 3, 4), (pins.biclique(3, 5), 3, 5),
          (pins.biclique(2, 1001), 2, 1001)]
    for s in range(30):
        rng = np.random.default_rng(500 + s)
        a, b = int(rng.integers(1, 25)), int(rng.integers(1, 25))
        g = synth.random_tiny(500 + s, a, b, int(rng.integers(1, a * b + 1)))
        gs.append((g.edges, a, b))
    for s in range(6):
        g = synth.chunglu(300 + 50 * s, 200, 2500 + 300 * s, 2.0 + 0.1 * s, 2.4, seed=900 + s)
        gs.append((g.edges, g.nU, g.nL))
    gs.append((synth.small().edges, 2000, 1500))
    return gs


def test_batch_matches_oracle_per_graph(h):
    gs = mixed_graphs()
    outs, st = bt.bt_decompose_batch(h, gs)
    assert st["graphs"] == len(gs) and st["launches"] == 1
    for (e, nU, nL), (sup, phi) in zip(gs, outs):
        sr, pr = oracle.bitruss(e, nU, nL)
        np.testing.assert_array_equal(sup, sr)
        np.testing.assert_array_equal(phi.astype(np.uint64), pr)


def test_batch_split_into_several_unions(h):
    gs = mixed_graphs()
    whole, _ = bt.bt_decompose_batch(h, gs)
    parts, st = bt.bt_decompose_batch(h, gs, max_edges_per_launch=6000)
    assert st["launches"] > 3
    for (s0, p0), (s1, p1) in zip(whole, parts):
        np.testing.assert_array_equal(s0, s1)
        np.testing.assert_array_equal(p0, p1)


def test_batch_tie_reading_same_results(h):
    gs = mixed_graphs()[:12]
    a, _ = bt.bt_decompose_batch(h, gs)
    b, _ = bt.bt_decompose_batch(h, gs, flags=bt.BT_TIE_LOWER_FIRST)
    for (s0, p0), (s1, p1) in zip(a, b):
        np.testing.assert_array_equal(s0, s1)
        np.testing.assert_array_equal(p0, p1)


def test_batch_distribution_alone_vs_together(h):
    """Graphs of the batched workload's distribution (sizes log-uniform in
    [100, 200,000]): the union result equals each graph decomposed alone."""
    idx = [0, 1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233, 377, 610, 987]
    graphs = [synth.batch_graph(i) for i in idx]
    gs = [(g.edges, g.nU, g.nL) for g in graphs]
    outs, st = bt.bt_decompose_batch(h, gs)
    for (e, nU, nL), (sup, phi) in zip(gs, outs):
        s1, p1, _ = bt.bt_decompose(h, e, nU, nL)
        np.testing.assert_array_equal(sup, s1)
        np.testing.assert_array_equal(phi, p1)
        if e.shape[0] <= 20000:
            sr, pr = oracle.bitruss(e, nU, nL)
            np.testing.assert_array_equal(phi.astype(np.uint64), pr)


def test_batch_device_pointers(h):
    torch = pytest.importorskip("torch")
    gs = mixed_graphs()[:10]
    host, _ = bt.bt_decompose_batch(h, gs)
    dgs = [(torch.from_numpy(np.ascontiguousarray(e)).cuda(), nU, nL) for e, nU, nL in gs]
    dev, _ = bt.bt_decompose_batch(h, dgs)
    for (s0, p0), (s1, p1) in zip(host, dev):
        np.testing.assert_array_equal(s0, s1.cpu().numpy().view(np.uint64))
        np.testing.assert_array_equal(p0, p1.cpu().numpy().view(np.uint32))


def test_batch_reports_bad_graph(h):
    gs = mixed_graphs()[:6]
    bad = np.array([[0, 0], [5, 0]], np.int32)  # upper id 5 outside nU = 3
    gs.insert(4, (bad, 3, 3))
    with pytest.raises(bt.BitrussError) as ei:
        bt.bt_decompose_batch(h, gs)
    assert ei.value.code == bt.BT_ERR_RANGE and "graph 4" in str(ei.value)
    # handle still usable
    outs, _ = bt.bt_decompose_batch(h, gs[:4])
    assert len(outs) == 4


def test_128_entry_peel_items_exact(h):
    # 128-entry peel items (four slots a lane, 512-thread blocks) run on
    # indexes of over 2^30 twin pairs; forced here on graphs whose planted
    # dense bicliques give blooms of many pairs, against the oracle
    planted = [synth.chunglu(2000, 1500, 20000, 2.2, 2.5, seed=7, nplant=6, plant_lo=10, plant_hi=40,
                             plant_p=0.9),
               synth.chunglu(5000, 3000, 60000, 2.0, 2.3, seed=9, nplant=10, plant_lo=20, plant_hi=80,
                             plant_p=0.9)]
    gs = [(g.edges, g.nU, g.nL) for g in planted] + [(pins.biclique(40, 50), 40, 50)]
    outs, st = bt.bt_decompose_batch(h, gs, count_threads=512, peel_item=128)
    assert st["peel_item"] == 128
    for (e, nU, nL), (sup, phi) in zip(gs, outs):
        s0, p0 = oracle.bitruss(e, nU, nL)
        np.testing.assert_array_equal(sup, s0)
        np.testing.assert_array_equal(phi.astype(np.uint64), p0)


def test_autotuner_choice_cached_and_schedules_exact(h):
    gs = mixed_graphs()
    h2 = bt.bt_create(0)
    try:
        first, st1 = bt.bt_decompose_batch(h2, gs)
        again, st2 = bt.bt_decompose_batch(h2, gs)
    finally:
        h2.close()
    assert st1["tuned"] == 1 and st2["tuned"] == 2
    assert st1["count_threads"] in (256, 512, 1024) and st1["peel_item"] in (32, 64)
    assert (st1["count_threads"], st1["peel_item"]) == (st2["count_threads"], st2["peel_item"])
    for nt, seg in ((256, 64), (1024, 32), (512, 64), (512, 128)):
        forced, st = bt.bt_decompose_batch(h, gs, count_threads=nt, peel_item=seg)
        assert st["tuned"] == 0 and (st["count_threads"], st["peel_item"]) == (nt, seg)
        for (s0, p0), (s1, p1) in zip(first, forced):
            np.testing.assert_array_equal(s0, s1)
            np.testing.assert_array_equal(p0, p1)
        for (s0, p0), (s1, p1) in zip(first, again):
            np.testing.assert_array_equal(p0, p1)
