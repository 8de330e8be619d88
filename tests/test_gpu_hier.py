"""GPU parity of the bitruss hierarchy calls (bt_hierarchy, bt_k_bitruss)
against the oracle: the k-bitrusses of Def. 4 as the edges with phi >= k
(Def. 5), bit for bit on the edge order and on every H_k tried."""
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


def test_paper_example_hierarchy(h):
    # Section I / Example 1: H_2 = e0..e5, H_1 = e0..e8, H_0 = all 11 edges
    nU, nL, rows = pins.read_golden(os.path.join(GOLDEN, "paper_example_g.txt"))
    edges = np.array([(int(r[1]), int(r[2])) for r in rows], dtype=np.int32)
    _, phi, _ = bt.bt_decompose(h, edges, nU, nL)
    order, ps = bt.bt_hierarchy(h, phi)
    assert order.tolist() == list(range(11))
    assert ps.tolist() == [2] * 6 + [1] * 3 + [0] * 2
    for k, n in ((0, 11), (1, 9), (2, 6), (3, 0)):
        got = bt.bt_k_bitruss(h, phi, k)
        assert got.tolist() == list(range(n))
        assert got.tolist() == np.flatnonzero(oracle.k_bitruss(edges, nU, nL, k)).tolist()


@pytest.mark.parametrize("seed", range(3))
def test_small_graphs_against_definition(h, seed):
    # H_k by deletion (Def. 4) on the CPU against the GPU selection from GPU phi
    g = synth.random_tiny(300 + seed, 30, 25, 260)
    _, phi, _ = bt.bt_decompose(h, g.edges, g.nU, g.nL)
    for k in range(int(phi.max()) + 2):
        want = np.flatnonzero(oracle.k_bitruss(g.edges, g.nU, g.nL, k))
        np.testing.assert_array_equal(bt.bt_k_bitruss(h, phi, k), want.astype(np.uint32))


def test_workload_order_and_levels(h):
    # the 20k-edge Chung-Lu graph: order against the oracle's stable sort, and
    # every H_k as a prefix of it
    g = synth.small()
    _, phi, _ = bt.bt_decompose(h, g.edges, g.nU, g.nL)
    order, ps = bt.bt_hierarchy(h, phi)
    np.testing.assert_array_equal(order, oracle.hierarchy(phi))
    np.testing.assert_array_equal(ps, phi[order])
    for k in sorted({0, 1, 2, int(phi.max()) // 2, int(phi.max()), int(phi.max()) + 1}):
        sel = bt.bt_k_bitruss(h, phi, k)
        np.testing.assert_array_equal(sel, np.flatnonzero(phi >= k).astype(np.uint32))
        np.testing.assert_array_equal(np.sort(order[: sel.size]), sel)


def test_ragged_sizes_and_device_pointers(h):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    for m in (1, 31, 255, 4097, 1_000_003):  # a few sort tiles and a ragged tail
        phi = rng.integers(0, 1 << 20, size=m).astype(np.uint32)
        phi[rng.integers(0, m, size=m // 3 + 1)] = 7  # many ties
        order, ps = bt.bt_hierarchy(h, phi)
        np.testing.assert_array_equal(order, oracle.hierarchy(phi))
        d = torch.from_numpy(phi.view(np.int32)).cuda().view(torch.uint32)
        dorder, dps = bt.bt_hierarchy(h, d)
        np.testing.assert_array_equal(dorder.cpu().view(torch.int32).numpy().view(np.uint32), order)
        np.testing.assert_array_equal(dps.cpu().view(torch.int32).numpy().view(np.uint32), ps)
        for k in (0, 7, 8, 1 << 19, 1 << 21):
            want = np.flatnonzero(phi >= k).astype(np.uint32)
            np.testing.assert_array_equal(bt.bt_k_bitruss(h, phi, k), want)
            dsel = bt.bt_k_bitruss(h, d, k)
            np.testing.assert_array_equal(dsel.cpu().view(torch.int32).numpy().view(np.uint32), want)


def test_empty_and_errors(h):
    order, ps = bt.bt_hierarchy(h, np.zeros(0, np.uint32))
    assert order.size == 0 and ps.size == 0
    assert bt.bt_k_bitruss(h, np.zeros(0, np.uint32), 3).size == 0
    lib = bt.load()
    assert lib.bt_hierarchy(h.ptr, None, 5, None, None, 0) == bt.BT_ERR_ARG
    phi = np.zeros(4, np.uint32)
    out = np.zeros(4, np.uint32)
    assert lib.bt_hierarchy(h.ptr, phi.ctypes.data, 4, out.ctypes.data, None, 1 << 7) == bt.BT_ERR_ARG
