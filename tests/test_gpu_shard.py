"""The single-graph counting shard on one GPU (bt_count_support_part): each
part's supports equal the CPU oracle's supports from the butterflies anchored
in the part's priority-rank range (Lemma 3, Def. 7), the ranges tile all
ranks, and the parts add up to the full supports.  The sum over processes
(shard.count_support_sharded) runs here as a one-process group; its
two-process reduction is covered on the CPU by tests/test_dist_cpu.py."""
import os
import socket

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


def check_parts(h, edges, nU, nL, nparts, flags=0):
    lower_first = bool(flags & bt.BT_TIE_LOWER_FIRST)
    total = np.zeros(edges.shape[0], dtype=np.uint64)
    prev_hi = 0
    for p in range(nparts):
        sup, lo, hi = bt.bt_count_support_part(h, edges, nU, nL, p, nparts, flags=flags)
        assert lo == prev_hi and lo <= hi
        prev_hi = hi
        np.testing.assert_array_equal(sup, oracle.support_anchored(edges, nU, nL, lo, hi, lower_first))
        total += sup
    assert prev_hi == nU + nL
    np.testing.assert_array_equal(total, oracle.support(edges, nU, nL))
    np.testing.assert_array_equal(total, bt.bt_count_support(h, edges, nU, nL, flags=flags))


def test_paper_example_parts(h):
    nU, nL, rows = pins.read_golden(os.path.join(GOLDEN, "paper_example_anchored.txt"))
    edges = np.array([(int(r[1]), int(r[2])) for r in rows], dtype=np.int32)
    for flags in (0, bt.BT_TIE_LOWER_FIRST):
        for nparts in (1, 2, 3):
            check_parts(h, edges, nU, nL, nparts, flags)
    # the top vertex u2 (rank 8) alone: its three butterflies
    sup, lo, hi = bt.bt_count_support_part(h, edges, nU, nL, 1, 2)
    if (lo, hi) == (8, 9):
        assert sup.tolist() == [int(r[3]) for r in rows]


@pytest.mark.parametrize("nparts", [1, 2, 3, 5, 8])
def test_small_workload_parts(h, nparts):
    g = synth.small()
    check_parts(h, g.edges, g.nU, g.nL, nparts)


def test_medium_sample_parts_balanced(h):
    g = synth.vertex_sample(synth.medium(), 0.2, 7)
    check_parts(h, g.edges, g.nU, g.nL, 4)
    # the ranges hold about equal numbers of priority-obeyed wedges: the top
    # range (hubs) is short and the bottom one long
    ranges = [bt.bt_count_support_part(h, g.edges, g.nU, g.nL, p, 4)[1:] for p in range(4)]
    widths = [hi - lo for lo, hi in ranges]
    assert widths[0] > widths[-1]


def test_device_pointers_and_errors(h):
    torch = pytest.importorskip("torch")
    g = synth.small()
    d = torch.from_numpy(g.edges).cuda()
    sup_d, lo, hi = bt.bt_count_support_part(h, d, g.nU, g.nL, 1, 3)
    sup_h, lo2, hi2 = bt.bt_count_support_part(h, g.edges, g.nU, g.nL, 1, 3)
    assert (lo, hi) == (lo2, hi2)
    np.testing.assert_array_equal(sup_d.cpu().numpy().view(np.uint64), sup_h)
    with pytest.raises(bt.BitrussError) as ei:
        bt.bt_count_support_part(h, g.edges, g.nU, g.nL, 3, 3)
    assert ei.value.code == bt.BT_ERR_ARG


def test_sharded_helper_one_process_group(h):
    torch = pytest.importorskip("torch")
    import torch.distributed as dist
    from paper_2001_06111_gb300 import shard
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        g = synth.small()
        sup = shard.count_support_sharded(g.edges, g.nU, g.nL, handle=h)
        np.testing.assert_array_equal(sup, oracle.support(g.edges, g.nU, g.nL))
    finally:
        dist.destroy_process_group()
