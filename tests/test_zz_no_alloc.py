"""The allocation-free support count (bt_count_support_static).

It serves callers that cannot allocate device memory around a library call
(a host framework that owns and accounts for all GPU memory, or a
latency-critical loop that must avoid the synchronisation an allocation can
cause): scratch comes from a fixed array inside the library.  Its results
must equal those of the allocating entry point, bit for bit, on consecutive
calls that reuse the shared array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_2001_06111_gb300 import bitruss as bt
from paper_2001_06111_gb300 import build, synth

pytestmark = pytest.mark.gpu


def test_static_count_matches_allocating_count_on_two_calls():
    torch = pytest.importorskip("torch")
    build.build()
    graphs = [synth.chunglu(60000, 40000, 250000, 2.1, 2.4, seed=21, cap=5000),
              synth.small()]
    with bt.bt_create(0) as h:
        for g in graphs:
            want = bt.bt_count_support(h, g.edges, g.nU, g.nL)
            d_edges = torch.from_numpy(g.edges).cuda()
            d_sup = torch.full((g.m,), -1, dtype=torch.int64, device="cuda")
            bt.bt_count_support_static(d_edges, g.nU, g.nL, d_sup)
            got = d_sup.cpu().numpy().view(np.uint64)
            np.testing.assert_array_equal(got, want)
            # and the definition itself: the CPU oracle's direct enumeration
            np.testing.assert_array_equal(got, oracle.support(g.edges, g.nU, g.nL))


def test_static_count_rejects_oversize_graph():
    torch = pytest.importorskip("torch")
    build.build()
    d_edges = torch.zeros((300000, 2), dtype=torch.int32, device="cuda")
    d_sup = torch.empty(300000, dtype=torch.int64, device="cuda")
    with pytest.raises(bt.BitrussError) as ei:
        bt.bt_count_support_static(d_edges, 1000, 1000, d_sup)
    assert ei.value.code == bt.BT_ERR_TOO_LARGE
