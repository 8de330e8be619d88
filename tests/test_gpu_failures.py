"""Failure detection without a GPU fault (no paper counterpart).

Each case makes a bounded wait give up or a host step fail through the
library's test-only limits (bt_set_limits), checks the error the call
returns, and then checks that the same handle still decomposes a graph
exactly (against the CPU oracle):

* the peel's round limit   -> BT_ERR_NOCONVERGE;
* a held grid barrier with a short wait limit -> BT_ERR_CUDA (every block of
  the persistent peel kernel gives up its wait and returns);
* an injected device-allocation failure at every allocation of a call in
  turn -> BT_ERR_NOMEM.
"""
import numpy as np
import pytest

import oracle
from paper_2001_06111_gb300 import bitruss as bt
from paper_2001_06111_gb300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    build.build()
    handle = bt.bt_create(0)
    yield handle
    handle.close()


@pytest.fixture(scope="module")
def g():
    return synth.chunglu(600, 400, 6000, 2.2, 2.4, seed=42)


@pytest.fixture(scope="module")
def ref(g):
    return oracle.bitruss(g.edges, g.nU, g.nL)


def assert_exact(h, g, ref):
    sup, phi, _ = bt.bt_decompose(h, g.edges, g.nU, g.nL)
    np.testing.assert_array_equal(sup, ref[0])
    np.testing.assert_array_equal(phi.astype(np.uint64), ref[1])


def test_round_limit_gives_noconverge(h, g, ref):
    _, _, st = bt.bt_decompose(h, g.edges, g.nU, g.nL)
    assert st["rounds"] > 3
    bt.bt_set_limits(h, peel_round_limit=2)
    with pytest.raises(bt.BitrussError) as ei:
        bt.bt_decompose(h, g.edges, g.nU, g.nL)
    assert ei.value.code == bt.BT_ERR_NOCONVERGE
    bt.bt_set_limits(h)
    assert_exact(h, g, ref)


@pytest.mark.parametrize("barrier", [1, 2, 7])
def test_held_barrier_times_out_and_handle_recovers(h, g, ref, barrier):
    # 50 ms wait limit: block 0 never arrives at the chosen barrier, so every
    # block's bounded wait runs out, raises the error word and returns
    bt.bt_set_limits(h, barrier_timeout_ns=50_000_000, hold_barrier=barrier)
    with pytest.raises(bt.BitrussError) as ei:
        bt.bt_decompose(h, g.edges, g.nU, g.nL)
    assert ei.value.code == bt.BT_ERR_CUDA
    assert "barrier" in str(ei.value)
    bt.bt_set_limits(h)
    assert_exact(h, g, ref)


def test_short_barrier_limit_alone_is_harmless(h, g, ref):
    # a limit far above a barrier's microseconds changes nothing
    bt.bt_set_limits(h, barrier_timeout_ns=1_000_000_000)
    assert_exact(h, g, ref)
    bt.bt_set_limits(h)


def test_allocation_failure_at_each_allocation(h, g, ref):
    failures = 0
    for n in range(1, 400):
        bt.bt_set_limits(h, fail_alloc_at=n)
        try:
            sup, phi, _ = bt.bt_decompose(h, g.edges, g.nU, g.nL)
        except bt.BitrussError as e:
            assert e.code == bt.BT_ERR_NOMEM, (n, e)
            failures += 1
            continue
        # allocation n is beyond the last one of the call: it succeeded
        np.testing.assert_array_equal(sup, ref[0])
        np.testing.assert_array_equal(phi.astype(np.uint64), ref[1])
        break
    else:
        pytest.fail("a decomposition made 400 allocations or more")
    assert failures >= 20
    bt.bt_set_limits(h)
    assert_exact(h, g, ref)


def test_allocation_failure_in_count(h, g, ref):
    bt.bt_set_limits(h, fail_alloc_at=3)
    with pytest.raises(bt.BitrussError) as ei:
        bt.bt_count_support(h, g.edges, g.nU, g.nL)
    assert ei.value.code == bt.BT_ERR_NOMEM
    bt.bt_set_limits(h)
    np.testing.assert_array_equal(bt.bt_count_support(h, g.edges, g.nU, g.nL), ref[0])
