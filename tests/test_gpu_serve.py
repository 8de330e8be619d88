"""Serving with continuous batching (bt_server_*): requests that arrive while
the GPU is busy are batched together, every result equals the graph's
decomposition alone, and results of requests small enough for the CPU oracle
(<= 20,000 edges) equal the oracle's exactly."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2001_06111_gb300 import bitruss as bt
from paper_2001_06111_gb300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def alone():
    build.build()
    h = bt.bt_create(0)
    yield lambda e, nU, nL: bt.bt_decompose(h, e, nU, nL)[:2]
    h.close()


def test_requests_batched_while_busy_and_exact(alone):
    big = synth.vertex_sample(synth.medium(), 0.5, 3)  # keeps the worker busy
    small = [synth.batch_graph(i, hi=20000) for i in range(30)]
    with bt.Server(0, workers=1) as srv:
        ids = [srv.submit(big.edges, big.nU, big.nL, want_support=True)]
        ids += [srv.submit(g.edges, g.nU, g.nL, want_support=True) for g in small]
        results = [srv.poll(i, wait=True) for i in ids]
        st = srv.stats()
    assert st["completed"] == 31 and st["rejected"] == 0
    assert st["max_batch_graphs"] >= 2 and st["batches"] < 31
    for (info, (sup, phi)), g in zip(results, [big] + small):
        assert info["status"] == bt.BT_OK
        s1, p1 = alone(g.edges, g.nU, g.nL)
        np.testing.assert_array_equal(sup, s1)
        np.testing.assert_array_equal(phi, p1)
        if g.m <= 20000:
            sr, pr = oracle.bitruss(g.edges, g.nU, g.nL)
            np.testing.assert_array_equal(sup, sr)
            np.testing.assert_array_equal(phi.astype(np.uint64), pr)


def test_concurrent_workers_exact(alone):
    gs = [synth.batch_graph(100 + i, hi=50000) for i in range(24)]
    with bt.Server(0, workers=2) as srv:
        ids = [srv.submit(g.edges, g.nU, g.nL) for g in gs]
        res = [srv.poll(i, wait=True) for i in ids]
    for (info, (_, phi)), g in zip(res, gs):
        assert info["status"] == bt.BT_OK and info["latency_seconds"] >= info["queue_seconds"] >= 0
        np.testing.assert_array_equal(phi, alone(g.edges, g.nU, g.nL)[1])


def test_admission_rejects_oversized_request():
    build.build()
    g = synth.small()
    with bt.Server(0, memory_budget_bytes=1 << 20, workers=1) as srv:
        rid = srv.submit(g.edges, g.nU, g.nL)
        info, _ = srv.poll(rid, wait=True)
        assert info["status"] == bt.BT_ERR_NOMEM
        assert srv.stats()["rejected"] == 1


def test_large_requests_alone_small_ones_pass(alone):
    # threshold 30k edges: two large graphs, then small ones.  Large requests
    # run in batches of their own, the small-first worker takes the small ones
    # while the large ones run, and every result is exact.
    large = [synth.vertex_sample(synth.medium(), 0.3, s) for s in (5, 6)]
    small = [synth.batch_graph(200 + i, hi=20000) for i in range(20)]
    assert all(g.m >= 30000 for g in large) and all(g.m < 30000 for g in small)
    with bt.Server(0, workers=2, large_edges=30000) as srv:
        ids = [srv.submit(g.edges, g.nU, g.nL) for g in large + small]
        res = [srv.poll(i, wait=True) for i in ids]
        st = srv.stats()
    assert st["completed"] == 22 and st["batches"] >= 3
    for (info, (_, phi)), g in zip(res, large + small):
        assert info["status"] == bt.BT_OK
        np.testing.assert_array_equal(phi, alone(g.edges, g.nU, g.nL)[1])


def test_nonblocking_polls_while_batches_complete():
    """Polls with wait=0 in tight loops from several threads while workers
    finish batches: a request is reported (and released) only once its result
    and completion time are both published, and every result matches the
    oracle."""
    build.build()
    gs = [synth.batch_graph(300 + i, hi=8000) for i in range(48)]
    ref = [oracle.bitruss(g.edges, g.nU, g.nL) for g in gs]
    out = [None] * len(gs)
    with bt.Server(0, workers=2) as srv:
        ids = [srv.submit(g.edges, g.nU, g.nL, want_support=True) for g in gs]

        def poller(part):
            for i in part:
                t_end = time.time() + 120
                while True:
                    info, res = srv.poll(ids[i], wait=False)
                    if info["done"]:
                        out[i] = (info, res)
                        break
                    assert time.time() < t_end
        th = [threading.Thread(target=poller, args=(range(t, len(gs), 4),)) for t in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
    for (info, (sup, phi)), (sr, pr) in zip(out, ref):
        assert info["status"] == bt.BT_OK
        assert info["latency_seconds"] >= info["queue_seconds"] >= 0
        np.testing.assert_array_equal(sup, sr)
        np.testing.assert_array_equal(phi.astype(np.uint64), pr)


def test_cancel_queued_requests():
    """Requests still waiting when the queue is cancelled complete with
    BT_ERR_CANCELLED; the ones already in a batch finish exactly."""
    build.build()
    big = synth.vertex_sample(synth.medium(), 0.5, 3)  # keeps the one worker busy
    small = [synth.batch_graph(400 + i, hi=5000) for i in range(20)]
    with bt.Server(0, workers=1) as srv:
        ids = [srv.submit(big.edges, big.nU, big.nL)]
        ids += [srv.submit(g.edges, g.nU, g.nL) for g in small]
        time.sleep(0.05)
        n = srv.cancel_queued()
        res = [srv.poll(i, wait=True) for i in ids]
    assert n >= 1
    statuses = [info["status"] for info, _ in res]
    assert statuses.count(bt.BT_ERR_CANCELLED) == n
    for (info, (_, phi)), g in zip(res, [big] + small):
        if info["status"] == bt.BT_OK and g.m <= 20000:
            np.testing.assert_array_equal(phi.astype(np.uint64), oracle.bitruss(g.edges, g.nU, g.nL)[1])


def test_large_requests_share_a_batch(alone):
    """With large_batch = 2, large requests waiting behind a busy worker are
    decomposed together, each exactly as alone."""
    large = [synth.vertex_sample(synth.medium(), 0.3, s) for s in (5, 6, 8)]
    with bt.Server(0, workers=1, large_edges=30000, large_batch=2) as srv:
        ids = [srv.submit(g.edges, g.nU, g.nL) for g in large]
        res = [srv.poll(i, wait=True) for i in ids]
        st = srv.stats()
    assert st["max_batch_graphs"] == 2
    for (info, (_, phi)), g in zip(res, large):
        assert info["status"] == bt.BT_OK
        np.testing.assert_array_equal(phi, alone(g.edges, g.nU, g.nL)[1])
