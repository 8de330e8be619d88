"""The 30M-edge workload with 200 planted dense bicliques (deep peeling levels,
large blooms): exact parity on a vertex-induced sample, and at full size the
supports of sampled edges (recomputed one by one by the oracle), the local
fixpoint property of phi on sampled edges, phi <= support and
4 x butterflies = sum of supports."""
import numpy as np
import pytest

import oracle
from paper_2001_06111_gb300 import bitruss as bt
from paper_2001_06111_gb300 import build, synth
from tests.digests import assert_matches_digest, oracle_digest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def large():
    build.build()
    return synth.large()


@pytest.fixture(scope="module")
def h():
    build.build()
    handle = bt.bt_create(0)
    yield handle
    handle.close()


def test_large_vertex_sample_exact(h, large):
    g = synth.vertex_sample(large, 0.07, 5)
    sup, phi, _ = bt.bt_decompose(h, g.edges, g.nU, g.nL)
    sr, pr = oracle.bitruss(g.edges, g.nU, g.nL)
    np.testing.assert_array_equal(sup, sr)
    np.testing.assert_array_equal(phi.astype(np.uint64), pr)


def test_large_vertex_sample_exact_digest(h, large):
    """The largest vertex-induced sample of the 30M-edge workload the oracle
    finishes in about half an hour (its digests are computed offline): every
    support and bitruss number equals the oracle's.  The full 30M-edge graph
    is beyond the oracle; there it is checked by the properties below."""
    ref = oracle_digest("large-sample")
    g = synth.vertex_sample(large, ref["sample"]["frac"], ref["sample"]["seed"])
    sup, phi, _ = bt.bt_decompose(h, g.edges, g.nU, g.nL)
    assert_matches_digest(g, sup, phi, ref)


def test_large_full_size_properties(h, large):
    g = large
    sup, phi, st = bt.bt_decompose(h, g.edges, g.nU, g.nL)
    assert (phi.astype(np.uint64) <= sup).all()
    stats = bt.bt_build_index(h, g.edges, g.nU, g.nL)
    assert stats["n_butterflies"] * 4 == int(sup.sum())
    du = np.bincount(g.edges[:, 0], minlength=g.nU).astype(np.int64)
    dl = np.bincount(g.edges[:, 1], minlength=g.nL).astype(np.int64)
    cost = du[g.edges[:, 0]] * dl[g.edges[:, 1]]
    rng = np.random.default_rng(17)
    cheap = np.nonzero(cost <= 20_000_000)[0]
    which = np.sort(rng.choice(cheap, 300, replace=False)).astype(np.uint64)
    # include edges of the highest phi levels (inside planted bicliques)
    top = np.argsort(phi)[-20:].astype(np.uint64)
    which = np.unique(np.concatenate([which, top[cost[top] <= 200_000_000]]))
    np.testing.assert_array_equal(sup[which], oracle.support_sampled(g.edges, g.nU, g.nL, which))
    cnt, hv = oracle.local_check(g.edges, g.nU, g.nL, phi, which)
    assert (cnt >= phi[which]).all()
    np.testing.assert_array_equal(hv, phi[which].astype(np.uint64))
