"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point include/*.h declares; the host-only estimator
counts priority-obeyed wedges (Def. 10) like an independent numpy count."""
import glob
import os
import re

import numpy as np
import pytest

from paper_2001_06111_gb300 import bitruss, build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(bt_[a-z_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return bitruss.load()


def test_header_declares_the_path(lib):
    names = declared_functions()
    for want in ("bt_count_support", "bt_build_index", "bt_decompose", "bt_create", "bt_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(bitruss.EXPORTED) <= declared_functions() | {"bt_last_error"}


def _wedges_numpy(edges, nU, nL, lower_first=False):
    e = np.asarray(edges, dtype=np.int64)
    n = nU + nL
    gu = e[:, 0] if lower_first else nL + e[:, 0]
    gv = nU + e[:, 1] if lower_first else e[:, 1]
    deg = np.bincount(np.concatenate([gu, gv]), minlength=n)
    order = np.lexsort((np.arange(n), deg))
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    ru, rv = rank[gu], rank[gv]
    nbr = [[] for _ in range(n)]
    for a, b in zip(ru, rv):
        nbr[a].append(b)
        nbr[b].append(a)
    W = 0
    for u in range(n):
        for v in nbr[u]:
            if v < u:
                W += sum(1 for w in nbr[v] if w < u)
    return W


@pytest.mark.parametrize("lower_first", [False, True])
def test_estimate_counts_wedges(lib, lower_first):
    g = synth.chunglu(300, 200, 2500, 2.2, 2.4, seed=4)
    flags = bitruss.BT_TIE_LOWER_FIRST if lower_first else 0
    nbytes, W = bitruss.bt_estimate_bytes(g.edges, g.nU, g.nL, flags)
    assert W == _wedges_numpy(g.edges, g.nU, g.nL, lower_first)
    assert nbytes > 16 * W


def test_estimate_rejects_bad_ids(lib):
    with pytest.raises(bitruss.BitrussError):
        bitruss.bt_estimate_bytes(np.array([[0, 5]], np.int32), 1, 2)
