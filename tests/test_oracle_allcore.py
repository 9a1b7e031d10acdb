"""The oracle's all-core driver equals its single-threaded functions (CPU).

The all-core functions only cut an independent outer loop (table rows, path
ids, index vertices, queries) into ranges, one POSIX thread each; their
results must be identical to the single-threaded oracle, which the other CPU
pins hold to the paper. Thread counts that do not divide the ranges evenly
(3, 7) and more threads than items are included.
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def g():
    return synth.chung_lu(3000, 9, 2.2, ("uniform", 1, 40), seed=11)


@pytest.mark.parametrize("threads", [2, 3, 7])
def test_tables_paths_index(g, threads):
    t1 = oracle.alias_tables(g)
    tn = oracle.alias_tables(g, threads=threads)
    assert np.array_equal(t1[0], tn[0]) and np.array_equal(t1[1], tn[1])
    for mode in (oracle.PREFIX, oracle.ALIAS):
        for r0, R, T in ((0, 30_000, 5), (123_456, 7_777, 3), (2**33 + 5, 1_001, 9)):
            p1 = oracle.sample_paths(g, 9, R, T, mode, r0=r0, tables=t1)
            pn = oracle.sample_paths(g, 9, R, T, mode, r0=r0, tables=tn, threads=threads)
            assert np.array_equal(p1, pn), (mode, r0, R, T)
    off1, pid1 = oracle.build_index(g.n, p1)
    offn, pidn = oracle.build_index(g.n, p1, threads=threads)
    assert np.array_equal(off1, offn) and np.array_equal(pid1, pidn)


@pytest.mark.parametrize("threads", [3, 7])
def test_topk_and_theta(g, threads):
    P = oracle.sample_paths(g, 4, 40_000, 5, oracle.ALIAS)
    o = oracle.Oracle(g.n, P)
    q = np.concatenate([np.arange(0, g.n, 3), [0, 0, 1]]).astype(np.int32)   # repeats allowed
    for k in (1, 10, 64):
        a = o.topk_many(q, k)
        b = o.topk_many(q, k, threads=threads)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(o.theta_all(30), o.theta_all(30, threads=threads))


def test_more_threads_than_items():
    g = synth.graph_from_edges(4, [(0, 1), (1, 2), (2, 3)], [1, 2, 3])
    p1 = oracle.sample_paths(g, 1, 5, 4, oracle.ALIAS)
    pn = oracle.sample_paths(g, 1, 5, 4, oracle.ALIAS, threads=16)
    assert np.array_equal(p1, pn)
    off1, pid1 = oracle.build_index(g.n, p1)
    offn, pidn = oracle.build_index(g.n, p1, threads=16)
    assert np.array_equal(off1, offn) and np.array_equal(pid1, pidn)
    o = oracle.Oracle(g.n, p1)
    a = o.topk_many(np.arange(4, dtype=np.int32), 3)
    b = o.topk_many(np.arange(4, dtype=np.int32), 3, threads=16)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_knn_many(g):
    P = oracle.sample_paths(g, 4, 40_000, 5, oracle.ALIAS)
    th = oracle.Oracle(g.n, P).theta_all(20)
    q = np.arange(0, g.n, 5, dtype=np.int32)
    ids, d2 = oracle.knn_many(th, q, 7, threads=3)
    for i, v in enumerate(q):
        a, b = oracle.knn(th, int(v), 7)
        assert np.array_equal(ids[i], a) and np.array_equal(d2[i], b)
