"""Pins of the oracle's index-free counting (no GPU).

oracle.stream_counts restates Eq. (4) from its definition, path by path, for
path sets too large to hold (R above 2^31 - 1, the sample sizes the paper's
eps = sqrt(1/|E|) gives on its largest networks, Sec. 3.4 and Table 2).
oracle.paths_at draws single paths by id. Each test checks them against
something other than themselves: a brute-force incidence-matrix product, a
closed form, the index-based route of the oracle, and the invariance of sums
under the split of the path range.
"""
import numpy as np
import pytest

import oracle
import synth


def _graph():
    return synth.chung_lu(400, 6, 2.5, ("uniform", 1, 16), seed=3)


@pytest.mark.parametrize("mode", [oracle.PREFIX, oracle.ALIAS])
def test_stream_counts_equal_incidence_product(mode):
    # cnt(v, u) = number of paths holding both v and u: with the 0/1
    # path-vertex incidence matrix M (R x n), that is (M^T M)[v, u] for
    # u != v, and |P_v| is the column sum of M
    g = _graph()
    R, T = 6000, 4
    paths = oracle.sample_paths(g, 9, R, T, mode)
    M = np.zeros((R, g.n), dtype=np.float64)
    M[np.repeat(np.arange(R), T + 1), paths.ravel()] = 1.0
    C = (M.T @ M).astype(np.int64)             # exact: entries <= R < 2^53
    q = np.arange(g.n, dtype=np.int32)
    cnt, npaths = oracle.stream_counts(g, 9, 0, R, T, q, mode, threads=3)
    assert np.array_equal(npaths, M.sum(axis=0).astype(np.int64))
    np.fill_diagonal(C, 0)                     # the query itself is never a candidate
    assert np.array_equal(cnt.astype(np.int64), C)


def test_stream_topk_equals_index_route():
    # the same top-k through the inverted index (Algorithm 1 over P_v)
    g = _graph()
    R, T, k = 5000, 5, 12
    paths = oracle.sample_paths(g, 4, R, T, oracle.ALIAS)
    O = oracle.Oracle(g.n, paths)
    q = np.array([0, 7, 33, 399, 120], dtype=np.int32)
    cnt, npaths = oracle.stream_counts(g, 4, 0, R, T, q, oracle.ALIAS)
    assert np.array_equal(npaths, np.diff(O.off))
    for i, v in enumerate(q):
        ids, c = oracle.topk_from_counts(cnt[i], int(v), k)
        ref_ids, ref_c = O.topk(int(v), k)
        assert np.array_equal(ids, ref_ids)
        assert np.array_equal(c.astype(np.uint32), ref_c)


def test_stream_split_invariance_and_offset_ranges():
    # sums over a range equal the sums over any split of it, for any thread
    # count; ranges far from 0 draw with their own global path ids
    g = _graph()
    T = 3
    q = np.array([5, 6, 250], dtype=np.int32)
    r0 = 2**31 - 1500
    a, na = oracle.stream_counts(g, 2, r0, r0 + 3000, T, q, threads=1)
    b, nb = oracle.stream_counts(g, 2, r0, r0 + 3000, T, q, threads=4)
    c1, n1 = oracle.stream_counts(g, 2, r0, r0 + 1234, T, q)
    c2, n2 = oracle.stream_counts(g, 2, r0 + 1234, r0 + 3000, T, q)
    assert np.array_equal(a, b) and np.array_equal(na, nb)
    assert np.array_equal(a, c1 + c2) and np.array_equal(na, n1 + n2)
    # and they match the stored paths of the same ids
    paths = oracle.sample_paths(g, 2, 3000, T, r0=r0)
    M = np.zeros((3000, g.n), dtype=np.int64)
    M[np.repeat(np.arange(3000), T + 1), paths.ravel()] = 1
    assert np.array_equal(na, M.sum(axis=0))


def test_stream_two_vertex_closed_form():
    # one edge {0, 1}: every path alternates between the two vertices, so
    # both lie on all R paths and cnt(0, 1) = cnt(1, 0) = R
    g = synth.graph_from_edges(2, [(0, 1)], [5])
    R, T = 777, 5
    cnt, npaths = oracle.stream_counts(g, 1, 10**12, 10**12 + R, T, np.array([0, 1], np.int32), oracle.ALIAS)
    assert npaths.tolist() == [R, R]
    assert cnt.tolist() == [[0, R], [R, 0]]
    ids, c = oracle.topk_from_counts(cnt[0], 0, 3)
    assert ids.tolist() == [1, -1, -1] and c.tolist() == [R, 0, 0]


def test_stream_rejects_repeated_queries():
    g = _graph()
    with pytest.raises(ValueError):
        oracle.stream_counts(g, 1, 0, 10, 2, np.array([3, 3], np.int32))


@pytest.mark.parametrize("mode", [oracle.PREFIX, oracle.ALIAS])
def test_paths_at_equals_sampled_rows(mode):
    # single paths drawn by id equal the rows of a range draw, across 2^31
    g = _graph()
    T, r0, R = 6, 2**31 - 40, 80
    rows = oracle.sample_paths(g, 8, R, T, mode, r0=r0)
    ids = np.array([r0 + 79, r0, r0 + 40, r0 + 39, r0 + 40], dtype=np.int64)
    got = oracle.paths_at(g, 8, ids, T, mode, threads=2)
    assert np.array_equal(got, rows[ids - r0])


def test_topk_from_counts_order_and_padding():
    # (count desc, id asc), the query and zero counts excluded
    row = np.array([9, 0, 4, 9, 4, 1], dtype=np.uint64)
    ids, c = oracle.topk_from_counts(row, 0, 5)
    assert ids.tolist() == [3, 2, 4, 5, -1]
    assert c.tolist() == [9, 4, 4, 1, 0]
