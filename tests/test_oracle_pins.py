"""Pins of the CPU oracle to the paper and to mathematics (no GPU).

Each test checks the oracle against something other than itself: a closed
form, an exhaustive enumeration, exact rational path probabilities, brute force
over all vertex pairs, or an invariant the paper's definitions imply. The
paper (arXiv 1504.02577) prints no worked numeric example, so nothing here is
pinned to printed outputs.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

# --------------------------------------------------------------- Sec. 3.2 ---

def test_sample_size_paper_defaults():
    # Sec. 3.2: R = c/eps^2 (log2 C(T,2) + 1 + ln 1/delta), with the paper's
    # c = 0.5, delta = 0.1, T = 5 (Implementation Notes) and eps = 0.01:
    # log2(10) = 3.32192809..., ln(10) = 2.30258509..., sum + 1 = 6.62451318...
    # 0.5 * 10^4 * 6.62451318 = 33122.57 -> 33123 paths.
    assert oracle.sample_size(0.01, 0.1, 0.5, 5) == 33123


def test_sample_size_tencent6_rule():
    # eps = sqrt(1/|E|) makes R = ceil(0.5 |E| * 6.62451318...); Tencent6 has
    # |E| = 5,000,000 (Table 2): 16,561,282.97 -> 16,561,283.
    assert oracle.sample_size(math.sqrt(1 / 5_000_000), 0.1, 0.5, 5) == 16_561_283


def test_sample_size_reduces_to_theorem1_with_d1():
    # T = 2: C(2,2) = 1, log2(1) = 0, so the VC bound is d = 1 and the
    # formula is Theorem 1 with d = 1: c/eps^2 (1 + ln 1/delta).
    # eps = 0.05, delta = 0.2, c = 0.7: 280 * (1 + 1.6094379) = 730.64 -> 731.
    assert oracle.sample_size(0.05, 0.2, 0.7, 2) == 731
    # T = 3: C(3,2) = 3 -> d = log2(3) + 1 = 2.5849625; eps = 0.1, delta = 0.5,
    # c = 1: 100 * (2.5849625 + 0.6931472) = 327.81 -> 328.
    assert oracle.sample_size(0.1, 0.5, 1.0, 3) == 328


def test_sample_size_scaling_and_domain():
    a = oracle.sample_size(0.02, 0.1, 0.5, 5)
    b = oracle.sample_size(0.01, 0.1, 0.5, 5)
    assert abs(b - 4 * a) <= 4                          # R grows as 1/eps^2
    assert oracle.sample_size(0.01, 0.1, 1.0, 5) in (2 * b - 1, 2 * b)  # linear in c
    assert oracle.sample_size(0.01, 0.1, 0.5, 1) == -1   # C(1,2) = 0: undefined
    assert oracle.sample_size(0.0, 0.1, 0.5, 5) == -1
    assert oracle.sample_size(0.01, 1.0, 0.5, 5) == -1


# ---------------------------------------------------------------- Philox ---

def test_philox_is_a_bijection_on_a_sample():
    key = (0x12345678, 0x9ABCDEF0)
    outs = set()
    for i in range(20000):
        outs.add(tuple(oracle.philox4x32_10((i, 0, 7, 0), key)))
    assert len(outs) == 20000


def test_philox_output_is_uniform_and_avalanches():
    from scipy.stats import chisquare
    key = (1, 0)
    words = np.array([oracle.philox4x32_10((i, 0, 0, 0), key) for i in range(8192)], dtype=np.uint32)
    by = words.view(np.uint8).ravel()
    _, p = chisquare(np.bincount(by, minlength=256))
    assert p > 1e-4
    # one flipped counter bit changes about half of the 128 output bits
    flips = []
    for i in range(512):
        a = oracle.philox4x32_10((i, 5, 6, 7), key)
        b = oracle.philox4x32_10((i ^ 1 << (i % 32), 5, 6, 7), key)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert 60 < np.mean(flips) < 68


def test_draw_counter_layout():
    # draw(seed, stream, r, t, attempt) = Philox(ctr=(r_lo, r_hi, stream<<16|t, attempt), key=seed)
    seed = 0x0123456789ABCDEF
    r = (5 << 32) | 17
    d = oracle.draw(seed, 3, r, 4, 2)
    p = oracle.philox4x32_10((17, 5, (3 << 16) | 4, 2), (0x89ABCDEF, 0x01234567))
    assert (d == p).all()


# ---------------------------------------------------------------- Lemire ---

def test_lemire_matches_exact_integer_definition():
    rng = np.random.default_rng(7)
    for _ in range(4000):
        U = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        S = int(rng.integers(1, 2**40)) if rng.random() < 0.5 else int(rng.integers(1, 64))
        ok, v = oracle.lemire(U, S)
        prod = U * S
        accept = (prod % 2**64) >= (2**64 % S)
        assert ok == accept
        if ok:
            assert v == prod >> 64 and 0 <= v < S


def test_lemire_power_of_two_and_unit_ranges():
    rng = np.random.default_rng(3)
    for _ in range(1000):
        U = int(rng.integers(0, 2**63)) * 2 + 1
        b = int(rng.integers(0, 64))
        ok, v = oracle.lemire(U, 2**b)
        assert ok and v == U >> (64 - b)
        assert oracle.lemire(U, 1) == (True, 0)


def test_lemire_rejection_branch():
    # S = 2^63 + 1: 2^64 mod S = 2^63 - 1, so about half of all U are rejected.
    S = 2**63 + 1
    rej = 0
    rng = np.random.default_rng(11)
    for _ in range(2000):
        U = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        ok, v = oracle.lemire(U, S)
        rej += not ok
        if ok:
            assert v < S
    assert 850 < rej < 1150


# ------------------------------------------------------------- Eq. (3) ---

def _rows(seed=0, n=60):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        d = int(rng.integers(1, 8))
        yield rng.integers(1, 10, size=d).astype(np.uint32)


def test_prefix_selection_realises_eq3_exactly():
    # Every x in [0, S) is one equally likely draw; neighbour j must receive
    # exactly w_j of them, i.e. probability w_j / S = t_ij (Eq. 3).
    for w in _rows(1):
        S = int(w.sum())
        hits = np.zeros(len(w), dtype=np.int64)
        for x in range(S):
            hits[oracle.select_prefix(w, x)] += 1
        assert (hits == w.astype(np.int64)).all()


def test_alias_selection_realises_eq3_exactly():
    # Every (column c, coin u) in [0,d) x [0,S) is one equally likely draw;
    # neighbour j must receive exactly w_j * d of them (probability w_j / S).
    for w in _rows(2):
        d, S = len(w), int(w.sum())
        thr, al = oracle.alias_row(w)
        assert (thr <= S).all() and ((al >= 0) & (al < d)).all()
        hits = np.zeros(d, dtype=np.int64)
        for c in range(d):
            for u in range(S):
                hits[oracle.select_alias(thr, al, c, u)] += 1
        assert (hits == w.astype(np.int64) * d).all()


def test_alias_table_large_weights_exact():
    # Unequal large weights: count hits per column analytically (each column c
    # sends thr[c] coins to c and S - thr[c] coins to alias[c]).
    rng = np.random.default_rng(5)
    for _ in range(20):
        d = int(rng.integers(2, 400))
        w = rng.integers(1, 2**20, size=d).astype(np.uint32)
        S = int(w.sum())
        thr, al = oracle.alias_row(w)
        hits = np.zeros(d, dtype=object)
        for c in range(d):
            hits[c] += int(thr[c])
            hits[int(al[c])] += S - int(thr[c])
        assert all(int(hits[j]) == int(w[j]) * d for j in range(d))


# ------------------------------------------------- Algorithm 3 + Eq. (1) ---

TINY_EDGES = [(0, 1), (0, 2), (1, 2), (2, 3), (3, 4), (1, 4)]
TINY_W = [3, 1, 2, 5, 1, 4]


def _tiny():
    return synth.graph_from_edges(5, TINY_EDGES, TINY_W)


def _enumerate_paths(g, T):
    """All T-paths with their exact probability phi(p) = (1/N) prod t (Sec. 3.1, 3.2)."""
    out = {}
    for v0 in range(g.n):
        stack = [((v0,), Fraction(1, g.n))]
        while stack:
            p, pr = stack.pop()
            if len(p) == T + 1:
                out[p] = out.get(p, 0) + pr
                continue
            v = p[-1]
            s, e = g.row_ptr[v], g.row_ptr[v + 1]
            if e == s:
                stack.append((p + (v,), pr))
                continue
            tot = int(g.w[s:e].sum())
            for j in range(s, e):
                stack.append((p + (int(g.col[j]),), pr * Fraction(int(g.w[j]), tot)))
    return out


@pytest.mark.parametrize("mode", [oracle.PREFIX, oracle.ALIAS])
def test_path_distribution_matches_enumeration(mode):
    from scipy.stats import chisquare
    g = _tiny()
    T = 3
    exact = _enumerate_paths(g, T)
    assert sum(exact.values()) == 1
    R = 120_000
    P = oracle.sample_paths(g, 42, R, T, mode)
    # every step follows an edge
    for t in range(T):
        a, b = P[:, t], P[:, t + 1]
        for x, y in set(zip(a.tolist(), b.tolist())):
            assert y in g.col[g.row_ptr[x]:g.row_ptr[x + 1]]
    keys = list(exact)
    idx = {k: i for i, k in enumerate(keys)}
    obs = np.zeros(len(keys))
    for row in map(tuple, P.tolist()):
        obs[idx[row]] += 1
    exp = np.array([float(exact[k]) * R for k in keys])
    _, p = chisquare(obs, exp)
    assert p > 1e-4


def test_estimator_converges_to_eq1():
    # Eq. (1) computed exactly by enumeration vs the estimate |P_vi,vj| / R of
    # Eq. (4); Hoeffding with a union bound over the C(5,2) pairs at 1e-6.
    g = _tiny()
    T = 3
    exact = _enumerate_paths(g, T)
    S = {}
    for p, pr in exact.items():
        u = sorted(set(p))
        for a, b in itertools.combinations(u, 2):
            S[(a, b)] = S.get((a, b), 0) + pr
    R = 200_000
    P = oracle.sample_paths(g, 9, R, T, oracle.ALIAS)
    o = oracle.Oracle(g.n, P)
    tol = math.sqrt(math.log(2 * 10 / 1e-6) / (2 * R))
    for a in range(g.n):
        ids, cnt = o.topk(a, g.n - 1)
        got = {int(i): int(c) for i, c in zip(ids, cnt) if i >= 0}
        for b in range(g.n):
            if b == a:
                continue
            s = float(S.get((min(a, b), max(a, b)), 0))
            assert abs(got.get(b, 0) / R - s) <= tol


def test_isolated_vertex_stays_put():
    g = synth.graph_from_edges(4, [(0, 1), (1, 2)], [1, 1])     # vertex 3 isolated
    P = oracle.sample_paths(g, 5, 4000, 4, oracle.PREFIX)
    rows = P[P[:, 0] == 3]
    assert rows.shape[0] > 0 and (rows == 3).all()
    assert not (P[P[:, 0] != 3] == 3).any()


def test_modes_use_distinct_selection_but_same_start():
    g = synth.workload_graph("small")
    a = oracle.sample_paths(g, 1, 1000, 5, oracle.PREFIX)
    b = oracle.sample_paths(g, 1, 1000, 5, oracle.ALIAS)
    assert (a[:, 0] == b[:, 0]).all()
    assert (a[:, 1:] != b[:, 1:]).any()


def test_paths_are_counter_based():
    # Path r depends only on (seed, r): any sub-range reproduces the same rows.
    g = synth.workload_graph("small")
    full = oracle.sample_paths(g, 3, 500, 5, oracle.ALIAS)
    part = oracle.sample_paths(g, 3, 100, 5, oracle.ALIAS, r0=250)
    assert (full[250:350] == part).all()


# ------------------------------------------- inverted index (Sec. 3.1) ---

def test_index_is_the_set_of_paths_per_vertex(small_graph):
    g = small_graph
    P = oracle.sample_paths(g, 1, 20_000, 5, oracle.PREFIX)
    off, pid = oracle.build_index(g.n, P)
    brute = [[] for _ in range(g.n)]
    for r, row in enumerate(P.tolist()):
        for v in sorted(set(row)):
            brute[v].append(r)
    assert off[-1] == sum(len(set(row)) for row in P.tolist())
    for v in range(g.n):
        assert pid[off[v]:off[v + 1]].tolist() == brute[v]


# ---------------------------------------------- Algorithm 1 + Eq. (4) ---

def _brute_counts(n, P):
    """Full n x n co-occurrence matrix: each unordered pair of distinct vertices
    of each path counted once."""
    M = np.zeros((n, n), dtype=np.int64)
    for row in P.tolist():
        u = sorted(set(row))
        for a, b in itertools.combinations(u, 2):
            M[a, b] += 1
            M[b, a] += 1
    return M


@pytest.fixture(scope="module")
def small_case():
    g = synth.workload_graph("small")
    P = oracle.sample_paths(g, 1, 200_000, 5, oracle.ALIAS)
    return g, P, oracle.Oracle(g.n, P), _brute_counts(g.n, P)


def test_topk_equals_brute_force_for_every_vertex(small_case):
    g, P, o, M = small_case
    k = 10
    for v in range(g.n):
        row = M[v].copy()
        order = np.lexsort((np.arange(g.n), -row))
        order = [u for u in order if u != v and row[u] > 0][:k]
        ids, cnt = o.topk(v, k)
        want_ids = order + [-1] * (k - len(order))
        want_cnt = [int(row[u]) for u in order] + [0] * (k - len(order))
        assert ids.tolist() == want_ids
        assert cnt.tolist() == want_cnt


def test_count_invariants(small_case):
    g, P, o, M = small_case
    assert (M == M.T).all()                                   # symmetry
    sizes = np.diff(o.off)
    for v in range(0, g.n, 7):
        # row sum = sum over paths through v of (#distinct - 1)
        want = sum(len(set(P[r].tolist())) - 1 for r in o.pid[o.off[v]:o.off[v + 1]])
        assert M[v].sum() == want
        nz = np.nonzero(M[v])[0]
        assert (M[v, nz] <= np.minimum(sizes[v], sizes[nz])).all()


def test_theta_equals_sorted_brute_force(small_case):
    g, P, o, M = small_case
    D = 50
    for v in range(0, g.n, 3):
        row = np.delete(M[v], v)
        want = np.sort(row[row > 0])[::-1][:D]
        want = np.concatenate([want, np.zeros(D - want.shape[0], dtype=np.int64)])
        assert o.theta(v, D).tolist() == want.tolist()


def test_knn_equals_all_pairs_integer_l2(small_case):
    g, P, o, M = small_case
    D = 50
    theta = o.theta_all(D)
    T64 = theta.astype(np.int64)
    sq = (T64 * T64).sum(1)
    G = sq[:, None] + sq[None, :] - 2 * (T64 @ T64.T)
    k = 10
    for v in range(0, g.n, 5):
        d = G[v].copy()
        order = [u for u in np.lexsort((np.arange(g.n), d)) if u != v][:k]
        ids, d2 = oracle.knn(theta, v, k)
        assert ids.tolist() == order
        assert d2.tolist() == [int(d[u]) for u in order]


def test_padding_when_fewer_candidates_than_k():
    g = synth.graph_from_edges(4, [(0, 1), (1, 2)], [1, 1])
    P = oracle.sample_paths(g, 5, 50, 2, oracle.PREFIX)
    o = oracle.Oracle(g.n, P)
    ids, cnt = o.topk(3, 5)                  # isolated: no co-occurring vertex
    assert ids.tolist() == [-1] * 5 and cnt.tolist() == [0] * 5
    ids, cnt = o.topk(0, 5)                  # at most vertices 1 and 2
    assert ids.tolist()[2:] == [-1] * 3 and cnt.tolist()[2:] == [0] * 3
    assert o.theta(3, 4).tolist() == [0] * 4
    th = np.zeros((3, 2), dtype=np.uint32)
    ids, d2 = oracle.knn(th, 0, 4)
    assert ids.tolist() == [1, 2, -1, -1]
    assert d2.tolist() == [0, 0, 2**64 - 1, 2**64 - 1]


def test_revisited_vertex_counted_once_per_path():
    # a path that revisits both v and u contributes 1 to cnt(v,u)
    g = synth.graph_from_edges(2, [(0, 1)], [1])
    P = oracle.sample_paths(g, 1, 10, 5, oracle.PREFIX)   # 0,1,0,1,... alternates
    o = oracle.Oracle(g.n, P)
    ids, cnt = o.topk(0, 1)
    assert ids.tolist() == [1] and cnt.tolist() == [10]
    assert (np.diff(o.off) == 10).all()


def test_knn_cross_pins():
    # across "two graphs" that are the same one, the cross list is the
    # self-excluded list with the query itself (distance 0) merged in; and a
    # brute-force loop over a tiny pair of networks with ties
    rng = np.random.default_rng(3)
    th = rng.integers(0, 6, size=(40, 5)).astype(np.uint32)
    for v in range(40):
        ids, d2 = oracle.knn_cross(th, th, v, 9)
        sid, sd2 = oracle.knn(th, v, 8)
        keep = ids != v
        assert ids.tolist().count(v) == 1 and d2[ids.tolist().index(v)] == 0
        assert ids[keep].tolist() == sid.tolist() and d2[keep].tolist() == sd2.tolist()
    a = rng.integers(0, 4, size=(7, 3)).astype(np.uint32)
    b = rng.integers(0, 4, size=(5, 3)).astype(np.uint32)
    for v in range(7):
        brute = sorted((sum((int(x) - int(y)) ** 2 for x, y in zip(a[v], b[u])), u) for u in range(5))
        ids, d2 = oracle.knn_cross(a, b, v, 7)
        assert ids[:5].tolist() == [u for _, u in brute] and d2[:5].tolist() == [d for d, _ in brute]
        assert ids[5:].tolist() == [-1, -1] and d2[5:].tolist() == [2**64 - 1] * 2


@pytest.mark.parametrize("mode", ["prefix", "alias"])
def test_perfect_matching_closed_form(mode):
    # every vertex has exactly one neighbour, so a path never leaves the pair
    # {2i, 2i+1} it starts in: P_2i = P_2i+1 = the paths started in the pair,
    # cnt(2i, 2i+1) = |P_2i| and every other count is 0, theta(v) =
    # [|P_v|, 0, ...], and the k-NN distances are (|P_v| - |P_u|)^2
    pairs = 40
    rng = np.random.default_rng(11)
    g = synth.graph_from_edges(2 * pairs, [(2 * i, 2 * i + 1) for i in range(pairs)],
                               rng.integers(1, 1000, size=pairs).tolist())
    m = oracle.PREFIX if mode == "prefix" else oracle.ALIAS
    R, T = 3000, 4
    P = oracle.sample_paths(g, 2, R, T, m)
    assert set(map(frozenset, (set(row) for row in P.tolist()))) <= {frozenset({2 * i, 2 * i + 1})
                                                                     for i in range(pairs)}
    o = oracle.Oracle(g.n, P)
    sizes = np.diff(o.off)
    starts = np.bincount(P[:, 0] // 2, minlength=pairs)
    assert (sizes[0::2] == starts).all() and (sizes[1::2] == starts).all() and sizes.sum() == 2 * R
    q = np.arange(g.n, dtype=np.int32)
    ids, cnt = o.topk_many(q, 3)
    mate = q ^ 1
    assert (ids[:, 0] == np.where(sizes > 0, mate, -1)).all() and (cnt[:, 0] == sizes).all()
    assert (ids[:, 1:] == -1).all() and (cnt[:, 1:] == 0).all()
    th = o.theta_all(4)
    assert (th[:, 0] == sizes).all() and (th[:, 1:] == 0).all()
    for v in (0, 7, 33):
        kid, kd2 = oracle.knn(th, v, 6)
        brute = sorted(((int(sizes[v]) - int(sizes[u])) ** 2, u) for u in range(g.n) if u != v)[:6]
        assert kid.tolist() == [u for _, u in brute] and kd2.tolist() == [d for d, _ in brute]


def test_star_closed_form():
    # every path through a leaf also passes the centre (T >= 1: a walk
    # leaves a leaf for the centre, and one at the centre moves to a leaf),
    # so cnt(centre, leaf) = |P_leaf|, the centre's top-k is the leaves by
    # (|P_leaf| desc, id asc), and each leaf's count with the centre is its
    # own |P_leaf|
    leaves = 25
    rng = np.random.default_rng(5)
    g = synth.graph_from_edges(leaves + 1, [(0, u) for u in range(1, leaves + 1)],
                               rng.integers(1, 50, size=leaves).tolist())
    for T in (1, 2, 5):
        P = oracle.sample_paths(g, 4, 4000, T, oracle.ALIAS)
        o = oracle.Oracle(g.n, P)
        sizes = np.diff(o.off)
        assert sizes[0] == 4000                           # every path touches the centre
        k = 10
        ids, cnt = o.topk(0, k)
        order = sorted(range(1, leaves + 1), key=lambda u: (-int(sizes[u]), u))
        assert ids.tolist() == order[:k] and cnt.tolist() == [int(sizes[u]) for u in order[:k]]
        for leaf in (1, 9, leaves):
            lid, lcnt = o.topk(leaf, leaves)
            pos = lid.tolist().index(0)
            assert lcnt[pos] == sizes[leaf] and lcnt[0] == sizes[leaf]
