"""GPU parity of Panther++ (theta vectors and exact k-NN) against the CPU oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_02577_gb300 as pk
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return pk


def _vectors(pk, g, seed, R, T, D, queries=None, k=None, fp32=False, both=False):
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_ALIAS)
        P.sample_paths(seed, R, T, pk.MODE_ALIAS)
        P.build_index()
        P.vectors(D)
        out = {"theta": P.theta_tensor().cpu().numpy().view(np.uint32)}
        if k:
            q = torch.as_tensor(queries, dtype=torch.int32, device="cuda:0")
            forms = [False, True] if both else [fp32]
            for kk in (k if isinstance(k, (list, tuple)) else [k]):
                for f in forms:
                    ids, d2 = P.knn(q, kk, fp32=f)
                    P.sync()
                    key = ("fp32" if f else "bf16") + ("" if kk == k else f"_k{kk}")
                    out[key] = (ids.cpu().numpy(), d2.cpu().numpy().view(np.uint64))
            out["stats"] = pk.pantherpp_knn_stats(P.h.ctx)
        P.sync()
    return out


def _oracle_theta(g, seed, R, T, D):
    P = oracle.sample_paths(g, seed, R, T, oracle.ALIAS)
    return oracle.Oracle(g.n, P).theta_all(D)


@pytest.fixture(scope="module")
def small_case():
    g = synth.workload_graph("small")
    th = _oracle_theta(g, 1, 200_000, 5, 50)
    return g, th


def test_theta_bit_exact_small_workload(pk, small_case):
    g, th = small_case
    out = _vectors(pk, g, 1, 200_000, 5, 50)
    assert np.array_equal(out["theta"], th)
    assert th.max() > 256          # some rows are not BF16-exact: the bounded path runs


@pytest.mark.parametrize("k", [1, 10, 32])
def test_knn_exact_all_vertices_small_workload(pk, small_case, k):
    g, th = small_case
    q = np.arange(g.n, dtype=np.int32)
    out = _vectors(pk, g, 1, 200_000, 5, 50, queries=q, k=k, both=True)
    for form in ("bf16", "fp32"):
        ids, d2 = out[form]
        for v in range(g.n):
            rid, rd = oracle.knn(th, v, k)
            assert ids[v].tolist() == rid.tolist(), (form, v)
            assert d2[v].tolist() == rd.tolist(), (form, v)


def test_knn_large_counts_and_ragged_queries(pk):
    # a small dense graph with many paths: counts in the thousands, so most
    # rows are inexact in BF16 and the error bound decides the shortlist
    g = synth.chung_lu(700, 12, 2.4, ("uniform", 1, 20), seed=6)
    R, T, D, k = 600_000, 5, 50, 7
    th = _oracle_theta(g, 4, R, T, D)
    assert th.max() > 2000
    rng = np.random.default_rng(1)
    q = rng.integers(0, g.n, size=333).astype(np.int32)          # ragged, with repeats
    out = _vectors(pk, g, 4, R, T, D, queries=q, k=k, both=True)
    assert np.array_equal(out["theta"], th)
    for form in ("bf16", "fp32"):
        ids, d2 = out[form]
        for i, v in enumerate(q):
            rid, rd = oracle.knn(th, int(v), k)
            assert ids[i].tolist() == rid.tolist(), (form, i)
            assert d2[i].tolist() == rd.tolist(), (form, i)


def test_knn_shortlist_overflow_falls_back_exactly(pk):
    # counts in the tens of thousands on a dense graph: the BF16 error bound
    # covers hundreds of candidates per query, shortlists overflow and those
    # queries are answered by the exact brute-force pass
    g = synth.chung_lu(1500, 60, 2.2, ("uniform", 1, 4), seed=8)
    R, T, D, k = 4_000_000, 5, 50, 10
    th = _oracle_theta(g, 6, R, T, D)
    rng = np.random.default_rng(2)
    q = rng.integers(0, g.n, size=200).astype(np.int32)
    out = _vectors(pk, g, 6, R, T, D, queries=q, k=k, both=False)
    assert np.array_equal(out["theta"], th)
    assert out["stats"][2] > 0                          # some queries overflowed
    ids, d2 = out["bf16"]
    for i, v in enumerate(q):
        rid, rd = oracle.knn(th, int(v), k)
        assert ids[i].tolist() == rid.tolist() and d2[i].tolist() == rd.tolist(), i


def test_knn_mass_ties_and_padding(pk):
    # many identical vectors (distance-0 ties broken by id) and k larger than
    # the number of other vertices
    g = synth.graph_from_edges(9, [(0, 1), (2, 3), (4, 5), (6, 7)], [1, 1, 1, 1])   # 8 isolated
    R, T, D = 2000, 3, 4
    th = _oracle_theta(g, 2, R, T, D)
    q = np.arange(g.n, dtype=np.int32)
    out = _vectors(pk, g, 2, R, T, D, queries=q, k=12, both=True)
    assert np.array_equal(out["theta"], th)
    for form in ("bf16", "fp32"):
        ids, d2 = out[form]
        for v in range(g.n):
            rid, rd = oracle.knn(th, v, 12)
            assert ids[v].tolist() == rid.tolist()
            assert d2[v].tolist() == rd.tolist()


def test_knn_host_io_and_errors(pk, small_case):
    g, th = small_case
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_ALIAS)
        P.sample_paths(1, 200_000, 5, pk.MODE_ALIAS)
        P.build_index()
        P.vectors(50)
        q = np.array([3, 1999, 0, 77], dtype=np.int32)
        ids = np.empty((4, 5), np.int32)
        d2 = np.empty((4, 5), np.uint64)
        pk.pantherpp_knn(P.h.ctx, P.h.vecs, q, 4, 5, ids, d2, pk.KNN_BF16_SCREEN | pk.IO_HOST)
        for i, v in enumerate(q):
            rid, rd = oracle.knn(th, int(v), 5)
            assert ids[i].tolist() == rid.tolist() and d2[i].tolist() == rd.tolist()
        with pytest.raises(pk.PantherError):
            P.knn(torch.zeros(1, dtype=torch.int32, device="cuda:0"), 33)
        with pytest.raises(pk.PantherError):
            P.vectors(129)                              # wider than the counting path
        P.sync()


@pytest.mark.parametrize("D", [57, 64, 100, 128])
def test_wide_vectors_theta_and_knn(pk, small_case, D):
    # D > 56: no room for the exact squared norm in the 64 BF16 columns, so
    # either flag takes the FP32 screen (64 columns up to D = 64, 128 beyond)
    # with the exact rerank. theta of D > 64 counts through the top-k path
    # for k > 64. All must equal the oracle.
    g, _ = small_case
    R, T = 200_000, 5
    th = _oracle_theta(g, 1, R, T, D)
    q = np.concatenate([np.arange(0, g.n, 17), [5, 5]]).astype(np.int32)
    out = _vectors(pk, g, 1, R, T, D, queries=q, k=[10, 32], both=True)
    assert np.array_equal(out["theta"], th)
    for key, kk in (("bf16_k10", 10), ("fp32_k10", 10), ("bf16_k32", 32), ("fp32_k32", 32)):
        ids, d2 = out[key]
        for i, v in enumerate(q):
            rid, rd = oracle.knn(th, int(v), kk)
            assert ids[i].tolist() == rid.tolist() and d2[i].tolist() == rd.tolist(), (D, key, i)


def test_knn_workload_shape_sampled(pk):
    """A 200K-vertex graph shaped like the k-NN workload (mean degree 20, gamma 2.3,
    log-uniform weights), R = 5 paths per vertex, D = 50: all-vertex theta checked on
    a sample of rows, and the exact top-10 and top-32 of sampled queries (incl. the
    heaviest). One query tile against 782 candidate tiles: the candidate range is cut
    into pieces screened by different CTAs and merged."""
    g = synth.chung_lu(200_000, 20, 2.3, ("loguniform", 1, 1024), seed=1)
    R, T, D, k = 1_000_000, 5, 50, 10
    P = oracle.sample_paths(g, 1, R, T, oracle.ALIAS)
    o = oracle.Oracle(g.n, P)
    th = o.theta_all(D)
    sizes = np.diff(o.off)
    q = np.unique(np.concatenate([np.argsort(-sizes)[:40], np.arange(0, g.n, 4001)])).astype(np.int32)
    out = _vectors(pk, g, 1, R, T, D, queries=q, k=[k, 32], both=False)
    assert np.array_equal(out["theta"], th)
    for key, kk in (("bf16_k10", k), ("bf16_k32", 32)):
        ids, d2 = out[key]
        for i, v in enumerate(q):
            rid, rd = oracle.knn(th, int(v), kk)
            assert ids[i].tolist() == rid.tolist() and d2[i].tolist() == rd.tolist(), (key, i)


@pytest.mark.parametrize("fp32", [False, True])
def test_knn_cross_graph(pk, fp32):
    # two different networks (a dense one with inexact rows, a sparser one),
    # queries from the first, answers from the second, both forms exact; and
    # the same vector set on both sides keeps the query itself at distance 0
    ga = synth.chung_lu(900, 10, 2.4, ("uniform", 1, 20), seed=31)
    gb = synth.chung_lu(1300, 8, 2.2, ("loguniform", 1, 64), seed=32)
    R, T, D, k = 120_000, 5, 24, 12
    tha = _oracle_theta(ga, 7, R, T, D)
    thb = _oracle_theta(gb, 8, R, T, D)
    assert tha.max() > 256                       # some rows of the first graph are inexact in BF16
    rng = np.random.default_rng(4)
    q = rng.integers(0, ga.n, size=333).astype(np.int32)
    flag = pk.KNN_FP32 if fp32 else pk.KNN_BF16_SCREEN
    handles = []
    ctx = pk.panther_create(0)
    try:
        vh = []
        for g, seed in ((ga, 7), (gb, 8)):
            gh = pk.panther_build_graph(ctx, g.n, g.m, g.row_ptr, g.col, g.w, pk.MEM_HOST, pk.MODE_ALIAS)
            ph = pk.panther_sample_paths(ctx, gh, seed, R, T, pk.MODE_ALIAS)
            ih = pk.panther_build_index(ctx, ph)
            vh.append(pk.pantherpp_vectors(ctx, ih, ph, D))
            handles += [(pk.panther_free_index, ih), (pk.panther_free_paths, ph), (pk.panther_free_graph, gh)]
        ids = np.empty((q.size, k), np.int32)
        d2 = np.empty((q.size, k), np.uint64)
        pk.pantherpp_knn_cross(ctx, vh[0], vh[1], q, q.size, k, ids, d2, flag | pk.IO_HOST)
        for i, v in enumerate(q):
            rid, rd = oracle.knn_cross(tha, thb, int(v), k)
            assert ids[i].tolist() == rid.tolist() and d2[i].tolist() == rd.tolist(), i
        pk.pantherpp_knn_cross(ctx, vh[0], vh[0], q, q.size, k, ids, d2, flag | pk.IO_HOST)
        for i, v in enumerate(q):
            rid, rd = oracle.knn_cross(tha, tha, int(v), k)
            assert ids[i].tolist() == rid.tolist() and d2[i].tolist() == rd.tolist(), i
        bad = pk.pantherpp_vectors(ctx, handles[0][1], handles[1][1], D - 1)
        with pytest.raises(pk.PantherError):
            pk.pantherpp_knn_cross(ctx, vh[0], bad, q, q.size, k, ids, d2, flag | pk.IO_HOST)   # D differs
        pk.pantherpp_free_vecs(bad)
        for v_ in vh:
            pk.pantherpp_free_vecs(v_)
        for free, h in handles:
            free(h)
    finally:
        pk.panther_destroy(ctx)


@pytest.mark.parametrize("case", ["small", "large_counts"])
def test_screen_values_within_the_proven_bound(pk, case):
    """Every tensor-core screened value y_hat (BF16 inputs, FP32 accumulation)
    lies within the error bound the rerank relies on,
    |y_hat - y| <= (0.0157 |a||b| + 1.6e-5 |b|^2 + 1) * 1.0001 with
    y = |b|^2 - 2 a.b exact, and equals y exactly when both rows hold only
    entries <= 256 (BF16-exact rows)."""
    if case == "small":
        g, seed, R = synth.workload_graph("small"), 1, 200_000
    else:
        g, seed, R = synth.chung_lu(700, 12, 2.4, ("uniform", 1, 20), seed=6), 4, 600_000
    T, D = 5, 50
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_ALIAS)
        P.sample_paths(seed, R, T, pk.MODE_ALIAS)
        P.build_index()
        P.vectors(D)
        theta = P.theta_tensor().cpu().numpy().view(np.uint32).astype(np.int64)
        npad = pk.pantherpp_debug_screen(P.h.ctx, P.h.vecs)
        norm2 = (theta ** 2).sum(axis=1)
        q = np.unique(np.concatenate([np.argsort(-norm2)[:64], np.arange(0, g.n, max(1, g.n // 64))]))[:128]
        q = q.astype(np.int32)
        y = torch.empty((q.size, npad), dtype=torch.float32, device="cuda:0")
        cid = torch.empty(npad, dtype=torch.int32, device="cuda:0")
        pk.pantherpp_debug_screen(P.h.ctx, P.h.vecs, torch.as_tensor(q, device="cuda:0"), q.size, y, cid)
        y, cid = y.cpu().numpy().astype(np.float64), cid.cpu().numpy()
    assert npad % 256 == 0 and sorted(cid[cid >= 0].tolist()) == list(range(g.n))
    ok = cid >= 0
    c = cid[ok]
    exact_row = theta.max(axis=1) <= 256
    if case == "large_counts":
        assert (~exact_row).sum() > 100
    for i, v in enumerate(q):
        y_exact = norm2[c] - 2 * (theta[c] @ theta[v])           # int64, exact here
        err = np.abs(y[i][ok] - y_exact.astype(np.float64))
        bound = (0.0157 * np.sqrt(float(norm2[v])) * np.sqrt(norm2[c].astype(np.float64))
                 + 1.6e-5 * norm2[c] + 1.0) * 1.0001
        assert (err <= bound).all(), (v, float((err / bound).max()))
        if exact_row[v]:
            assert (err[exact_row[c]] == 0).all(), v
