"""GPU parity of the top-k tiers that the default inputs do not reach.

Every tier of Algorithm 1's counting (Eq. (4) counts, then the top-k by count
desc, id asc) must give the oracle's rows bit for bit. `panther_topk_stats`
reports how many queries each tier took, so the tests assert that the tier
they target really ran:
  - the bucketed two-pass hub tier (b_scatter / b_count), with and without
    bucket overflow (an overflowing query is counted again in a device table),
    and the device-table hub tier, reached on a small graph through the
    test-only routing knob (a lower hub bound);
  - paths of T = 8..31 steps (rows of 16 and 32 entries), where the lane and
    group tiers are off and the warp, CTA and hub tiers run the 16- and
    32-wide row kernels; theta (Sec. 3.3) and its k-NN too.
"""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def pk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_02577_gb300 as pk
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return pk


@pytest.fixture(scope="module")
def small():
    g = synth.workload_graph("small")
    ref = oracle.sample_paths(g, 1, 200_000, 5, oracle.ALIAS)
    return g, ref, oracle.Oracle(g.n, ref)


def _topk_routed(pk, g, R, T, seed, queries, k, hub_min_cap, route):
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_ALIAS)
        P.sample_paths(seed, R, T, pk.MODE_ALIAS)
        P.build_index()
        pk.panther_debug_topk_route(P.h.ctx, hub_min_cap, route)
        q = torch.as_tensor(queries, dtype=torch.int32, device="cuda:0")
        ids, cnt = P.topk(q, k)
        P.sync()
        st = pk.panther_topk_stats(P.h.ctx)
        return ids.cpu().numpy(), cnt.cpu().numpy().astype(np.uint32), st


@pytest.mark.parametrize("k", [10, 64])
def test_bucketed_hub_tier_with_overflow(pk, small, k):
    # every query with more than 256 candidates is a hub query and every hub
    # query goes through the buckets; queries with several 819-path chunks
    # overflow their single bucket and are counted again in device tables
    g, ref, o = small
    q = np.arange(g.n, dtype=np.int32)
    ids, cnt, st = _topk_routed(pk, g, 200_000, 5, 1, q, k, 256, 1)
    rid, rcnt = o.topk_many(q, k, threads=THREADS)
    assert np.array_equal(ids, rid) and np.array_equal(cnt, rcnt)
    assert st[5] > 1000 and st[6] >= st[5] and st[8] > 0 and st[7] >= st[8]


def test_bucketed_hub_tier_without_overflow(pk, small):
    # queries of one chunk each: their buckets never fill, so the bucketed
    # tier alone answers them
    g, ref, o = small
    sizes = np.diff(o.off)
    q = np.nonzero((sizes > 60) & (sizes < 700))[0].astype(np.int32)
    assert q.size > 200
    ids, cnt, st = _topk_routed(pk, g, 200_000, 5, 1, q, 10, 256, 1)
    rid, rcnt = o.topk_many(q, 10, threads=THREADS)
    assert np.array_equal(ids, rid) and np.array_equal(cnt, rcnt)
    assert st[5] == q.size and st[6] >= q.size and st[8] == 0 and st[7] == 0


@pytest.mark.parametrize("k", [1, 33])
def test_device_table_hub_tier(pk, small, k):
    g, ref, o = small
    q = np.arange(0, g.n, 3, dtype=np.int32)
    ids, cnt, st = _topk_routed(pk, g, 200_000, 5, 1, q, k, 256, 2)
    rid, rcnt = o.topk_many(q, k, threads=THREADS)
    assert np.array_equal(ids, rid) and np.array_equal(cnt, rcnt)
    assert st[5] > 300 and st[7] >= st[5] and st[6] == 0


def test_default_routing_reports_tiers(pk):
    # the 20,000-vertex hub graph: every tier of the default routing is used,
    # and the sizes add up to the batch
    g = synth.chung_lu(20_000, 12, 2.05, ("uniform", 1, 5), seed=2)
    R, T = 300_000, 5
    q = np.arange(g.n, dtype=np.int32)
    ids, cnt, st = _topk_routed(pk, g, R, T, 3, q, 10, 0, 0)
    o = oracle.Oracle(g.n, oracle.sample_paths(g, 3, R, T, oracle.ALIAS, threads=THREADS))
    sizes = np.diff(o.off)
    empty = int(((sizes == 0) | (np.minimum(sizes * T, g.n - 1) == 0)).sum())
    assert st[0] == g.n and sum(st[1:6]) + empty == g.n
    assert st[1] > 0 and st[2] > 0 and st[3] > 0 and st[4] > 0 and st[5] > 0
    pick = np.unique(np.concatenate([np.argsort(-sizes)[:200], np.arange(0, g.n, 13)])).astype(np.int32)
    rid, rcnt = o.topk_many(pick, 10, threads=THREADS)
    assert np.array_equal(ids[pick], rid) and np.array_equal(cnt[pick], rcnt)


@pytest.mark.parametrize("T", [8, 10, 15, 20, 31, 32, 63, 64, 100, 127])
def test_long_paths_topk_theta_knn(pk, small, T):
    # rows of 16, 32, 64 and 128 entries; from T = 32 on the counting kernels
    # walk one path per warp (lanes hold entries l, l+32, ...)
    g = small[0]
    R, D = (40_000 if T <= 31 else 12_000), 50
    ref = oracle.sample_paths(g, 2, R, T, oracle.ALIAS, threads=THREADS)
    o = oracle.Oracle(g.n, ref)
    q = np.arange(g.n, dtype=np.int32)
    kq = np.arange(0, g.n, 7, dtype=np.int32)
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_ALIAS)
        P.sample_paths(2, R, T, pk.MODE_ALIAS)
        assert np.array_equal(P.paths_tensor().cpu().numpy(), ref)
        P.build_index()
        off_t, pid_t = (t.cpu().numpy() for t in P.index_tensors())
        qt = torch.as_tensor(q, device="cuda:0")
        got = {}
        for k in (10, 64):
            ids, cnt = P.topk(qt, k)
            P.sync()
            got[k] = (ids.cpu().numpy(), cnt.cpu().numpy().astype(np.uint32), pk.panther_topk_stats(P.h.ctx))
        P.vectors(D)
        theta = P.theta_tensor().cpu().numpy().view(np.uint32)
        nids, nd2 = P.knn(torch.as_tensor(kq, device="cuda:0"), 10)
        P.sync()
        nids, nd2 = nids.cpu().numpy(), nd2.cpu().numpy().view(np.uint64)
    assert np.array_equal(off_t, o.off) and np.array_equal(pid_t, o.pid[: pid_t.size])
    for k, (ids, cnt, st) in got.items():
        rid, rcnt = o.topk_many(q, k, threads=THREADS)
        assert np.array_equal(ids, rid), (T, k)
        assert np.array_equal(cnt, rcnt), (T, k)
        assert st[1] == 0 and st[2] == 0            # rows wider than 8: no lane or group tier
        assert st[3] + st[4] + st[5] > 0
    rth = o.theta_all(D, threads=THREADS)
    assert np.array_equal(theta, rth)
    for i, v in enumerate(kq):
        a, b = oracle.knn(rth, int(v), 10)
        assert np.array_equal(nids[i], a) and np.array_equal(nd2[i], b), (T, v)


@pytest.mark.parametrize("T,route", [(64, 1), (100, 2), (127, 1), (40, 0)])
def test_long_paths_hub_tiers_and_plain(pk, T, route):
    # the 20,000-vertex hub graph with long paths: every query whose bound
    # exceeds 256 candidates is a hub query, counted through the buckets
    # (route 1) or device tables (route 2) with the one-path-per-warp
    # insertion; route 0 keeps the default tiers. The plain form (one launch
    # per query, device table above the CTA bound) answers the same rows.
    g = synth.chung_lu(20_000, 12, 2.05, ("uniform", 1, 5), seed=2)
    R = 6_000
    ref = oracle.sample_paths(g, 5, R, T, oracle.ALIAS, threads=THREADS)
    o = oracle.Oracle(g.n, ref)
    sizes = np.diff(o.off)
    q = np.unique(np.concatenate([np.argsort(-sizes)[:40], np.arange(0, g.n, 157)])).astype(np.int32)
    for k in (10, 40):
        ids, cnt, st = _topk_routed(pk, g, R, T, 5, q, k, 256 if route else 0, route)
        rid, rcnt = o.topk_many(q, k, threads=THREADS)
        assert np.array_equal(ids, rid) and np.array_equal(cnt, rcnt), (T, route, k)
        if route:
            assert st[5] > 0 and (st[6] if route == 1 else st[7]) > 0
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_ALIAS)
        P.sample_paths(5, R, T, pk.MODE_ALIAS)
        P.build_index()
        ids, cnt = P.topk(torch.as_tensor(q[:60], device="cuda:0"), 10, plain=True)
        P.sync()
    rid, rcnt = o.topk_many(q[:60], 10, threads=THREADS)
    assert np.array_equal(ids.cpu().numpy(), rid) and np.array_equal(cnt.cpu().numpy().astype(np.uint32), rcnt)


def test_long_path_revisits_and_limits(pk):
    # a 6-vertex graph walked for 127 steps: every row repeats its vertices
    # many times (each must count once); T = 128 is refused
    g = synth.graph_from_edges(6, [(0, 1), (1, 2), (2, 0), (3, 4)], [1, 2, 3, 4])
    R, T = 3_000, 127
    ref = oracle.sample_paths(g, 8, R, T, oracle.ALIAS)
    o = oracle.Oracle(g.n, ref)
    q = np.arange(6, dtype=np.int32)
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_ALIAS)
        P.sample_paths(8, R, T, pk.MODE_ALIAS)
        assert np.array_equal(P.paths_tensor().cpu().numpy(), ref)
        P.build_index()
        off_t, pid_t = (t.cpu().numpy() for t in P.index_tensors())
        ids, cnt = P.topk(torch.as_tensor(q, device="cuda:0"), 5)
        P.sync()
        with pytest.raises(pk.PantherError):
            P.sample_paths(8, 10, 128, pk.MODE_ALIAS)
    assert np.array_equal(off_t, o.off) and np.array_equal(pid_t, o.pid[: pid_t.size])
    rid, rcnt = o.topk_many(q, 5)
    assert np.array_equal(ids.cpu().numpy(), rid) and np.array_equal(cnt.cpu().numpy().astype(np.uint32), rcnt)


@pytest.mark.parametrize("k", [65, 100, 128])
def test_topk_k_above_64(pk, small, k):
    # 64 < k <= 128: queries of up to 32 paths stay in the group tiers, every
    # other query is counted in a device table with 128-entry lists; all
    # 2,000 vertices (many with fewer than k candidates: padding), a batch of
    # short path lists that the group tiers take, the plain form on a subset,
    # and a long-path case
    g, ref, o = small
    q = np.arange(g.n, dtype=np.int32)
    ids, cnt, st = _topk_routed(pk, g, 200_000, 5, 1, q, k, 0, 0)
    rid, rcnt = o.topk_many(q, k, threads=THREADS)
    assert np.array_equal(ids, rid) and np.array_equal(cnt, rcnt)
    assert st[7] > 1000 and st[1] == st[3] == st[4] == 0 and st[7] >= st[5]
    R3 = 5_000                                        # about 15 paths per vertex
    ref3 = oracle.sample_paths(g, 4, R3, 5, oracle.ALIAS, threads=THREADS)
    o3 = oracle.Oracle(g.n, ref3)
    ids3, cnt3, st3 = _topk_routed(pk, g, R3, 5, 4, q, k, 0, 0)
    rid3, rcnt3 = o3.topk_many(q, k, threads=THREADS)
    assert np.array_equal(ids3, rid3) and np.array_equal(cnt3, rcnt3)
    assert st3[2] > 1000 and st3[1] == st3[3] == st3[4] == 0
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_ALIAS)
        P.sample_paths(1, 200_000, 5, pk.MODE_ALIAS)
        P.build_index()
        sub = torch.as_tensor(q[::97], device="cuda:0")
        pids, pcnt = P.topk(sub, k, plain=True)
        P.sync()
    assert np.array_equal(pids.cpu().numpy(), rid[::97])
    assert np.array_equal(pcnt.cpu().numpy().astype(np.uint32), rcnt[::97])
    T, R = 100, 6_000
    ref2 = oracle.sample_paths(g, 3, R, T, oracle.ALIAS, threads=THREADS)
    o2 = oracle.Oracle(g.n, ref2)
    q2 = np.arange(0, g.n, 5, dtype=np.int32)
    ids2, cnt2, _ = _topk_routed(pk, g, R, T, 3, q2, k, 0, 0)
    rid2, rcnt2 = o2.topk_many(q2, k, threads=THREADS)
    assert np.array_equal(ids2, rid2) and np.array_equal(cnt2, rcnt2)
