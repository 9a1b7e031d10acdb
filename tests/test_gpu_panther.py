"""GPU parity of the Panther path against the CPU oracle (bit-exact, integer outputs).

Everything goes through the C ABI (libpanther.so) via the ctypes binding.
Inputs are seeded synthetic Chung-Lu graphs; expected values come only from
oracle/.
"""
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


@pytest.fixture(scope="module")
def small():
    return synth.workload_graph("small")


def _run(pk, g, seed, R, T, mode, k=None, queries=None, plain=False, budget=None):
    with pk.Panther(0) as P:
        if budget:
            pk.panther_set_scratch_budget(P.h.ctx, budget)
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_BOTH)
        P.sample_paths(seed, R, T, mode)
        out = {"paths": P.paths_tensor().cpu().numpy()}
        P.build_index()
        off, pid = P.index_tensors()
        out["off"], out["pid"] = off.cpu().numpy(), pid.cpu().numpy()
        if k:
            q = torch.as_tensor(queries if queries is not None else np.arange(g.n, dtype=np.int32),
                                dtype=torch.int32, device="cuda:0")
            ids, cnt = P.topk(q, k, plain=plain)
            P.sync()
            out["ids"], out["cnt"] = ids.cpu().numpy(), cnt.cpu().numpy().astype(np.uint32)
        P.sync()
        out["launches"] = P.launches()
    return out


# ------------------------------------------------------------ Philox ---

def test_philox_matches_curand_and_oracle(pk):
    ctx = pk.panther_create(0)
    try:
        for (k0, k1, r0, c2, c3) in [(1, 0, 0, 0, 0), (0xDEADBEEF, 0x12345678, 2**32 - 5, 7, 3),
                                     (0xFFFFFFFF, 0xFFFFFFFF, 2**40, 0xFFFF, 0x10)]:
            n = 4096
            out = torch.empty((n, 4), dtype=torch.int32, device="cuda:0")
            ref = torch.empty((n, 4), dtype=torch.int32, device="cuda:0")
            pk.panther_debug_philox(ctx, k0, k1, r0, c2, c3, n, out, ref)
            a = out.cpu().numpy().view(np.uint32)
            b = ref.cpu().numpy().view(np.uint32)
            assert np.array_equal(a, b), "device Philox differs from curand"
            for i in (0, 1, 17, n - 1):
                r = r0 + i
                o = oracle.philox4x32_10((r & 0xFFFFFFFF, r >> 32, c2, c3), (k0, k1))
                assert np.array_equal(o, b[i]), "oracle Philox differs from curand"
    finally:
        pk.panther_destroy(ctx)


# ------------------------------------------------------------ tables ---

def _tables(pk, g):
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_BOTH)
        al = torch.empty((max(g.m, 1), 4), dtype=torch.int32, device="cuda:0")
        wide = pk.panther_debug_graph_tables(P.h.graph, al, None)
        pre = torch.empty((max(g.m, 1), 4 if wide else 2), dtype=torch.int32, device="cuda:0")
        pk.panther_debug_graph_tables(P.h.graph, None, pre)
        return al.cpu().numpy().view(np.uint32), pre.cpu().numpy().view(np.uint32), wide


def _big_row_graph():
    # a hub of degree 5000 (CTA-per-row path) with skewed weights, plus a ring
    n = 6000
    rng = np.random.default_rng(4)
    edges, ws = [], []
    for u in range(1, 5001):
        edges.append((0, u))
        ws.append(int(rng.integers(1, 2**20)) if u % 7 else 1)
    for u in range(1, n - 1):
        edges.append((u, u + 1))
        ws.append(int(rng.integers(1, 50)))
    return synth.graph_from_edges(n, edges, ws)


def _hub_rows_graph():
    # rows split into 1, 1, 2 and 5 segments of 4096 entries: equal weights
    # (every entry exactly at capacity), random, one dominant weight, and
    # log-uniform weights; plus a path through the other vertices
    n = 30_000
    rng = np.random.default_rng(9)
    edges, ws = [], []
    for hub, deg in enumerate([2049, 4096, 4097, 20_000]):
        for j, u in enumerate(range(4, 4 + deg)):
            edges.append((hub, u))
            if hub == 0:
                ws.append(7)
            elif hub == 1:
                ws.append(int(rng.integers(1, 2**20)))
            elif hub == 2:
                ws.append(2**24 if j == 1234 else 1)
            else:
                ws.append(int(np.exp(rng.uniform(0, np.log(2**16)))))
    for u in range(4, n - 1):
        edges.append((u, u + 1))
        ws.append(int(rng.integers(1, 50)))
    return synth.graph_from_edges(n, edges, ws)


_SHORT_DEGS = [17, 24, 32, 33, 50, 64, 65, 100, 128, 129, 511, 512, 513, 1000, 2048]


def _short_rows_graph():
    # rows on both sides of the 8/16/32-lane and warp boundaries (32, 64, 128)
    # and across the warp rows up to the longest (2048), with equal, random,
    # one dominant, and log-uniform weights
    n = 3000
    rng = np.random.default_rng(13)
    edges, ws = [], []
    for r in range(4 * len(_SHORT_DEGS)):
        deg = _SHORT_DEGS[r % len(_SHORT_DEGS)]
        nb = rng.choice(np.arange(100, n), size=deg, replace=False)
        for j, u in enumerate(nb):
            edges.append((r, int(u)))
            kind = r // len(_SHORT_DEGS)
            if kind == 0:
                ws.append(5)
            elif kind == 1:
                ws.append(int(rng.integers(1, 2**16)))
            elif kind == 2:
                ws.append(2**20 if j == 3 else 1)
            else:
                ws.append(int(np.exp(rng.uniform(0, np.log(2**12)))))
    return synth.graph_from_edges(n, edges, ws)


@pytest.mark.parametrize("which", ["small", "bigrow", "hubrows", "shortrows", "wide"])
def test_transition_tables_match_oracle(pk, small, which):
    if which == "small":
        g = small
    elif which == "bigrow":
        g = _big_row_graph()
    elif which == "hubrows":
        g = _hub_rows_graph()
    elif which == "shortrows":
        g = _short_rows_graph()
        deg = np.diff(g.row_ptr)
        assert all((deg == d).sum() >= 4 for d in _SHORT_DEGS)
    else:
        # row sums beyond 2^32 switch the prefix table to 64-bit entries
        g = synth.graph_from_edges(40, [(0, i) for i in range(1, 40)] + [(1, 2)],
                                   [2**31 + i for i in range(1, 40)] + [5])
    al, pre, wide = _tables(pk, g)
    thr, ali = oracle.alias_tables(g)
    gthr = al[:, 0].astype(np.uint64) | (al[:, 1].astype(np.uint64) << np.uint64(32))
    assert np.array_equal(gthr[:g.m], thr[:g.m])
    assert np.array_equal(al[:g.m, 2], g.col.view(np.uint32))
    # alias column stored as the neighbour id
    row_of = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    want_alias = g.col[g.row_ptr[row_of] + ali[:g.m]]
    assert np.array_equal(al[:g.m, 3].view(np.int32), want_alias)
    # prefix: inclusive cumulative weight per row
    cum = np.zeros(g.m, dtype=np.uint64)
    for v in range(g.n):
        a, b = g.row_ptr[v], g.row_ptr[v + 1]
        cum[a:b] = np.cumsum(g.w[a:b].astype(np.uint64))
    if wide:
        gcum = pre[:, 0].astype(np.uint64) | (pre[:, 1].astype(np.uint64) << np.uint64(32))
        assert np.array_equal(gcum[:g.m], cum) and np.array_equal(pre[:g.m, 2].view(np.int32), g.col)
    else:
        assert np.array_equal(pre[:g.m, 0].astype(np.uint64), cum)
        assert np.array_equal(pre[:g.m, 1].view(np.int32), g.col)
    assert wide == (which == "wide")


def test_invalid_graph_is_rejected(pk):
    g = synth.graph_from_edges(5, [(0, 1), (1, 2), (3, 4)], [1, 2, 3])
    with pk.Panther(0) as P:
        w = g.w.copy()
        w[0] = 7           # asymmetric weight
        with pytest.raises(pk.PantherError):
            P.build_graph(g.row_ptr, g.col, w)
        col = g.col.copy()
        col[0] = 0         # self-loop
        with pytest.raises(pk.PantherError):
            P.build_graph(g.row_ptr, col, g.w)
        rp = g.row_ptr.copy()
        rp[2] = rp[3] + 1  # offsets not monotone
        with pytest.raises(pk.PantherError):
            P.build_graph(rp, g.col, g.w)
        P.build_graph(g.row_ptr, g.col, g.w)   # the valid graph still builds


# ------------------------------------------------------------- paths ---

@pytest.mark.parametrize("mode", ["prefix", "alias"])
def test_paths_and_index_bit_exact_small_workload(pk, small, mode):
    m = pk.MODE_PREFIX if mode == "prefix" else pk.MODE_ALIAS
    om = oracle.PREFIX if mode == "prefix" else oracle.ALIAS
    R, T = 200_000, 5
    out = _run(pk, small, 1, R, T, m)
    ref = oracle.sample_paths(small, 1, R, T, om)
    assert np.array_equal(out["paths"], ref)
    off, pid = oracle.build_index(small.n, ref)
    assert np.array_equal(out["off"], off)
    assert np.array_equal(out["pid"], pid)


@pytest.mark.parametrize("T", [1, 2, 7, 9, 15, 20, 31, 32, 47, 63, 64, 99, 127])
@pytest.mark.parametrize("mode", ["alias", "prefix"])
def test_paths_other_lengths(pk, T, mode):
    g = synth.chung_lu(3000, 6, 2.2, ("uniform", 1, 1000), seed=9)
    R = 3001     # ragged: not a multiple of any tile
    out = _run(pk, g, 12345, R, T, pk.MODE_ALIAS if mode == "alias" else pk.MODE_PREFIX)
    ref = oracle.sample_paths(g, 12345, R, T, oracle.ALIAS if mode == "alias" else oracle.PREFIX)
    assert np.array_equal(out["paths"], ref)
    off, pid = oracle.build_index(g.n, ref)
    assert np.array_equal(out["off"], off) and np.array_equal(out["pid"], pid)


@pytest.mark.parametrize("T,budget", [(5, 1 << 20), (5, 3 << 20), (64, 2 << 20), (3, 10 << 20)])
def test_index_in_chunks_equals_one_pass(pk, small, T, budget):
    # an index budget too small for one radix sort over all pairs: the rows
    # are sorted in chunks of consecutive paths and appended per vertex; the
    # index must equal the one-pass index and the oracle's (ragged R, long
    # rows, a budget that leaves two chunks)
    R = 200_001 if T < 64 else 20_001
    with pk.Panther(0) as P:
        P.build_graph(small.row_ptr, small.col, small.w, pk.MODE_ALIAS)
        P.sample_paths(4, R, T, pk.MODE_ALIAS)
        P.build_index()
        off1, pid1 = (t.cpu().numpy() for t in P.index_tensors())
        launches1 = P.launches()
        pk.panther_set_index_budget(P.h.ctx, budget)
        P.build_index()
        chunk_launches = P.launches() - launches1
        off2, pid2 = (t.cpu().numpy() for t in P.index_tensors())
        ids, cnt = P.topk(torch.arange(small.n, dtype=torch.int32, device="cuda:0"), 10)
        P.sync()
        paths = P.paths_tensor().cpu().numpy()
        with pytest.raises(pk.PantherError):
            pk.panther_set_index_budget(P.h.ctx, 1000)          # below 1 MiB
    assert chunk_launches > 12                                   # several chunks ran
    assert np.array_equal(off1, off2) and np.array_equal(pid1, pid2)
    off, pid = oracle.build_index(small.n, paths)
    assert np.array_equal(off2, off) and np.array_equal(pid2, pid)
    o = oracle.Oracle(small.n, paths, off, pid)
    rid, rcnt = o.topk_many(np.arange(small.n, dtype=np.int32), 10)
    assert np.array_equal(ids.cpu().numpy(), rid) and np.array_equal(cnt.cpu().numpy().astype(np.uint32), rcnt)


def test_paths_wide_prefix_and_isolated(pk):
    # 64-bit cumulative weights and isolated vertices (the walk stays put)
    edges = [(0, i) for i in range(1, 30)] + [(1, 2), (2, 3)]
    ws = [2**31 + 17 * i for i in range(1, 30)] + [3, 4]
    g = synth.graph_from_edges(40, edges, ws)
    for m, om in ((pk.MODE_PREFIX, oracle.PREFIX), (pk.MODE_ALIAS, oracle.ALIAS)):
        out = _run(pk, g, 99, 5000, 6, m)
        ref = oracle.sample_paths(g, 99, 5000, 6, om)
        assert np.array_equal(out["paths"], ref)


def test_counter_based_seeds_differ(pk, small):
    a = _run(pk, small, 1, 1000, 5, pk.MODE_ALIAS)["paths"]
    b = _run(pk, small, 2, 1000, 5, pk.MODE_ALIAS)["paths"]
    assert not np.array_equal(a, b)
    assert np.array_equal(a, oracle.sample_paths(small, 1, 1000, 5, oracle.ALIAS))


# ------------------------------------------------------------- top-k ---

@pytest.mark.parametrize("k", [1, 10, 33, 64])
def test_topk_all_vertices_small_workload(pk, small, k):
    R, T = 200_000, 5
    out = _run(pk, small, 1, R, T, pk.MODE_ALIAS, k=k)
    ref = oracle.sample_paths(small, 1, R, T, oracle.ALIAS)
    o = oracle.Oracle(small.n, ref)
    rid, rcnt = o.topk_many(np.arange(small.n), k)
    assert np.array_equal(out["ids"], rid)
    assert np.array_equal(out["cnt"], rcnt)


def test_topk_plain_equals_batched_and_oracle(pk, small):
    R, T, k = 50_000, 5, 10
    rng = np.random.default_rng(0)
    q = rng.integers(0, small.n, size=300).astype(np.int32)
    a = _run(pk, small, 5, R, T, pk.MODE_PREFIX, k=k, queries=q, plain=True)
    b = _run(pk, small, 5, R, T, pk.MODE_PREFIX, k=k, queries=q, plain=False)
    assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["cnt"], b["cnt"])
    o = oracle.Oracle(small.n, oracle.sample_paths(small, 5, R, T, oracle.PREFIX))
    rid, rcnt = o.topk_many(q, k)
    assert np.array_equal(a["ids"], rid) and np.array_equal(a["cnt"], rcnt)
    assert a["launches"] > b["launches"] + 250      # one launch per query


def test_topk_global_tier_hubs(pk):
    # hubs whose candidate bound exceeds the shared-memory table; a small
    # scratch budget forces several rounds of global tables
    g = synth.chung_lu(20_000, 12, 2.05, ("uniform", 1, 5), seed=2)
    R, T, k = 300_000, 5, 12
    hubs = synth.hub_set(g, 0.002)
    q = np.concatenate([hubs, np.arange(0, 20_000, 97, dtype=np.int32)]).astype(np.int32)
    out = _run(pk, g, 3, R, T, pk.MODE_ALIAS, k=k, queries=q, budget=64 << 20)
    ref = oracle.sample_paths(g, 3, R, T, oracle.ALIAS)
    o = oracle.Oracle(g.n, ref)
    sizes = np.diff(o.off)
    assert sizes[hubs].max() * 5 > 20_000            # some query is in the global tier
    rid, rcnt = o.topk_many(q, k)
    assert np.array_equal(out["ids"], rid)
    assert np.array_equal(out["cnt"], rcnt)


@pytest.mark.parametrize("k", [1, 10, 40])
def test_topk_group_tiers(pk, k):
    # about 12 paths per vertex: most queries have 7..16 paths (the sort-based
    # tiers of 8 and 16 lanes per query); low-degree cycles make paths revisit
    # vertices, so equal keys inside one path must count once
    g = synth.chung_lu(5000, 6, 2.5, ("uniform", 1, 3), seed=11)
    R, T = 10_000, 5
    out = _run(pk, g, 12, R, T, pk.MODE_ALIAS, k=k)
    o = oracle.Oracle(g.n, oracle.sample_paths(g, 12, R, T, oracle.ALIAS))
    sizes = np.diff(o.off)
    assert ((sizes > 6) & (sizes <= 8)).sum() > 500 and ((sizes > 8) & (sizes <= 16)).sum() > 1000
    rid, rcnt = o.topk_many(np.arange(g.n, dtype=np.int32), k)
    assert np.array_equal(out["ids"], rid)
    assert np.array_equal(out["cnt"], rcnt)


def test_topk_hub_threshold_retry(pk):
    # A 30,000-leaf star whose centre is a hub query: its first-round filter
    # (candidates u with hundreds of paths or more) keeps at most the twelve
    # secondary hubs, whose counts with the centre lie far below that, so the
    # centre is counted again with its k-th count as the threshold, or with no
    # threshold at all when fewer than k candidates survive.
    n = 40_000
    edges = [(0, u) for u in range(1, 30_001)]
    for s_ in range(1, 13):
        edges += [(s_, 30_001 + 300 * (s_ - 1) + j) for j in range(300) if 30_001 + 300 * (s_ - 1) + j < n]
    g = synth.graph_from_edges(n, edges, [1] * len(edges))
    R, T = 200_000, 5
    q = np.array([0, 1, 2, 12, 500, 30_001, 0], dtype=np.int32)
    ref = oracle.sample_paths(g, 5, R, T, oracle.ALIAS)
    o = oracle.Oracle(g.n, ref)
    sizes = np.diff(o.off)
    assert sizes[0] * 5 > 30_000 and sizes[1:13].min() >= 255
    for k in (10, 20, 1):
        out = _run(pk, g, 5, R, T, pk.MODE_ALIAS, k=k, queries=q)
        rid, rcnt = o.topk_many(q, k)
        assert np.array_equal(out["ids"], rid), k
        assert np.array_equal(out["cnt"], rcnt), k
    assert rcnt[0].max() < 255        # so the first round cannot be the answer


def test_topk_large_hub_thresholds(pk):
    # Hubs with 1e5 to 3e5 paths: the first-round filters sit in the hundreds
    # of paths (above the exact range of the one-byte path codes), their k-th
    # counts in the thousands, so the filtered round is the answer; k = 40
    # lowers the filters (k = 1 keeps those of k = 10: the divisor is at least 10)
    g = synth.chung_lu(20_000, 12, 2.05, ("uniform", 1, 5), seed=2)
    R, T = 2_000_000, 5
    ref = oracle.sample_paths(g, 3, R, T, oracle.ALIAS)
    o = oracle.Oracle(g.n, ref)
    sizes = np.diff(o.off)
    hubs = np.argsort(-sizes)[:40].astype(np.int32)
    assert sizes[hubs[0]] > 250_000 and sizes[hubs[5]] > 80_000
    q = np.concatenate([hubs, np.arange(0, g.n, 211, dtype=np.int32)]).astype(np.int32)
    for k in (10, 40, 1):
        out = _run(pk, g, 3, R, T, pk.MODE_ALIAS, k=k, queries=q)
        rid, rcnt = o.topk_many(q, k)
        assert np.array_equal(out["ids"], rid), k
        assert np.array_equal(out["cnt"], rcnt), k
        assert (rcnt[:6, -1] > sizes[hubs[:6]] * 0.003 * 10 / max(k, 10)).all()


def test_topk_edge_cases(pk):
    g = synth.graph_from_edges(6, [(0, 1), (1, 2), (2, 0), (3, 4)], [1, 2, 3, 4])  # 5 isolated
    R, T = 400, 3
    q = np.array([5, 0, 0, 3, 1, 5], dtype=np.int32)          # duplicates, isolated
    out = _run(pk, g, 8, R, T, pk.MODE_ALIAS, k=7, queries=q)
    o = oracle.Oracle(g.n, oracle.sample_paths(g, 8, R, T, oracle.ALIAS))
    rid, rcnt = o.topk_many(q, 7)
    assert np.array_equal(out["ids"], rid) and np.array_equal(out["cnt"], rcnt)
    assert (out["ids"][0] == -1).all() and (out["cnt"][0] == 0).all()
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w)
        P.sample_paths(1, 10, 2)
        P.build_index()
        empty = torch.empty(0, dtype=torch.int32, device="cuda:0")
        P.topk(empty, 3)                                        # q = 0 is a no-op
        bad = torch.tensor([0, 6], dtype=torch.int32, device="cuda:0")
        P.topk(bad, 3)
        with pytest.raises(pk.PantherError):
            P.sync()                                            # out-of-range query reported
        with pytest.raises(pk.PantherError):
            P.topk(torch.zeros(1, dtype=torch.int32, device="cuda:0"), 129)


def test_topk_host_io(pk, small):
    with pk.Panther(0) as P:
        P.build_graph(small.row_ptr, small.col, small.w)
        P.sample_paths(1, 20_000, 5)
        P.build_index()
        q = np.arange(0, small.n, 3, dtype=np.int32)
        ids = np.empty((q.shape[0], 5), np.int32)
        cnt = np.empty((q.shape[0], 5), np.uint32)
        pk.panther_topk(P.h.ctx, P.h.index, P.h.paths, q, q.shape[0], 5, ids, cnt,
                        pk.TOPK_BATCHED | pk.IO_HOST)
    o = oracle.Oracle(small.n, oracle.sample_paths(small, 1, 20_000, 5, oracle.ALIAS))
    rid, rcnt = o.topk_many(q, 5)
    assert np.array_equal(ids, rid) and np.array_equal(cnt, rcnt)


def test_topk_host_io_large_batch_in_chunks(pk, small):
    # 4.5M queries (repeats of the 2,000 vertices) with host buffers: the call
    # answers them in chunks whose rows are copied back while the next chunk
    # computes; the rows equal the device-memory call's and the oracle's
    rng = np.random.default_rng(4)
    q = rng.integers(0, small.n, size=4_500_000).astype(np.int32)
    k = 10
    with pk.Panther(0) as P:
        P.build_graph(small.row_ptr, small.col, small.w)
        P.sample_paths(1, 20_000, 5)
        P.build_index()
        ids = np.empty((q.shape[0], k), np.int32)
        cnt = np.empty((q.shape[0], k), np.uint32)
        pk.panther_topk(P.h.ctx, P.h.index, P.h.paths, q, q.shape[0], k, ids, cnt,
                        pk.TOPK_BATCHED | pk.IO_HOST)
        st = pk.panther_topk_stats(P.h.ctx)
        dids, dcnt = P.topk(torch.as_tensor(q, device="cuda:0"), k)
        P.sync()
    assert st[0] == q.shape[0]
    assert np.array_equal(ids, dids.cpu().numpy()) and np.array_equal(cnt, dcnt.cpu().numpy().astype(np.uint32))
    o = oracle.Oracle(small.n, oracle.sample_paths(small, 1, 20_000, 5, oracle.ALIAS))
    rid, rcnt = o.topk_many(np.arange(small.n, dtype=np.int32), k)
    assert np.array_equal(ids, rid[q]) and np.array_equal(cnt, rcnt[q])


def test_batched_workload_full_size_sampled(pk):
    """N=1M Chung-Lu (mean degree 20, gamma 2.3, log-uniform weights), R from the
    sample-size bound (eps 0.01, delta 0.1, c 0.5), 16,384 queries (half from the
    top-1% degree set), top-5: every path compared, and top-5 of a sample of
    queries including the heaviest."""
    g = synth.workload_graph("batched")
    R = oracle.sample_size(0.01, 0.1, 0.5, 5)
    assert R == 33123
    q = synth.query_mix(g, 8192, 8192, seed=1)
    out = _run(pk, g, 1, R, 5, pk.MODE_ALIAS, k=5, queries=q)
    ref = oracle.sample_paths(g, 1, R, 5, oracle.ALIAS)
    assert np.array_equal(out["paths"], ref)
    off, pid = oracle.build_index(g.n, ref)
    assert np.array_equal(out["off"], off) and np.array_equal(out["pid"], pid)
    o = oracle.Oracle(g.n, ref, off, pid)
    sizes = np.diff(off)[q]
    pick = np.unique(np.concatenate([np.argsort(-sizes)[:64], np.arange(0, q.shape[0], 37)]))
    rid, rcnt = o.topk_many(q[pick], 5)
    assert np.array_equal(out["ids"][pick], rid)
    assert np.array_equal(out["cnt"][pick], rcnt)


def test_autotuner_keeps_results_exact(pk):
    g = synth.workload_graph("batched", n=200_000)
    R, T, k = 40_000, 5, 5
    q = synth.query_mix(g, 2048, 2048, seed=3)
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_ALIAS)
        P.sample_paths(11, R, T, pk.MODE_ALIAS)
        P.build_index()
        qt = torch.as_tensor(q, device="cuda:0")
        shape = P.tune_topk(qt, k)
        # one of the tuner's candidate shapes (which one wins depends on timing)
        assert shape[0] in (128, 256, 512, 1024) and shape[1] % 32 == 0 and 1 <= shape[2] <= 8
        ids, cnt = P.topk(qt, k)
        P.sync()
        ids, cnt = ids.cpu().numpy(), cnt.cpu().numpy().astype(np.uint32)
    o = oracle.Oracle(g.n, oracle.sample_paths(g, 11, R, T, oracle.ALIAS))
    rid, rcnt = o.topk_many(q, k)
    assert np.array_equal(ids, rid) and np.array_equal(cnt, rcnt)
