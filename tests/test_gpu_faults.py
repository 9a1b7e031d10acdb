"""Failure handling without a device fault: a bounded device wait that runs
out (a flag nothing sets), injected allocation failures at every allocation
of every step, and a serving wait that times out. After each, the context
keeps working and the results still equal the oracle's."""
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


def _graph():
    return synth.chung_lu(3000, 8, 2.3, ("uniform", 1, 9), seed=21)


R, T, K, D = 30_000, 5, 10, 16


def _reference(g):
    P = oracle.sample_paths(g, 3, R, T, oracle.ALIAS)
    o = oracle.Oracle(g.n, P)
    q = np.arange(0, g.n, 7, dtype=np.int32)
    ids, cnt = o.topk_many(q, K)
    th = o.theta_all(D)
    kn = [oracle.knn(th, int(v), K) for v in q]
    return q, ids, cnt, kn


def _steps(pk, ctx, g, q):
    """The path as a list of (name, call) where each call takes the handles so far."""
    h = {}

    def graph():
        h["g"] = pk.panther_build_graph(ctx, g.n, g.m, g.row_ptr, g.col, g.w, pk.MEM_HOST, pk.MODE_ALIAS)

    def paths():
        h["p"] = pk.panther_sample_paths(ctx, h["g"], 3, R, T, pk.MODE_ALIAS)

    def index():
        h["ix"] = pk.panther_build_index(ctx, h["p"])

    def topk():
        ids = np.empty((q.size, K), np.int32)
        cnt = np.empty((q.size, K), np.uint32)
        pk.panther_topk(ctx, h["ix"], h["p"], q, q.size, K, ids, cnt, pk.TOPK_BATCHED | pk.IO_HOST)
        h["topk"] = (ids, cnt)

    def vectors():
        h["v"] = pk.pantherpp_vectors(ctx, h["ix"], h["p"], D)

    def knn():
        ids = np.empty((q.size, K), np.int32)
        d2 = np.empty((q.size, K), np.uint64)
        pk.pantherpp_knn(ctx, h["v"], q, q.size, K, ids, d2, pk.KNN_BF16_SCREEN | pk.IO_HOST)
        h["knn"] = (ids, d2)

    return h, [("graph", graph), ("paths", paths), ("index", index), ("topk", topk), ("vectors", vectors),
               ("knn", knn)]


def test_wait_timeout_reported_and_context_usable(pk):
    g = _graph()
    q, rid, rcnt, _ = _reference(g)
    ctx = pk.panther_create(0)
    try:
        with pytest.raises(pk.PantherError) as e:
            pk.panther_debug_wait_timeout(ctx, 1 << 20)
        assert e.value.code == pk.ETIMEOUT
        pk.panther_sync(ctx)                      # the status word was cleared
        h, steps = _steps(pk, ctx, g, q)
        for _, call in steps[:4]:
            call()
        assert np.array_equal(h["topk"][0], rid) and np.array_equal(h["topk"][1], rcnt)
        for key, free in (("ix", pk.panther_free_index), ("p", pk.panther_free_paths), ("g", pk.panther_free_graph)):
            free(h[key])
    finally:
        pk.panther_destroy(ctx)


def test_injected_allocation_failures(pk):
    g = _graph()
    q, rid, rcnt, kn = _reference(g)
    ctx = pk.panther_create(0)
    try:
        h, steps = _steps(pk, ctx, g, q)
        for name, call in steps:
            failures = 0
            for nth in range(64):
                pk.panther_debug_fail_alloc(ctx, nth)
                try:
                    call()
                except pk.PantherError as e:
                    assert e.code == pk.ENOMEM, (name, nth, str(e))
                    failures += 1
                    continue
                break
            pk.panther_debug_fail_alloc(ctx, -1)
            assert failures >= 1, name            # every step allocates, so the first one failed
            pk.panther_sync(ctx)
        assert np.array_equal(h["topk"][0], rid) and np.array_equal(h["topk"][1], rcnt)
        ids, d2 = h["knn"]
        for i in range(q.size):
            assert ids[i].tolist() == kn[i][0].tolist() and d2[i].tolist() == kn[i][1].tolist(), i
        pk.pantherpp_free_vecs(h["v"])
        pk.panther_free_index(h["ix"])
        pk.panther_free_paths(h["p"])
        pk.panther_free_graph(h["g"])
    finally:
        pk.panther_destroy(ctx)


def test_serve_wait_times_out_then_completes(pk):
    g = _graph()
    ctx = pk.panther_create(0)
    gh = pk.panther_build_graph(ctx, g.n, g.m, g.row_ptr, g.col, g.w, pk.MEM_HOST, pk.MODE_ALIAS)
    ph = pk.panther_sample_paths(ctx, gh, 3, R, T, pk.MODE_ALIAS)
    ih = pk.panther_build_index(ctx, ph)
    pk.panther_sync(ctx)
    srv = pk.panther_serve_create(0, ih, ph, None, 64 << 20, 8, 1)
    try:
        q = np.arange(g.n, dtype=np.int32)
        ids = np.empty((g.n, K), np.int32)
        cnt = np.empty((g.n, K), np.uint32)
        t = pk.panther_serve_submit(srv, 0, q, K, ids, cnt)
        try:
            pk.panther_serve_wait(srv, t, 1e-7)   # far too short: times out, the request stays queued
            timed_out = False
        except pk.PantherError as e:
            assert e.code == pk.ETIMEOUT
            timed_out = True
        if timed_out:
            pk.panther_serve_wait(srv, t, 120.0)
        o = oracle.Oracle(g.n, oracle.sample_paths(g, 3, R, T, oracle.ALIAS))
        rid, rcnt = o.topk_many(q, K)
        assert np.array_equal(ids, rid) and np.array_equal(cnt, rcnt)
    finally:
        pk.panther_serve_destroy(srv)
        pk.panther_free_index(ih)
        pk.panther_free_paths(ph)
        pk.panther_free_graph(gh)
        pk.panther_destroy(ctx)
