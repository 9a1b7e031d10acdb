"""The request loop: mixed top-k / k-NN requests from several host threads give
the same result as the same request alone and as the CPU oracle (top-k rows of
Algorithm 1, exact k-NN of Sec. 3.3 on the oracle's theta); admission by
memory budget."""
import os
import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_02577_gb300 as pk
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = synth.workload_graph("small")
    ctx = pk.panther_create(0)
    gh = pk.panther_build_graph(ctx, g.n, g.m, g.row_ptr, g.col, g.w, pk.MEM_HOST, pk.MODE_ALIAS)
    ph = pk.panther_sample_paths(ctx, gh, 1, 200_000, 5, pk.MODE_ALIAS)
    ih = pk.panther_build_index(ctx, ph)
    vh = pk.pantherpp_vectors(ctx, ih, ph, 50)
    pk.panther_sync(ctx)
    yield pk, g, ctx, ih, ph, vh
    pk.pantherpp_free_vecs(vh)
    pk.panther_free_index(ih)
    pk.panther_free_paths(ph)
    pk.panther_free_graph(gh)
    pk.panther_destroy(ctx)


def _alone(pk, ctx, ih, ph, vh, kind, q, k):
    ids = np.empty((q.shape[0], k), np.int32)
    if kind == 0:
        vals = np.empty((q.shape[0], k), np.uint32)
        pk.panther_topk(ctx, ih, ph, q, q.shape[0], k, ids, vals, pk.TOPK_BATCHED | pk.IO_HOST)
    else:
        vals = np.empty((q.shape[0], k), np.uint64)
        pk.pantherpp_knn(ctx, vh, q, q.shape[0], k, ids, vals, pk.KNN_BF16_SCREEN | pk.IO_HOST)
    return ids, vals


def test_mixed_requests_equal_alone(env):
    pk, g, ctx, ih, ph, vh = env
    srv = pk.panther_serve_create(0, ih, ph, vh, 256 << 20, 1000, 3)
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(90):
        kind = 0 if rng.random() < 0.75 else 1
        k = int(rng.choice([5, 10, 50])) if kind == 0 else 10
        size = int(np.floor(4097 ** rng.random())) if kind == 0 else int(np.floor(1025 ** rng.random()))
        size = max(1, min(size, 600))
        q = rng.integers(0, g.n, size=size).astype(np.int32)
        ids = np.empty((size, k), np.int32)
        vals = np.empty((size, k), np.uint32 if kind == 0 else np.uint64)
        reqs.append((kind, q, k, ids, vals))
    tickets = [None] * len(reqs)
    lat = [None] * len(reqs)

    def client(lo, hi):
        for i in range(lo, hi):
            kind, q, k, ids, vals = reqs[i]
            tickets[i] = pk.panther_serve_submit(srv, kind, q, k, ids, vals)
        for i in range(lo, hi):
            lat[i] = pk.panther_serve_wait(srv, tickets[i], 120.0)

    th = [threading.Thread(target=client, args=(j * 30, (j + 1) * 30)) for j in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    st = pk.panther_serve_stats(srv)
    pk.panther_serve_destroy(srv)
    assert st[0] == st[1] == 90
    assert st[3] >= 2 or st[4] >= 2        # requests were batched or batches overlapped
    assert all(x is not None and x >= 0 for x in lat)
    for kind, q, k, ids, vals in reqs:
        a_ids, a_vals = _alone(pk, ctx, ih, ph, vh, kind, q, k)
        assert np.array_equal(ids, a_ids)
        assert np.array_equal(vals, a_vals)
    # every result against the oracle (same paths: seed 1, R = 200,000, T = 5)
    th = os.cpu_count() or 1
    o = oracle.Oracle(g.n, oracle.sample_paths(g, 1, 200_000, 5, oracle.ALIAS, threads=th))
    theta = o.theta_all(50, threads=th)
    for kind, q, k, ids, vals in reqs:
        if kind == 0:
            rid, rcnt = o.topk_many(q, k, threads=th)
            assert np.array_equal(ids, rid) and np.array_equal(vals, rcnt)
        else:
            for i, v in enumerate(q):
                rid, rd = oracle.knn(theta, int(v), k)
                assert np.array_equal(ids[i], rid) and np.array_equal(vals[i], rd)


def test_admission_and_refusal(env):
    pk, g, ctx, ih, ph, vh = env
    # a budget that holds only a few hundred queries per worker
    srv = pk.panther_serve_create(0, ih, ph, vh, 1 << 20, 4, 1)
    big = np.zeros(5000, np.int32)
    ids = np.empty((5000, 5), np.int32)
    vals = np.empty((5000, 5), np.uint32)
    with pytest.raises(pk.PantherError):
        pk.panther_serve_submit(srv, 0, big, 5, ids, vals)          # larger than the budget: EBUSY
    q = np.arange(10, dtype=np.int32)
    outs = [(np.empty((10, 5), np.int32), np.empty((10, 5), np.uint32)) for _ in range(6)]
    tk, refused = [], 0
    for o in outs:
        try:
            tk.append(pk.panther_serve_submit(srv, 0, q, 5, o[0], o[1]))
        except pk.PantherError:
            refused += 1
    for t in tk:
        pk.panther_serve_wait(srv, t, 60.0)
    st = pk.panther_serve_stats(srv)
    pk.panther_serve_destroy(srv)
    assert st[5] >= 1 and refused == st[5] - 1
    bad = np.array([g.n], np.int32)
    srv = pk.panther_serve_create(0, ih, ph, vh, 64 << 20, 4, 1)
    with pytest.raises(pk.PantherError):
        pk.panther_serve_submit(srv, 0, bad, 5, ids, vals)           # query out of range
    pk.panther_serve_destroy(srv)
