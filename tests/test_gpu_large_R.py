"""Path sets of more than 2^31 - 1 paths, checked against the oracle.

The paper sizes R from its bound with eps = sqrt(1/|E|) (Sec. 3.4), which on
its largest networks reaches about 3.3e9 paths (Table 2). The library keeps
path ids as uint32 (R <= 2^32 - 1), so ids from 2^31 up must travel through
the sampler, the radix sort (single pass and chunked), every counting tier,
theta and the k-NN unchanged. R here is 2^31 + 2^25 + 7, so about 33.5
million ids lie above 2^31 - 1.

The oracle cannot hold 2.2e9 paths and their index, so it counts from the
definition (oracle.stream_counts: paths drawn one by one, Eq. (4) and |P_v|
accumulated, nothing stored) and draws single paths by id (oracle.paths_at).
An index list is proven equal to P_v by three facts: it ascends strictly,
every listed path holds v, and its length is |P_v|.

Device memory: 70 GB of rows and two 17 GB indexes, plus the index build's
temporary buffers (the build goes to chunks of paths when they do not fit):
the tests want about 150 GB free.
"""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
THREADS = os.cpu_count() or 1
R_BIG = 2**31 + 2**25 + 7
DEV = "cuda:0"


@pytest.fixture(scope="module")
def pk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_02577_gb300 as pk
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info(0)
    if free < 150e9:
        pytest.skip("needs about 150 GB of free device memory")
    return pk


def _u32(t):
    """int32 storage of uint32 values, widened."""
    return t.to(torch.int64) & 0xFFFFFFFF


def _index(pk, ix, n):
    off_ptr, pid_ptr, n_, nnz = pk.panther_index_view(ix)
    assert n_ == n
    off = pk._device_view(torch, off_ptr, (n + 1,), torch.int64, 0)
    pid = pk._device_view(torch, pid_ptr, (max(nnz, 1),), torch.int32, 0)[:nnz]
    return off, pid, nnz


def test_r_above_2_32_is_refused(pk):
    g = synth.graph_from_edges(2, [(0, 1)], [1])
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_ALIAS)
        with pytest.raises(pk.PantherError) as ei:
            P.sample_paths(1, 2**32, 3, pk.MODE_ALIAS)
        assert ei.value.code == pk.EOVERFLOW


def test_two_vertex_graph_closed_form(pk):
    # one edge {0, 1}: every path alternates between the two vertices, so both
    # lie on all R paths: P_0 = P_1 = {0 .. R-1} and cnt(0,1) = R > 2^31.
    # Their queries have 2.2e9 paths and one candidate each.
    g = synth.graph_from_edges(2, [(0, 1)], [5])
    R = R_BIG
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_ALIAS)
        P.sample_paths(3, R, 5, pk.MODE_ALIAS)
        P.build_index()
        P.sync()
        off, pid, nnz = _index(pk, P.h.index, 2)
        assert nnz == 2 * R
        assert off.cpu().tolist() == [0, R, 2 * R]
        step = 1 << 28
        for v in (0, 1):
            for s in range(0, R, step):
                e = min(R, s + step)
                want = torch.arange(s, e, dtype=torch.int64, device=DEV)
                assert torch.equal(_u32(pid[v * R + s: v * R + e]), want), (v, s)
        del want
        q = torch.tensor([0, 1], dtype=torch.int32, device=DEV)
        before = pk.panther_topk_stats(P.h.ctx)
        ids, cnt = P.topk(q, 3)
        after = pk.panther_topk_stats(P.h.ctx)
        assert ids.cpu().tolist() == [[1, -1, -1], [0, -1, -1]]
        assert _u32(cnt).cpu().tolist() == [[R, 0, 0], [R, 0, 0]]
        assert after[5] - before[5] == 2                  # both through the hub tier
        P.vectors(D=2)
        assert _u32(P.theta_tensor()).cpu().tolist() == [[R, 0], [R, 0]]
        nn, d2 = P.knn(q, 1)
        assert nn.cpu().tolist() == [[1], [0]] and d2.cpu().tolist() == [[0], [0]]


def test_chung_lu_against_streaming_oracle(pk):
    # the small-graph shape (Chung-Lu n = 2,000, mean degree 10, exponent
    # 2.5, weights uniform in [1, 16]) with T = 1 and R = 2^31 + 2^25 + 7
    g = synth.chung_lu(2000, 10, 2.5, ("uniform", 1, 16), seed=1)
    R, T, k, D, seed = R_BIG, 1, 10, 16, 7
    cuts = [(0, 500), (2**31 - 1000, 2**31 + 1000), (R - 777, R)]
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_ALIAS)
        P.sample_paths(seed, R, T, pk.MODE_ALIAS)
        P.build_index()
        P.sync()
        rows_ptr, R_, L, stride = pk.panther_paths_view(P.h.paths)
        assert R_ == R and L == T + 1
        rows = pk._device_view(torch, rows_ptr, (R, stride), torch.int32, 0)
        gpu_rows = [rows[a:b, :L].cpu().numpy() for a, b in cuts]
        off, pid, nnz = _index(pk, P.h.index, g.n)
        gpu_off = off.cpu().numpy()
        # the chunked build (a small budget, several chunks of paths whose ids
        # cross 2^31) gives the same index
        pk.panther_set_index_budget(P.h.ctx, 8 << 30)
        ix2 = pk.panther_build_index(P.h.ctx, P.h.paths)
        pk.panther_sync(P.h.ctx)
        off2, pid2, nnz2 = _index(pk, ix2, g.n)
        assert nnz2 == nnz and torch.equal(off2, off) and torch.equal(pid2, pid)
        del off2, pid2
        pk.panther_free_index(ix2)
        pk.panther_set_index_budget(P.h.ctx, 0)
        sizes = np.diff(gpu_off)
        rng = np.random.default_rng(5)
        check_v = list(np.argsort(sizes, kind="stable")[:3]) + [int(rng.integers(0, g.n))]
        lists = {int(v): _u32(pid[gpu_off[v]:gpu_off[v + 1]]).cpu().numpy() for v in check_v}
        del off, pid
        allq = torch.arange(g.n, dtype=torch.int32, device=DEV)
        ids, cnt = P.topk(allq, k)
        ids, cnt = ids.cpu().numpy(), _u32(cnt).cpu().numpy()
        P.vectors(D=D)
        theta = _u32(P.theta_tensor()).cpu().numpy()
        nn, d2 = P.knn(allq, k)
        nn, d2 = nn.cpu().numpy(), d2.cpu().numpy().astype(np.uint64)
        del rows
    tables = oracle.alias_tables(g)
    for (a, b), got in zip(cuts, gpu_rows):
        ref = oracle.sample_paths(g, seed, b - a, T, oracle.ALIAS, r0=a, tables=tables, threads=THREADS)
        assert np.array_equal(got, ref), f"paths {a}..{b} differ"
    cnt_ref, npaths = oracle.stream_counts(g, seed, 0, R, T, np.arange(g.n, dtype=np.int32), oracle.ALIAS,
                                           tables=tables, threads=THREADS)
    assert np.array_equal(sizes, npaths), "|P_v| differs"
    assert int(npaths.sum()) == nnz
    for v, lst in lists.items():
        assert lst.size == npaths[v]
        assert np.all(np.diff(lst) > 0), f"P_{v} does not ascend"
        assert lst[-1] > 2**31 - 1                       # the list reaches ids above 2^31 - 1
        held = oracle.paths_at(g, seed, lst, T, oracle.ALIAS, tables=tables, threads=THREADS)
        assert np.all((held == v).any(axis=1)), f"P_{v} lists a path without {v}"
    th_ref = np.zeros((g.n, D), dtype=np.uint64)
    for v in range(g.n):
        rid, rc = oracle.topk_from_counts(cnt_ref[v], v, k)
        assert np.array_equal(ids[v], rid) and np.array_equal(cnt[v], rc), f"top-{k} of {v} differs"
        row = cnt_ref[v].copy()
        row[v] = 0
        top = np.sort(row)[::-1][:D]
        th_ref[v, :top.size] = top
    assert np.array_equal(theta, th_ref), "theta differs"
    rnn, rd2 = oracle.knn_many(th_ref.astype(np.uint32), np.arange(g.n, dtype=np.int32), k, threads=THREADS)
    assert np.array_equal(nn, rnn) and np.array_equal(d2, rd2), "k-NN differs"
