"""The 50M-vertex workload the benchmark times, checked against the oracle.

Chung-Lu graph n = 50,000,000, mean degree 16, exponent 2.1, weights uniform
in [1, 255], seed 1; R = 1e8 paths of T = 5 steps (alias selection), the
inverted index of all of them, and top-10 of every vertex in the batched,
autotuned form the benchmark runs. Compared bit for bit with the oracle (its
all-core driver, identical to the single-threaded code): every path
(Algorithm 3), the whole index (Sec. 3.1: off and pid), and the top-10 rows
(Algorithm 1, Eq. (4)) of 2,000 uniformly drawn vertices plus the 64 vertices
with the most paths, whose counts run through the hub tiers (pruned device
tables and buckets) that only this size reaches.
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


def test_scale_workload_paths_index_topk(pk):
    p = synth.WORKLOADS["scale"]
    g = synth.workload_graph("scale")
    R, T, k = p["R"], p["T"], p["k"]
    assert g.n == 50_000_000 and g.m == 800_000_000
    with pk.Panther(0) as P:
        dev = "cuda:0"
        P.build_graph(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev),
                      torch.from_numpy(g.w.view(np.int32)).to(dev), pk.MODE_ALIAS)
        P.sample_paths(1, R, T, pk.MODE_ALIAS)
        P.build_index()
        allq = torch.arange(g.n, dtype=torch.int32, device=dev)
        P.tune_topk(allq, k)
        ids, cnt = P.topk(allq, k)
        P.sync()
        st = pk.panther_topk_stats(P.h.ctx)
        gpu_paths = P.paths_tensor().cpu().numpy()
        off_t, pid_t = P.index_tensors()
        gpu_off, gpu_pid = off_t.cpu().numpy(), pid_t.cpu().numpy()
        del off_t, pid_t
        ids, cnt = ids.cpu().numpy(), cnt.cpu().numpy().astype(np.uint32)
    assert st[5] > 0 and st[6] + st[7] >= st[5]          # hub queries were counted
    tables = oracle.alias_tables(g, threads=THREADS)
    ref = oracle.sample_paths(g, 1, R, T, oracle.ALIAS, tables=tables, threads=THREADS)
    del tables
    assert np.array_equal(gpu_paths, ref), "paths differ from the oracle"
    del gpu_paths
    off, pid = oracle.build_index(g.n, ref, threads=THREADS)
    assert np.array_equal(gpu_off, off), "index offsets differ"
    assert np.array_equal(gpu_pid, pid), "index path ids differ"
    del gpu_off, gpu_pid
    o = oracle.Oracle(g.n, ref, off, pid)
    sizes = np.diff(off)
    rng = np.random.default_rng(2024)
    heavy = np.argsort(-sizes, kind="stable")[:64]
    q = np.unique(np.concatenate([heavy, rng.integers(0, g.n, 2000)])).astype(np.int32)
    assert sizes[heavy[0]] > 1_000_000
    rid, rcnt = o.topk_many(q, k, threads=THREADS)
    assert np.array_equal(ids[q], rid), "top-10 ids differ"
    assert np.array_equal(cnt[q], rcnt), "top-10 counts differ"


def test_knn_workload_theta_all_and_sampled_knn(pk):
    """The 10M-vertex Panther++ workload (Chung-Lu mean degree 20, exponent
    2.3, log-uniform weights in [1, 1024], R = 5e7, T = 5, D = 50): theta of
    every vertex equal to the oracle's (Sec. 3.3), and the exact top-10
    nearest vectors (BF16 screen + exact rerank, the form the benchmark
    times) of 96 uniform queries and the 32 vertices with the largest theta
    norms equal to the oracle's all-pairs search."""
    p = synth.WORKLOADS["knn"]
    g = synth.workload_graph("knn")
    R, T, D, k = p["R"], p["T"], p["D"], p["k"]
    with pk.Panther(0) as P:
        dev = "cuda:0"
        P.build_graph(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev),
                      torch.from_numpy(g.w.view(np.int32)).to(dev), pk.MODE_ALIAS)
        P.sample_paths(1, R, T, pk.MODE_ALIAS)
        P.build_index()
        P.vectors(D)
        theta = P.theta_tensor().cpu().numpy().view(np.uint32)
        norm2 = (theta.astype(np.int64) ** 2).sum(axis=1)
        rng = np.random.default_rng(77)
        q = np.concatenate([np.argsort(-norm2, kind="stable")[:32], rng.integers(0, g.n, 96)]).astype(np.int32)
        ids, d2 = P.knn(torch.as_tensor(q, device=dev), k)
        P.sync()
        ids, d2 = ids.cpu().numpy(), d2.cpu().numpy().view(np.uint64)
    tables = oracle.alias_tables(g, threads=THREADS)
    ref = oracle.sample_paths(g, 1, R, T, oracle.ALIAS, tables=tables, threads=THREADS)
    del tables
    o = oracle.Oracle(g.n, ref)
    rth = o.theta_all(D, threads=THREADS)
    assert np.array_equal(theta, rth), "theta differs from the oracle"
    assert rth.max() > 256                              # inexact BF16 rows exist: the bound decides
    rid, rd = oracle.knn_many(rth, q, k, threads=THREADS)
    assert np.array_equal(ids, rid), "k-NN ids differ"
    assert np.array_equal(d2, rd), "k-NN distances differ"


def test_index_beyond_2pow31_pairs(pk):
    """More (vertex, path) pairs than an int32 position can address: 450M
    paths of T = 5 on a 2,000-vertex graph give about 2.5e9 pairs (the regime
    of the paper's own sample size, R = c/eps^2 (...) with eps = sqrt(1/|E|),
    on large graphs). Every path, the whole index (int64 offsets past 2^31)
    and the top-10 of 40 vertices equal the oracle's."""
    g = synth.workload_graph("small")
    R, T, k = 450_000_000, 5, 10
    q = np.arange(0, g.n, 50, dtype=np.int32)
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, g.w, pk.MODE_ALIAS)
        P.sample_paths(21, R, T, pk.MODE_ALIAS)
        P.build_index()
        ids, cnt = P.topk(torch.as_tensor(q, device="cuda:0"), k)
        P.sync()
        ids, cnt = ids.cpu().numpy(), cnt.cpu().numpy().astype(np.uint32)
        _, _, _, nnz = pk.panther_index_view(P.h.index)
        assert nnz > 2**31
        gpu_paths = P.paths_tensor().cpu().numpy()
        ref = oracle.sample_paths(g, 21, R, T, oracle.ALIAS, threads=THREADS)
        assert np.array_equal(gpu_paths, ref), "paths differ from the oracle"
        del gpu_paths
        off_t, pid_t = P.index_tensors()
        gpu_off = off_t.cpu().numpy()
        gpu_pid = pid_t.cpu().numpy()
        del off_t, pid_t
    off, pid = oracle.build_index(g.n, ref, threads=THREADS)
    assert off[-1] == nnz
    assert np.array_equal(gpu_off, off), "index offsets differ"
    assert np.array_equal(gpu_pid, pid), "index path ids differ"
    del gpu_pid
    o = oracle.Oracle(g.n, ref, off, pid)
    rid, rcnt = o.topk_many(q, k, threads=THREADS)
    assert np.array_equal(ids, rid) and np.array_equal(cnt, rcnt)
