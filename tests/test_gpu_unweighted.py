"""The unweighted fast path (Eq. (3) with t_ij = 1/deg(i), the paper's
unweighted social networks, Sec. 5.1): no transition table; a step reads one
column entry. Its paths must equal the oracle's prefix-mode paths of the same
graph with every weight 1 (the same draw words and rejections), bit for bit;
the index and top-k over them must equal the oracle's."""
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


def _unit(g):
    return synth.Graph(g.n, g.row_ptr, g.col, np.ones_like(g.w), g.draws, g.max_degree, g.isolated)


@pytest.mark.parametrize("T", [1, 5, 9, 31])
def test_unweighted_paths_index_topk(pk, T):
    g = synth.workload_graph("small")
    R, k = 60_000, 10
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, None, pk.MODE_UNWEIGHTED)     # no weights at all
        P.sample_paths(3, R, T, pk.MODE_UNWEIGHTED)
        paths = P.paths_tensor().cpu().numpy()
        P.build_index()
        off, pid = P.index_tensors()
        ids, cnt = P.topk(torch.arange(g.n, dtype=torch.int32, device="cuda:0"), k)
        P.sync()
        off, pid, ids, cnt = off.cpu().numpy(), pid.cpu().numpy(), ids.cpu().numpy(), cnt.cpu().numpy()
    u = _unit(g)
    ref = oracle.sample_paths(u, 3, R, T, oracle.PREFIX)
    assert np.array_equal(paths, ref)
    roff, rpid = oracle.build_index(g.n, ref)
    assert np.array_equal(off, roff) and np.array_equal(pid, rpid)
    o = oracle.Oracle(g.n, ref, roff, rpid)
    rid, rcnt = o.topk_many(np.arange(g.n, dtype=np.int32), k, threads=THREADS)
    assert np.array_equal(ids, rid) and np.array_equal(cnt.astype(np.uint32), rcnt)


def test_unweighted_equals_gpu_prefix_with_unit_weights_and_ignores_weights(pk):
    # the 1M-vertex batched workload graph: the unweighted mode on the weighted
    # graph ignores its weights and equals prefix mode on the unit-weight graph
    g = synth.workload_graph("batched")
    R, T = 200_000, 5
    dev = "cuda:0"
    with pk.Panther(0) as P:
        P.build_graph(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev),
                      torch.from_numpy(g.w.view(np.int32)).to(dev), pk.MODE_UNWEIGHTED | pk.MODE_ALIAS)
        P.sample_paths(9, R, T, pk.MODE_UNWEIGHTED)
        a = P.paths_tensor().cpu().numpy()
    with pk.Panther(0) as P:
        P.build_graph(g.row_ptr, g.col, np.ones_like(g.w), pk.MODE_PREFIX)
        P.sample_paths(9, R, T, pk.MODE_PREFIX)
        b = P.paths_tensor().cpu().numpy()
    assert np.array_equal(a, b)
    ref = oracle.sample_paths(_unit(g), 9, R, T, oracle.PREFIX, threads=THREADS)
    assert np.array_equal(a, ref)


def test_unweighted_validation_and_mode_errors(pk):
    # an asymmetric structure is refused without weights too; sampling in a
    # mode the graph was not built for is refused
    n = 4
    rp = np.array([0, 2, 3, 4, 4], np.int64)
    col = np.array([1, 2, 0, 0], np.int32)          # 0->1, 0->2, 1->0, 2->0: symmetric
    with pk.Panther(0) as P:
        P.build_graph(rp, col, None, pk.MODE_UNWEIGHTED)
        with pytest.raises(pk.PantherError):
            P.sample_paths(1, 10, 3, pk.MODE_ALIAS)
        P.sample_paths(1, 10, 3, pk.MODE_UNWEIGHTED)
        P.sync()
        bad = np.array([1, 2, 0, 1], np.int32)       # 2->1 without 1->2
        with pytest.raises(pk.PantherError):
            P.build_graph(rp, bad, None, pk.MODE_UNWEIGHTED)
        with pytest.raises(pk.PantherError):
            P.build_graph(rp, col, None, pk.MODE_ALIAS)   # weights needed for a table
