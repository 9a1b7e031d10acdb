"""The binding checks caller buffers before the C call (no GPU needed).

A buffer with the wrong element size (a numpy default int64 query array where
the ABI reads int32) or fewer elements than the call writes is refused with
ValueError before any pointer reaches the library. Well-formed buffers pass
through, and the library then rejects the NULL context with EINVAL, which
shows that the call was made.
"""
import numpy as np
import pytest

import paper_1504_02577_gb300 as pk

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1504_02577_gb300 import build
    build.build()
    pk.load_library()


def _reaches_library(fn, *args):
    with pytest.raises(pk.PantherError) as ei:
        fn(*args)
    assert ei.value.code == pk.EINVAL


@pytest.mark.parametrize("lib", ["numpy", "torch"])
def test_topk_buffers(lib):
    q, k = 7, 5
    if lib == "numpy":
        good_q = np.zeros(q, np.int32)
        wide_q = np.zeros(q, np.int64)
        ids, cnt = np.empty((q, k), np.int32), np.empty((q, k), np.uint32)
        short = np.empty((q, k - 1), np.int32)
    else:
        good_q = torch.zeros(q, dtype=torch.int32)
        wide_q = torch.zeros(q, dtype=torch.int64)
        ids, cnt = torch.empty((q, k), dtype=torch.int32), torch.empty((q, k), dtype=torch.int32)
        short = torch.empty((q, k - 1), dtype=torch.int32)
    _reaches_library(pk.panther_topk, 0, 0, 0, good_q, q, k, ids, cnt)
    _reaches_library(pk.panther_tune_topk, 0, 0, 0, good_q, q, k, ids, cnt)
    with pytest.raises(ValueError, match="queries"):
        pk.panther_topk(0, 0, 0, wide_q, q, k, ids, cnt)
    with pytest.raises(ValueError, match="out_ids"):
        pk.panther_topk(0, 0, 0, good_q, q, k, short, cnt)
    with pytest.raises(ValueError, match="out_counts"):
        pk.panther_tune_topk(0, 0, 0, good_q, q, k, ids, short)
    with pytest.raises(ValueError, match="queries"):
        pk.panther_topk(0, 0, 0, good_q[: q - 1], q, k, ids, cnt)


def test_knn_buffers():
    q, k = 4, 3
    good_q = np.arange(q, dtype=np.int32)
    ids, d2 = np.empty((q, k), np.int32), np.empty((q, k), np.uint64)
    _reaches_library(pk.pantherpp_knn, 0, 0, good_q, q, k, ids, d2)
    _reaches_library(pk.pantherpp_knn_cross, 0, 0, 0, good_q, q, k, ids, d2)
    with pytest.raises(ValueError, match="out_dist2"):
        pk.pantherpp_knn(0, 0, good_q, q, k, ids, np.empty((q, k), np.uint32))
    with pytest.raises(ValueError, match="out_ids"):
        pk.pantherpp_knn_cross(0, 0, 0, good_q, q, k, np.empty((q, k), np.int64), d2)


def test_graph_buffers():
    n, m = 3, 4
    rp = np.array([0, 2, 3, 4], np.int64)
    col = np.array([1, 2, 0, 0], np.int32)
    w = np.ones(m, np.uint32)
    _reaches_library(pk.panther_build_graph, 0, n, m, rp, col, w, pk.MEM_HOST)
    with pytest.raises(ValueError, match="row_ptr"):
        pk.panther_build_graph(0, n, m, rp.astype(np.int32), col, w, pk.MEM_HOST)
    with pytest.raises(ValueError, match="col"):
        pk.panther_build_graph(0, n, m + 1, rp, col, np.ones(m + 1, np.uint32), pk.MEM_HOST)
    with pytest.raises(ValueError, match="w"):
        pk.panther_build_graph(0, n, m, rp, col, w.astype(np.float64), pk.MEM_HOST)


def test_serve_and_noalloc_buffers():
    q, k = 3, 2
    good_q = np.zeros(q, np.int32)
    _reaches_library(pk.panther_serve_submit, 0, 0, good_q, k, np.empty((q, k), np.int32),
                     np.empty((q, k), np.uint32))
    _reaches_library(pk.panther_serve_submit, 0, 1, good_q, k, np.empty((q, k), np.int32),
                     np.empty((q, k), np.uint64))
    with pytest.raises(ValueError, match="out_vals"):
        pk.panther_serve_submit(0, 1, good_q, k, np.empty((q, k), np.int32), np.empty((q, k), np.uint32))
    _reaches_library(pk.panther_build_index_noalloc, 0, 0, np.empty(4, np.int64), np.empty(8, np.int32), 8)
    with pytest.raises(ValueError, match="dev_pid"):
        pk.panther_build_index_noalloc(0, 0, np.empty(4, np.int64), np.empty(8, np.int64), 8)
    # a pid buffer shorter than the capacity the library is told it has
    with pytest.raises(ValueError, match="dev_pid"):
        pk.panther_build_index_noalloc(0, 0, np.empty(4, np.int64), np.empty(7, np.int32), 8)
    with pytest.raises(ValueError, match="dev_pid"):
        pk.panther_build_index_noalloc(0, 0, np.empty(4, np.int64), torch.empty(7, dtype=torch.int32), 8)
    with pytest.raises(ValueError, match="dev_off"):
        pk.panther_build_index_noalloc(0, 0, np.empty(4, np.int32), np.empty(8, np.int32), 8)


def test_raw_pointers_and_null_pass_unchecked():
    # integers are raw pointers and None is NULL: nothing to inspect, the
    # library decides (here: EINVAL for the NULL context)
    _reaches_library(pk.panther_topk, 0, 0, 0, None, 0, 1, None, None)
    _reaches_library(pk.pantherpp_knn, 0, 0, 0, 0, 1, 0, 0)
