"""Path ranges (resume from any path id) and checkpoint files of paths and
index: a range equals the same rows of a run from 0 and the oracle's; a
saved and reloaded index answers exactly like the original; damaged files
are refused before any use."""
import os

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


def _rows(pk, ph):
    rows, R, L, stride = pk.panther_paths_view(ph)
    t = pk._device_view(torch, rows, (R, stride), torch.int32, 0)
    return t[:, :L].cpu().numpy()


@pytest.mark.parametrize("mode", ["alias", "prefix"])
def test_path_range_equals_full_run_and_oracle(pk, mode):
    g = synth.workload_graph("small")
    m = pk.MODE_ALIAS if mode == "alias" else pk.MODE_PREFIX
    ctx = pk.panther_create(0)
    try:
        gh = pk.panther_build_graph(ctx, g.n, g.m, g.row_ptr, g.col, g.w, pk.MEM_HOST, pk.MODE_BOTH)
        full = pk.panther_sample_paths(ctx, gh, 5, 6000, 5, m)
        part = pk.panther_sample_paths_range(ctx, gh, 5, 1234, 3000, 5, m)
        pk.panther_sync(ctx)
        a, b = _rows(pk, full), _rows(pk, part)
        assert np.array_equal(b, a[1234:4234])
        ref = oracle.sample_paths(g, 5, 3000, 5, oracle.ALIAS if mode == "alias" else oracle.PREFIX, r0=1234)
        assert np.array_equal(b, ref)
        for h in (part, full):
            pk.panther_free_paths(h)
        pk.panther_free_graph(gh)
    finally:
        pk.panther_destroy(ctx)


def test_checkpoint_round_trip_and_damaged_files(pk, tmp_path):
    g = synth.workload_graph("small")
    ctx = pk.panther_create(0)
    ctx2 = pk.panther_create(0)
    try:
        gh = pk.panther_build_graph(ctx, g.n, g.m, g.row_ptr, g.col, g.w, pk.MEM_HOST, pk.MODE_ALIAS)
        ph = pk.panther_sample_paths_range(ctx, gh, 9, 777, 50_000, 5, pk.MODE_ALIAS)
        ih = pk.panther_build_index(ctx, ph)
        pk.panther_sync(ctx)
        fp, fi = str(tmp_path / "p.bin"), str(tmp_path / "i.bin")
        pk.panther_save_paths(ph, fp)
        pk.panther_save_index(ih, fi)
        ph2 = pk.panther_load_paths(ctx2, fp)
        ih2 = pk.panther_load_index(ctx2, fi)
        assert np.array_equal(_rows(pk, ph), _rows(pk, ph2))
        q = np.arange(g.n, dtype=np.int32)
        outs = []
        for c, p_, i_ in ((ctx, ph, ih), (ctx2, ph2, ih2)):
            ids = np.empty((g.n, 10), np.int32)
            cnt = np.empty((g.n, 10), np.uint32)
            pk.panther_topk(c, i_, p_, q, g.n, 10, ids, cnt, pk.TOPK_BATCHED | pk.IO_HOST)
            outs.append((ids, cnt))
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
        o = oracle.Oracle(g.n, oracle.sample_paths(g, 9, 50_000, 5, oracle.ALIAS, r0=777))
        rid, rcnt = o.topk_many(q, 10)
        assert np.array_equal(outs[1][0], rid) and np.array_equal(outs[1][1], rcnt)

        raw = open(fi, "rb").read()
        bad = []
        b1 = bytearray(raw); b1[0:8] = b"NOTANIDX"; bad.append(bytes(b1))          # wrong magic
        bad.append(raw[: len(raw) // 2])                                            # truncated
        b3 = bytearray(raw)                                                         # offsets decrease
        off = np.frombuffer(bytes(b3[64:64 + 8 * (g.n + 1)]), dtype=np.int64).copy()
        off[g.n // 2] = off[g.n // 2 + 1] + 5
        b3[64:64 + 8 * (g.n + 1)] = off.tobytes(); bad.append(bytes(b3))
        b4 = bytearray(raw)                                                         # a path id >= R
        pid0 = 64 + 8 * (g.n + 1)
        b4[pid0:pid0 + 4] = np.int32(50_000).tobytes(); bad.append(bytes(b4))
        for i, data in enumerate(bad):
            f = str(tmp_path / f"bad{i}.bin")
            open(f, "wb").write(data)
            with pytest.raises(pk.PantherError) as e:
                pk.panther_load_index(ctx2, f)
            assert e.value.code == pk.EINVAL, i
        with pytest.raises(pk.PantherError):
            pk.panther_load_paths(ctx2, fi)                                         # an index is not paths
        # an index and paths that do not belong together are refused
        ids = np.empty((1, 10), np.int32)
        cnt = np.empty((1, 10), np.uint32)
        short = pk.panther_load_paths(ctx2, fp)
        pk.panther_free_index(ih2)
        ih_other = pk.panther_build_index(ctx2, short)
        pk.panther_sync(ctx2)
        full_other = pk.panther_sample_paths(ctx, gh, 9, 1000, 5, pk.MODE_ALIAS)
        with pytest.raises(pk.PantherError) as e:
            pk.panther_topk(ctx, ih_other, full_other, q[:1], 1, 10, ids, cnt, pk.TOPK_BATCHED | pk.IO_HOST)
        assert e.value.code == pk.EINVAL
        for h in (ih_other,):
            pk.panther_free_index(h)
        for h in (short, ph2, ph, full_other):
            pk.panther_free_paths(h)
        pk.panther_free_index(ih)
        pk.panther_free_graph(gh)
    finally:
        pk.panther_destroy(ctx2)
        pk.panther_destroy(ctx)
