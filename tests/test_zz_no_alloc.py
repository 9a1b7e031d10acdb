"""The allocation-free index build (panther_build_index_noalloc).

Some callers cannot call cudaMalloc: an application that owns a fixed share
of the GPU and tracks every byte, or a loop where an allocation could stall
the device. For them the library offers an index build whose temporary
buffers live in one static device array; the caller passes the outputs. This
file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_index_equals_allocating_index_twice():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1504_02577_gb300 as pk
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = synth.workload_graph("small")
    ctx = pk.panther_create(0)
    try:
        gh = pk.panther_build_graph(ctx, g.n, g.m, g.row_ptr, g.col, g.w, pk.MEM_HOST, pk.MODE_ALIAS)
        for seed, R in ((1, 200_000), (7, 123_457)):        # two calls in a row, different sizes
            ph = pk.panther_sample_paths(ctx, gh, seed, R, 5, pk.MODE_ALIAS)
            ih = pk.panther_build_index(ctx, ph)
            off_ptr, pid_ptr, n, nnz = pk.panther_index_view(ih)
            cap = R * 6
            off = torch.full((g.n + 1,), -7, dtype=torch.int64, device="cuda:0")
            pid = torch.full((cap,), -7, dtype=torch.int32, device="cuda:0")
            torch.cuda.synchronize()
            got = pk.panther_build_index_noalloc(ctx, ph, off, pid, cap)
            pk.panther_sync(ctx)
            ref_off = torch.empty(g.n + 1, dtype=torch.int64, device="cuda:0")
            ref_pid = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda:0")
            # copy the allocating index's arrays through torch views (the
            # library stream was synchronised above)
            ref_off.copy_(pk._device_view(torch, off_ptr, (g.n + 1,), torch.int64, 0))
            ref_pid[:nnz].copy_(pk._device_view(torch, pid_ptr, (nnz,), torch.int32, 0))
            torch.cuda.synchronize()
            assert got == nnz
            assert torch.equal(off, ref_off)
            assert torch.equal(pid[:nnz], ref_pid[:nnz])
            pk.panther_free_index(ih)
            pk.panther_free_paths(ph)
        # sizes beyond the static scratch are refused before any launch
        big = pk.panther_sample_paths(ctx, gh, 3, 800_000, 5, pk.MODE_ALIAS)
        big_pid = torch.empty(800_000 * 6, dtype=torch.int32, device="cuda:0")
        with pytest.raises(pk.PantherError) as ei:
            pk.panther_build_index_noalloc(ctx, big, off, big_pid, 800_000 * 6)
        assert ei.value.code == pk.EOVERFLOW
        # the binding refuses caller buffers shorter than the call writes
        with pytest.raises(ValueError, match="dev_off"):
            pk.panther_build_index_noalloc(ctx, big, off[: g.n], big_pid, 800_000 * 6)
        with pytest.raises(ValueError, match="dev_pid"):
            pk.panther_build_index_noalloc(ctx, big, off, big_pid[:100], 800_000 * 6)
        pk.panther_free_paths(big)
        pk.panther_free_graph(gh)
    finally:
        pk.panther_destroy(ctx)
