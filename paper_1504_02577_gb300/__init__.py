"""Python binding of libpanther (the C ABI declared in include/panther.h).

The functions below carry the same names as the C entry points and only
marshal arguments: numpy arrays (host) or torch tensors (device) become raw
pointers, the torch current stream becomes the context stream. Every step of
the hot path runs in the library's CUDA kernels; if the shared library is
missing or cannot be loaded, importing the binding's loader raises.

Build the library first with ``python -m paper_1504_02577_gb300.build`` (or
``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpanther.so")

# status codes and flags (include/panther.h)
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EOVERFLOW, EBUSY = range(7)
MEM_HOST, MEM_DEVICE = 0, 1
MODE_PREFIX, MODE_ALIAS, MODE_BOTH, MODE_UNWEIGHTED = 1, 2, 3, 4
TOPK_BATCHED, TOPK_PLAIN = 0, 1
KNN_BF16_SCREEN, KNN_FP32 = 0, 2
IO_HOST = 0x100

_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EOVERFLOW", 6: "EBUSY"}

_vp, _i64, _u64, _u32, _i32, _int, _dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                          ctypes.c_int32, ctypes.c_int, ctypes.c_double)
_P = ctypes.POINTER

# name -> (argtypes, restype); mirrors include/panther.h
SIGNATURES = {
    "panther_create": ([_P(_vp), _int, _vp], _int),
    "panther_destroy": ([_vp], None),
    "panther_last_error": ([_vp], ctypes.c_char_p),
    "panther_sync": ([_vp], _int),
    "panther_set_scratch_budget": ([_vp, _i64], _int),
    "panther_set_index_budget": ([_vp, _i64], _int),
    "panther_launch_count": ([_vp], _i64),
    "panther_sample_size": ([_dbl, _dbl, _dbl, _int, _P(_i64)], _int),
    "panther_build_graph": ([_vp, _i64, _i64, _vp, _vp, _vp, _int, _int, _P(_vp)], _int),
    "panther_sample_paths": ([_vp, _vp, _u64, _i64, _int, _int, _P(_vp)], _int),
    "panther_paths_view": ([_vp, _P(_vp), _P(_i64), _P(_int), _P(_int)], _int),
    "panther_paths_info": ([_vp, _P(_i64), _P(_i64), _P(_int), _P(_i64)], _int),
    "panther_build_index": ([_vp, _vp, _P(_vp)], _int),
    "panther_index_view": ([_vp, _P(_vp), _P(_vp), _P(_i64), _P(_i64)], _int),
    "panther_build_index_noalloc": ([_vp, _vp, _vp, _vp, _i64, _P(_i64)], _int),
    "panther_topk": ([_vp, _vp, _vp, _vp, _i64, _int, _vp, _vp, _int], _int),
    "panther_tune_topk": ([_vp, _vp, _vp, _vp, _i64, _int, _vp, _vp, _P(_int)], _int),
    "panther_set_topk_shape": ([_vp, _int, _int, _int], _int),
    "pantherpp_vectors": ([_vp, _vp, _vp, _int, _P(_vp)], _int),
    "pantherpp_vecs_view": ([_vp, _P(_vp), _P(_i64), _P(_int)], _int),
    "pantherpp_knn": ([_vp, _vp, _vp, _i64, _int, _vp, _vp, _int], _int),
    "pantherpp_knn_cross": ([_vp, _vp, _vp, _vp, _i64, _int, _vp, _vp, _int], _int),
    "pantherpp_knn_stats": ([_vp, _P(_i64)], _int),
    "panther_topk_stats": ([_vp, _P(_i64)], _int),
    "pantherpp_debug_screen": ([_vp, _vp, _vp, _i64, _vp, _vp, _P(_i64)], _int),
    "panther_debug_topk_route": ([_vp, _i64, _int], _int),
    "panther_debug_graph_tables": ([_vp, _vp, _vp, _P(_int)], _int),
    "panther_debug_philox": ([_vp, _u32, _u32, _u64, _u32, _u32, _i64, _vp, _vp], _int),
    "panther_debug_fail_alloc": ([_vp, _i64], _int),
    "panther_sample_paths_range": ([_vp, _vp, _u64, _i64, _i64, _int, _int, _P(_vp)], _int),
    "panther_save_paths": ([_vp, ctypes.c_char_p], _int),
    "panther_load_paths": ([_vp, ctypes.c_char_p, _P(_vp)], _int),
    "panther_save_index": ([_vp, ctypes.c_char_p], _int),
    "panther_load_index": ([_vp, ctypes.c_char_p, _P(_vp)], _int),
    "panther_debug_wait_timeout": ([_vp, _i64], _int),
    "panther_free_graph": ([_vp], None),
    "panther_free_paths": ([_vp], None),
    "panther_free_index": ([_vp], None),
    "pantherpp_free_vecs": ([_vp], None),
    "panther_serve_create": ([_int, _vp, _vp, _vp, _i64, _int, _int, _P(_vp)], _int),
    "panther_serve_submit": ([_vp, _int, _vp, _i64, _int, _vp, _vp, _P(_i64)], _int),
    "panther_serve_wait": ([_vp, _i64, _dbl, _P(_dbl)], _int),
    "panther_serve_stats": ([_vp, _P(_i64)], _int),
    "panther_serve_destroy": ([_vp], None),
}

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libpanther.so and attach the signatures. Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libpanther.so not found at {path}: build it with "
                               "`python -m paper_1504_02577_gb300.build`")
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


class PantherError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


def _ptr(x) -> int | None:
    """Raw pointer of a numpy array or torch tensor (None passes NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    return int(x)


def _buf(x, itemsize: int, count: int, what: str):
    """Raw pointer of a caller buffer after checking its element size and that
    it holds at least `count` elements (numpy arrays and torch tensors; a plain
    integer is taken as a raw pointer and None as NULL, unchecked). The C side
    cannot see either property: a wrong element type would be read as garbage
    and a short buffer written past its end."""
    if x is None or isinstance(x, (int, np.integer)):
        return _ptr(x)
    if isinstance(x, np.ndarray):
        size, n = x.dtype.itemsize, x.size
    elif hasattr(x, "element_size") and hasattr(x, "numel"):
        size, n = x.element_size(), x.numel()
    else:
        return _ptr(x)
    if size != itemsize:
        raise ValueError(f"{what}: elements of {itemsize} bytes expected, got {size}")
    if n < count:
        raise ValueError(f"{what}: at least {count} elements expected, got {n}")
    return _ptr(x)


def _check(ctx: int | None, rc: int):
    if rc != OK:
        msg = load_library().panther_last_error(ctx).decode() if ctx else ""
        raise PantherError(rc, msg)


# ------------------------------------------------------- C-named wrappers ---
def panther_create(device: int = 0, stream: int | None = None) -> int:
    h = _vp()
    _check(None, load_library().panther_create(ctypes.byref(h), device, stream))
    return h.value


def panther_destroy(ctx: int) -> None:
    load_library().panther_destroy(ctx)


def panther_last_error(ctx: int) -> str:
    return (load_library().panther_last_error(ctx) or b"").decode()


def panther_sync(ctx: int) -> None:
    _check(ctx, load_library().panther_sync(ctx))


def panther_set_scratch_budget(ctx: int, nbytes: int) -> None:
    _check(ctx, load_library().panther_set_scratch_budget(ctx, nbytes))


def panther_set_index_budget(ctx: int, nbytes: int) -> None:
    """Temporary device bytes of an index build (0: free memory); above it the build runs in chunks."""
    _check(ctx, load_library().panther_set_index_budget(ctx, nbytes))


def panther_launch_count(ctx: int) -> int:
    return int(load_library().panther_launch_count(ctx))


def panther_sample_size(eps: float, delta: float, c: float, T: int) -> int:
    R = _i64()
    _check(None, load_library().panther_sample_size(eps, delta, c, T, ctypes.byref(R)))
    return R.value


def panther_build_graph(ctx: int, n: int, m: int, row_ptr, col, w, mem: int, modes: int = MODE_BOTH) -> int:
    h = _vp()
    # w may be None for MODE_UNWEIGHTED alone (every weight 1)
    _check(ctx, load_library().panther_build_graph(ctx, n, m, _buf(row_ptr, 8, n + 1, "row_ptr"),
                                                   _buf(col, 4, m, "col"), _buf(w, 4, m, "w"), mem, modes,
                                                   ctypes.byref(h)))
    return h.value


def panther_sample_paths(ctx: int, g: int, seed: int, R: int, T: int, mode: int) -> int:
    h = _vp()
    _check(ctx, load_library().panther_sample_paths(ctx, g, seed, R, T, mode, ctypes.byref(h)))
    return h.value


def panther_paths_view(p: int):
    rows, R, L, stride = _vp(), _i64(), _int(), _int()
    _check(None, load_library().panther_paths_view(p, ctypes.byref(rows), ctypes.byref(R), ctypes.byref(L),
                                                   ctypes.byref(stride)))
    return rows.value, R.value, L.value, stride.value


def panther_build_index(ctx: int, p: int) -> int:
    h = _vp()
    _check(ctx, load_library().panther_build_index(ctx, p, ctypes.byref(h)))
    return h.value


def panther_paths_info(p: int):
    """(n, R, T, r0) of a path handle."""
    n, R, T, r0 = _i64(), _i64(), _int(), _i64()
    _check(None, load_library().panther_paths_info(p, ctypes.byref(n), ctypes.byref(R), ctypes.byref(T),
                                                   ctypes.byref(r0)))
    return n.value, R.value, T.value, r0.value


def panther_build_index_noalloc(ctx: int, p: int, dev_off, dev_pid, pid_capacity: int) -> int:
    """Index into caller buffers with no device allocation; returns nnz.

    dev_pid must hold pid_capacity 32-bit elements (uint32 path ids; the library writes up to
    R*(T+1) of them and trusts pid_capacity) and dev_off n+1 int64 elements,
    n taken from the paths handle; both are checked here, before the call. A
    NULL handle (p = 0) skips the dev_off check: the library refuses it."""
    n_off = panther_paths_info(p)[0] + 1 if p else 0
    nnz = _i64()
    _check(ctx, load_library().panther_build_index_noalloc(ctx, p, _buf(dev_off, 8, n_off, "dev_off"),
                                                           _buf(dev_pid, 4, pid_capacity, "dev_pid"), pid_capacity,
                                                           ctypes.byref(nnz)))
    return nnz.value


def panther_index_view(ix: int):
    off, pid, n, nnz = _vp(), _vp(), _i64(), _i64()
    _check(None, load_library().panther_index_view(ix, ctypes.byref(off), ctypes.byref(pid), ctypes.byref(n),
                                                   ctypes.byref(nnz)))
    return off.value, pid.value, n.value, nnz.value


def panther_topk(ctx: int, ix: int, p: int, queries, q: int, k: int, out_ids, out_counts,
                 flags: int = TOPK_BATCHED) -> None:
    _check(ctx, load_library().panther_topk(ctx, ix, p, _buf(queries, 4, q, "queries"), q, k,
                                            _buf(out_ids, 4, q * k, "out_ids"),
                                            _buf(out_counts, 4, q * k, "out_counts"), flags))


def panther_tune_topk(ctx: int, ix: int, p: int, queries, q: int, k: int, out_ids, out_counts):
    chosen = (_int * 3)()
    _check(ctx, load_library().panther_tune_topk(ctx, ix, p, _buf(queries, 4, q, "queries"), q, k,
                                                 _buf(out_ids, 4, q * k, "out_ids"),
                                                 _buf(out_counts, 4, q * k, "out_counts"), chosen))
    return list(chosen)


def panther_set_topk_shape(ctx: int, threads: int, table_slots: int, ctas_per_sm: int) -> None:
    _check(ctx, load_library().panther_set_topk_shape(ctx, threads, table_slots, ctas_per_sm))


def pantherpp_vectors(ctx: int, ix: int, p: int, D: int) -> int:
    h = _vp()
    _check(ctx, load_library().pantherpp_vectors(ctx, ix, p, D, ctypes.byref(h)))
    return h.value


def pantherpp_vecs_view(v: int):
    th, n, D = _vp(), _i64(), _int()
    _check(None, load_library().pantherpp_vecs_view(v, ctypes.byref(th), ctypes.byref(n), ctypes.byref(D)))
    return th.value, n.value, D.value


def pantherpp_knn(ctx: int, v: int, queries, q: int, k: int, out_ids, out_dist2, flags: int = KNN_BF16_SCREEN):
    _check(ctx, load_library().pantherpp_knn(ctx, v, _buf(queries, 4, q, "queries"), q, k,
                                             _buf(out_ids, 4, q * k, "out_ids"),
                                             _buf(out_dist2, 8, q * k, "out_dist2"), flags))


def pantherpp_knn_cross(ctx: int, vq: int, vc: int, queries, q: int, k: int, out_ids, out_dist2,
                        flags: int = KNN_BF16_SCREEN):
    """Queries are vertices of vq's graph, answers vertices of vc's graph (none excluded)."""
    _check(ctx, load_library().pantherpp_knn_cross(ctx, vq, vc, _buf(queries, 4, q, "queries"), q, k,
                                                   _buf(out_ids, 4, q * k, "out_ids"),
                                                   _buf(out_dist2, 8, q * k, "out_dist2"), flags))


def pantherpp_knn_stats(ctx: int):
    a = (_i64 * 4)()
    _check(ctx, load_library().pantherpp_knn_stats(ctx, a))
    return list(a)


def pantherpp_debug_screen(ctx: int, v: int, queries=None, q: int = 0, out_y=None, out_cid=None) -> int:
    """BF16 screening values y_hat[q][npad] and candidate ids[npad]; returns npad.
    With no outputs only npad is returned (to size them)."""
    npad = _i64()
    if out_y is None and out_cid is None:
        _check(ctx, load_library().pantherpp_debug_screen(ctx, v, None, 0, None, None, ctypes.byref(npad)))
        return npad.value
    _check(ctx, load_library().pantherpp_debug_screen(ctx, v, 0, 0, None, None, ctypes.byref(npad)))
    n = npad.value
    _check(ctx, load_library().pantherpp_debug_screen(ctx, v, _buf(queries, 4, q, "queries"), q,
                                                      _buf(out_y, 4, q * n, "out_y"), _buf(out_cid, 4, n, "out_cid"),
                                                      ctypes.byref(npad)))
    return npad.value


def panther_topk_stats(ctx: int):
    """Tier sizes of the last top-k call: queries, lane, group, warp, CTA, hub,
    hub via buckets, hub via tables, bucket overflows, second passes."""
    a = (_i64 * 10)()
    _check(ctx, load_library().panther_topk_stats(ctx, a))
    return list(a)


def panther_debug_topk_route(ctx: int, hub_min_cap: int, route: int) -> None:
    """Test-only hub routing: hub_min_cap > 0 lowers the hub-tier bound; route
    1 = every hub query through buckets, 2 = through device tables."""
    _check(ctx, load_library().panther_debug_topk_route(ctx, hub_min_cap, route))


def panther_debug_graph_tables(g: int, dev_alias16, dev_prefix):
    wide = _int()
    _check(None, load_library().panther_debug_graph_tables(g, _ptr(dev_alias16), _ptr(dev_prefix),
                                                           ctypes.byref(wide)))
    return wide.value


def panther_debug_philox(ctx: int, k0: int, k1: int, r0: int, c2: int, c3: int, count: int, dev_out, dev_ref):
    _check(ctx, load_library().panther_debug_philox(ctx, k0, k1, r0, c2, c3, count, _ptr(dev_out), _ptr(dev_ref)))


def panther_sample_paths_range(ctx: int, g: int, seed: int, r0: int, R: int, T: int, mode: int) -> int:
    """Paths r0 .. r0+R-1 of the sequence of `seed` (row i = path r0 + i)."""
    out = _vp()
    _check(ctx, load_library().panther_sample_paths_range(ctx, g, seed, r0, R, T, mode, ctypes.byref(out)))
    return out.value


def panther_save_paths(p: int, path: str) -> None:
    _check(None, load_library().panther_save_paths(p, os.fsencode(path)))


def panther_load_paths(ctx: int, path: str) -> int:
    out = _vp()
    _check(ctx, load_library().panther_load_paths(ctx, os.fsencode(path), ctypes.byref(out)))
    return out.value


def panther_save_index(ix: int, path: str) -> None:
    _check(None, load_library().panther_save_index(ix, os.fsencode(path)))


def panther_load_index(ctx: int, path: str) -> int:
    out = _vp()
    _check(ctx, load_library().panther_load_index(ctx, os.fsencode(path), ctypes.byref(out)))
    return out.value


def panther_debug_fail_alloc(ctx: int, nth: int) -> None:
    """Test-only: the nth device allocation of ctx from now on fails once (ENOMEM); nth < 0 cancels."""
    _check(ctx, load_library().panther_debug_fail_alloc(ctx, nth))


def panther_debug_wait_timeout(ctx: int, limit_cycles: int) -> None:
    """Test-only: a bounded device wait on a flag nothing sets; raises PantherError(ETIMEOUT)."""
    _check(ctx, load_library().panther_debug_wait_timeout(ctx, limit_cycles))


def panther_free_graph(g: int) -> None:
    load_library().panther_free_graph(g)


def panther_free_paths(p: int) -> None:
    load_library().panther_free_paths(p)


def panther_free_index(ix: int) -> None:
    load_library().panther_free_index(ix)


def pantherpp_free_vecs(v: int) -> None:
    load_library().pantherpp_free_vecs(v)


def panther_serve_create(device: int, ix: int, p: int, v: int | None, mem_budget: int, max_inflight: int,
                         streams: int) -> int:
    h = _vp()
    _check(None, load_library().panther_serve_create(device, ix, p, v, mem_budget, max_inflight, streams,
                                                     ctypes.byref(h)))
    return h.value


def panther_serve_submit(s: int, kind: int, queries: np.ndarray, k: int, out_ids: np.ndarray,
                         out_vals: np.ndarray) -> int:
    t = _i64()
    q = int(queries.shape[0])
    _check(None, load_library().panther_serve_submit(s, kind, _buf(queries, 4, q, "queries"), q, k,
                                                     _buf(out_ids, 4, q * k, "out_ids"),
                                                     _buf(out_vals, 4 if kind == 0 else 8, q * k, "out_vals"),
                                                     ctypes.byref(t)))
    return t.value


def panther_serve_wait(s: int, ticket: int, timeout_s: float = 60.0) -> float:
    lat = _dbl()
    _check(None, load_library().panther_serve_wait(s, ticket, timeout_s, ctypes.byref(lat)))
    return lat.value


def panther_serve_stats(s: int):
    a = (_i64 * 6)()
    _check(None, load_library().panther_serve_stats(s, a))
    return list(a)


def panther_serve_destroy(s: int) -> None:
    load_library().panther_serve_destroy(s)


# --------------------------------------------------- torch-facing helpers ---
@dataclass
class Handles:
    ctx: int
    graph: int | None = None
    paths: int | None = None
    index: int | None = None
    vecs: int | None = None


class Panther:
    """Owns one context and the handles of one graph; tensors in, tensors out.

    A thin convenience over the C-named wrappers: device memory and the stream
    come from torch, every computation runs in libpanther.
    """

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.torch = torch
        self.device = device
        # the library enqueues on this (non-default) stream; results are handed
        # back to the caller's current stream by _enter/_leave
        self.stream = stream if stream is not None else torch.cuda.Stream(device)
        self.h = Handles(panther_create(device, self.stream.cuda_stream))

    def _enter(self, *inputs):
        """Order the library stream after the caller's stream (inputs ready)."""
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def _leave(self, *outputs):
        """Order the caller's stream after the library stream; keep outputs alive."""
        cur = self.torch.cuda.current_stream(self.device)
        cur.wait_stream(self.stream)
        for t in outputs:
            if t is not None and hasattr(t, "record_stream"):
                t.record_stream(cur)

    def close(self):
        h = self.h
        if h.vecs:
            pantherpp_free_vecs(h.vecs)
        if h.index:
            panther_free_index(h.index)
        if h.paths:
            panther_free_paths(h.paths)
        if h.graph:
            panther_free_graph(h.graph)
        panther_destroy(h.ctx)
        self.h = Handles(0)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def build_graph(self, row_ptr, col, w=None, modes: int = MODE_BOTH):
        n = int(row_ptr.shape[0]) - 1
        m = int(col.shape[0])
        mem = MEM_HOST if isinstance(row_ptr, np.ndarray) else MEM_DEVICE
        if self.h.graph:
            panther_free_graph(self.h.graph)
            self.h.graph = None          # not left dangling if the build below fails
        self._enter()
        self.h.graph = panther_build_graph(self.h.ctx, n, m, row_ptr, col, w, mem, modes)
        self.n = n
        return self.h.graph

    def sample_paths(self, seed: int, R: int, T: int, mode: int = MODE_ALIAS):
        if self.h.paths:
            panther_free_paths(self.h.paths)
            self.h.paths = None
        self.h.paths = panther_sample_paths(self.h.ctx, self.h.graph, seed, R, T, mode)
        return self.h.paths

    def paths_tensor(self):
        """int32[R][T+1] copy of the sampled rows (device)."""
        torch = self.torch
        rows, R, L, stride = panther_paths_view(self.h.paths)
        with torch.cuda.stream(self.stream):
            t = _device_view(torch, rows, (R, stride), torch.int32, self.device)[:, :L].contiguous()
        self._leave(t)
        return t

    def build_index(self):
        if self.h.index:
            panther_free_index(self.h.index)
            self.h.index = None
        self.h.index = panther_build_index(self.h.ctx, self.h.paths)
        return self.h.index

    def index_tensors(self):
        """(off int64[n+1], pid[nnz]) copies; pid holds uint32 path ids in
        int32 storage (ids from 2^31 up read negative: widen with
        ``pid.to(torch.int64) & 0xFFFFFFFF``)."""
        torch = self.torch
        off, pid, n, nnz = panther_index_view(self.h.index)
        with torch.cuda.stream(self.stream):
            o = _device_view(torch, off, (n + 1,), torch.int64, self.device).clone()
            p = _device_view(torch, pid, (max(nnz, 1),), torch.int32, self.device)[:nnz].clone()
        self._leave(o, p)
        return o, p

    def topk(self, queries, k: int, plain: bool = False):
        torch = self.torch
        q = int(queries.shape[0])
        self._enter()
        with torch.cuda.stream(self.stream):
            ids = torch.empty((q, k), dtype=torch.int32, device=queries.device)
            cnt = torch.empty((q, k), dtype=torch.int32, device=queries.device)
        queries.record_stream(self.stream)
        panther_topk(self.h.ctx, self.h.index, self.h.paths, queries, q, k, ids, cnt,
                     TOPK_PLAIN if plain else TOPK_BATCHED)
        self._leave(ids, cnt)
        return ids, cnt

    def tune_topk(self, queries, k: int):
        """Autotune the batched top-k launch shape on this batch; returns the chosen shape."""
        torch = self.torch
        q = int(queries.shape[0])
        self._enter()
        with torch.cuda.stream(self.stream):
            ids = torch.empty((q, k), dtype=torch.int32, device=queries.device)
            cnt = torch.empty((q, k), dtype=torch.int32, device=queries.device)
        shape = panther_tune_topk(self.h.ctx, self.h.index, self.h.paths, queries, q, k, ids, cnt)
        self._leave(ids, cnt)
        return shape

    def vectors(self, D: int = 50):
        if self.h.vecs:
            pantherpp_free_vecs(self.h.vecs)
            self.h.vecs = None
        self.h.vecs = pantherpp_vectors(self.h.ctx, self.h.index, self.h.paths, D)
        return self.h.vecs

    def theta_tensor(self):
        torch = self.torch
        th, n, D = pantherpp_vecs_view(self.h.vecs)
        with torch.cuda.stream(self.stream):
            t = _device_view(torch, th, (n, D), torch.int32, self.device).clone()
        self._leave(t)
        return t

    def knn(self, queries, k: int, fp32: bool = False):
        torch = self.torch
        q = int(queries.shape[0])
        self._enter()
        with torch.cuda.stream(self.stream):
            ids = torch.empty((q, k), dtype=torch.int32, device=queries.device)
            d2 = torch.empty((q, k), dtype=torch.int64, device=queries.device)
        queries.record_stream(self.stream)
        pantherpp_knn(self.h.ctx, self.h.vecs, queries, q, k, ids, d2, KNN_FP32 if fp32 else KNN_BF16_SCREEN)
        self._leave(ids, d2)
        return ids, d2

    def sync(self):
        panther_sync(self.h.ctx)

    def launches(self) -> int:
        return panther_launch_count(self.h.ctx)


def _device_view(torch, ptr: int, shape, dtype, device: int):
    """A torch tensor aliasing library-owned device memory (valid while the handle lives)."""
    numel = 1
    for s in shape:
        numel *= s
    if numel == 0:
        return torch.empty(shape, dtype=dtype, device=f"cuda:{device}")
    esz = torch.empty((), dtype=dtype).element_size()

    class _CAI:
        __cuda_array_interface__ = {
            "shape": tuple(shape),
            "typestr": {1: "|u1", 2: "<i2", 4: "<i4", 8: "<i8"}[esz] if dtype != torch.float32 else "<f4",
            "data": (ptr, False),
            "version": 3,
            "strides": None,
        }

    t = torch.as_tensor(_CAI(), device=f"cuda:{device}")
    return t.view(dtype) if t.dtype != dtype else t
