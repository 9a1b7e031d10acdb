"""CPU oracle for the Panther / Panther++ hot path (TEST INFRASTRUCTURE ONLY).

Plain, slow, single-threaded C (``panther_oracle.c``) behind ctypes. Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package; the product path never does, and shares no code with it.
Functions that take ``threads > 1`` run the all-core driver of the same file:
it cuts one independent outer loop (rows, path ids, index vertices, queries)
into ranges, one POSIX thread each, with identical results.

Every function states the passage of the paper it follows (arXiv 1504.02577):
Algorithm 3 (path generation), Eq. (3) (transition probabilities), the
inverted index of Sec. 3.1, Algorithm 1 with Eq. (4) (counting + top-k),
Sec. 3.3 / Algorithm 2 (Panther++ vectors and nearest neighbours) and the
sample-size bound of Sec. 3.2 (Theorem 1 with Lemma 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "panther_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

PREFIX, ALIAS = 0, 1


def build() -> str:
    """Compile the oracle with plain gcc (no fast-math, no vectorisation tricks)."""
    if os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-pthread", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i64, u64, u32, i32, dbl, ci = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                               ctypes.c_uint32, ctypes.c_int32, ctypes.c_double,
                                               ctypes.c_int)
            sig = {
                "po_philox4x32_10": ([vp, vp, vp], None),
                "po_draw": ([u64, u32, u64, u32, u32, vp], None),
                "po_lemire": ([u64, u64, vp], ci),
                "po_sample_size": ([dbl, dbl, dbl, ci], i64),
                "po_select_prefix": ([vp, i64, u64], i64),
                "po_alias_row": ([vp, i64, vp, vp], None),
                "po_select_alias": ([vp, vp, i64, u64, u64], i64),
                "po_alias_tables": ([i64, vp, vp, vp, vp], None),
                "po_sample_paths": ([i64, vp, vp, vp, vp, vp, u64, i64, i64, ci, ci, vp], ci),
                "po_build_index": ([i64, i64, ci, vp, vp, vp], i64),
                "po_topk": ([i64, ci, vp, vp, vp, i32, ci, vp, vp, vp], i64),
                "po_theta": ([i64, ci, vp, vp, vp, i32, ci, vp, vp], None),
                "po_dist2": ([vp, vp, ci, vp], ci),
                "po_knn": ([i64, ci, vp, i32, ci, vp, vp], ci),
                "po_row_sums": ([i64, i64, vp, vp, vp], None),
                "po_sample_paths_rs": ([i64, vp, vp, vp, vp, vp, vp, u64, i64, i64, ci, ci, vp], ci),
                "po_index_range": ([i64, ci, vp, i64, i64, vp, vp], None),
                "po_mt_alias_tables": ([i64, vp, vp, vp, vp, ci], ci),
                "po_mt_sample_paths": ([i64, vp, vp, vp, vp, vp, u64, i64, i64, ci, ci, vp, ci], ci),
                "po_mt_build_index": ([i64, i64, ci, vp, vp, vp, ci], i64),
                "po_mt_topk_many": ([i64, ci, vp, vp, vp, vp, i64, ci, vp, vp, ci], ci),
                "po_mt_theta_many": ([i64, ci, vp, vp, vp, vp, i64, ci, vp, ci], ci),
                "po_mt_knn_many": ([i64, ci, vp, vp, i64, ci, vp, vp, ci], ci),
                "po_mt_paths_at": ([i64, vp, vp, vp, vp, vp, u64, vp, i64, ci, ci, vp, ci], ci),
                "po_mt_stream_counts": ([i64, vp, vp, vp, vp, vp, u64, i64, i64, ci, ci, vp, i64, vp, vp, ci], ci),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _p(a: np.ndarray | None) -> int | None:
    return None if a is None else a.ctypes.data


# ---------------------------------------------------------------- RNG ---
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    _load().po_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def draw(seed: int, stream: int, r: int, t: int, attempt: int = 0) -> np.ndarray:
    out = np.empty(4, dtype=np.uint32)
    _load().po_draw(seed, stream, r, t, attempt, _p(out))
    return out


def lemire(U: int, S: int):
    out = np.zeros(1, dtype=np.uint64)
    ok = _load().po_lemire(U, S, _p(out))
    return bool(ok), int(out[0])


def sample_size(eps: float, delta: float, c: float, T: int) -> int:
    """Sec. 3.2: R = ceil(c/eps^2 (log2 C(T,2) + 1 + ln 1/delta)); -1 if undefined."""
    return int(_load().po_sample_size(eps, delta, c, T))


# ---------------------------------------------------------- selection ---
def select_prefix(w: np.ndarray, x: int) -> int:
    w = np.ascontiguousarray(w, dtype=np.uint32)
    return int(_load().po_select_prefix(_p(w), w.shape[0], x))


def alias_row(w: np.ndarray):
    w = np.ascontiguousarray(w, dtype=np.uint32)
    thr = np.empty(w.shape[0], dtype=np.uint64)
    al = np.empty(w.shape[0], dtype=np.int32)
    _load().po_alias_row(_p(w), w.shape[0], _p(thr), _p(al))
    return thr, al


def select_alias(thr: np.ndarray, al: np.ndarray, c: int, u: int) -> int:
    return int(_load().po_select_alias(_p(thr), _p(al), thr.shape[0], c, u))


def alias_tables(g, threads: int = 1):
    """Eq. (3) alias tables of every row (threads > 1: the all-core driver, same tables)."""
    thr = np.zeros(max(g.m, 1), dtype=np.uint64)
    al = np.zeros(max(g.m, 1), dtype=np.int32)
    if threads > 1:
        if _load().po_mt_alias_tables(g.n, _p(g.row_ptr), _p(g.w), _p(thr), _p(al), threads) != 0:
            raise MemoryError("po_mt_alias_tables failed")
    else:
        _load().po_alias_tables(g.n, _p(g.row_ptr), _p(g.w), _p(thr), _p(al))
    return thr, al


# -------------------------------------------------------------- paths ---
def sample_paths(g, seed: int, R: int, T: int, mode: int = PREFIX, r0: int = 0, tables=None,
                 threads: int = 1) -> np.ndarray:
    """Algorithm 3: paths r0 .. r0+R-1 as int32[R][T+1].

    threads > 1 runs the all-core driver: row sums once, then contiguous path
    ranges per thread (identical paths)."""
    lib = _load()
    thr = al = None
    if mode == ALIAS:
        thr, al = tables if tables is not None else alias_tables(g, threads)
    out = np.empty((R, T + 1), dtype=np.int32)
    col = g.col if g.m else np.zeros(1, np.int32)
    w = g.w if g.m else np.zeros(1, np.uint32)
    if threads > 1:
        rc = lib.po_mt_sample_paths(g.n, _p(g.row_ptr), _p(col), _p(w), _p(thr), _p(al),
                                    seed, r0, r0 + R, T, mode, _p(out), threads)
    else:
        rc = lib.po_sample_paths(g.n, _p(g.row_ptr), _p(col), _p(w), _p(thr), _p(al),
                                 seed, r0, r0 + R, T, mode, _p(out))
    if rc != 0:
        raise ValueError("po_sample_paths: bad arguments")
    return out


def paths_at(g, seed: int, ids, T: int, mode: int = PREFIX, tables=None, threads: int = 1) -> np.ndarray:
    """Algorithm 3 for the given path ids only: row i of the int32[m][T+1]
    result is path ids[i], drawn as sample_paths draws it."""
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    thr = al = None
    if mode == ALIAS:
        thr, al = tables if tables is not None else alias_tables(g, threads)
    out = np.empty((ids.shape[0], T + 1), dtype=np.int32)
    col = g.col if g.m else np.zeros(1, np.int32)
    w = g.w if g.m else np.zeros(1, np.uint32)
    if _load().po_mt_paths_at(g.n, _p(g.row_ptr), _p(col), _p(w), _p(thr), _p(al), seed, _p(ids), ids.shape[0],
                              T, mode, _p(out), max(1, threads)) != 0:
        raise ValueError("po_mt_paths_at: bad arguments")
    return out


def stream_counts(g, seed: int, r0: int, r1: int, T: int, queries, mode: int = PREFIX, tables=None,
                  threads: int = 1):
    """Eq. (4) and |P_v| from their definitions, with no index: paths
    r0..r1-1 are drawn one by one and dropped. Returns (cnt uint64[nq][n],
    npaths int64[n]): cnt[i][u] = number of those paths holding both
    queries[i] and u (u != queries[i]), npaths[v] = number holding v. For path
    sets too large to keep (memory: threads x (nq + 1) x n x 8 bytes)."""
    q = np.ascontiguousarray(queries, dtype=np.int32)
    thr = al = None
    if mode == ALIAS:
        thr, al = tables if tables is not None else alias_tables(g, threads)
    cnt = np.empty((q.shape[0], g.n), dtype=np.uint64)
    npaths = np.empty(g.n, dtype=np.int64)
    col = g.col if g.m else np.zeros(1, np.int32)
    w = g.w if g.m else np.zeros(1, np.uint32)
    if _load().po_mt_stream_counts(g.n, _p(g.row_ptr), _p(col), _p(w), _p(thr), _p(al), seed, r0, r1, T, mode,
                                   _p(q), q.shape[0], _p(cnt), _p(npaths), max(1, threads)) != 0:
        raise ValueError("po_mt_stream_counts: bad arguments (queries must be distinct vertices)")
    return cnt, npaths


def topk_from_counts(cnt_row: np.ndarray, v: int, k: int):
    """Top-k of one dense count row (Algorithm 1's selection): the u != v with
    cnt > 0 by (count desc, id asc), padded with (-1, 0)."""
    c = np.asarray(cnt_row, dtype=np.uint64).copy()
    c[v] = 0
    u = np.nonzero(c)[0]
    order = u[np.lexsort((u, -c[u].astype(np.int64)))][:k]
    ids = np.full(k, -1, dtype=np.int32)
    cnt = np.zeros(k, dtype=np.uint64)
    ids[:order.size] = order
    cnt[:order.size] = c[order]
    return ids, cnt


def build_index(n: int, paths: np.ndarray, threads: int = 1):
    """Sec. 3.1 inverted index: (off int64[n+1], pid int32[nnz]).

    threads > 1: one vertex range per thread (identical index)."""
    lib = _load()
    paths = np.ascontiguousarray(paths, dtype=np.int32)
    R, L = paths.shape
    off = np.empty(n + 1, dtype=np.int64)
    if threads > 1:
        nnz = lib.po_mt_build_index(n, R, L, _p(paths), _p(off), None, threads)
        pid = np.empty(max(nnz, 1), dtype=np.int32)
        lib.po_mt_build_index(n, R, L, _p(paths), _p(off), _p(pid), threads)
        return off, pid[:nnz]
    nnz = lib.po_build_index(n, R, L, _p(paths), _p(off), None)
    pid = np.empty(max(nnz, 1), dtype=np.int32)
    lib.po_build_index(n, R, L, _p(paths), _p(off), _p(pid))
    return off, pid[:nnz]


class Oracle:
    """Counting / top-k / theta over one (paths, index) pair, with reusable work space."""

    def __init__(self, n: int, paths: np.ndarray, off: np.ndarray | None = None, pid: np.ndarray | None = None):
        self.n = n
        self.paths = np.ascontiguousarray(paths, dtype=np.int32)
        self.L = self.paths.shape[1]
        if off is None:
            off, pid = build_index(n, self.paths)
        self.off, self.pid = off, (pid if pid.shape[0] else np.zeros(1, np.int32))
        self._work = np.zeros(n, dtype=np.uint32)
        self._lib = _load()

    def topk(self, v: int, k: int):
        """Algorithm 1 + Eq. (4): top-k (ids, counts) by (count desc, id asc)."""
        ids = np.empty(k, dtype=np.int32)
        cnt = np.empty(k, dtype=np.uint32)
        self._lib.po_topk(self.n, self.L, _p(self.paths), _p(self.off), _p(self.pid), int(v), k,
                          _p(self._work), _p(ids), _p(cnt))
        return ids, cnt

    def topk_many(self, queries, k: int, threads: int = 1):
        """topk for every query (threads > 1: query ranges per thread, identical rows)."""
        q = np.ascontiguousarray(queries, dtype=np.int32)
        ids = np.empty((q.shape[0], k), dtype=np.int32)
        cnt = np.empty((q.shape[0], k), dtype=np.uint32)
        if threads > 1:
            if self._lib.po_mt_topk_many(self.n, self.L, _p(self.paths), _p(self.off), _p(self.pid), _p(q),
                                         q.shape[0], k, _p(ids), _p(cnt), threads) != 0:
                raise MemoryError("po_mt_topk_many failed")
            return ids, cnt
        for i, v in enumerate(q):
            ids[i], cnt[i] = self.topk(int(v), k)
        return ids, cnt

    def theta(self, v: int, D: int) -> np.ndarray:
        """Sec. 3.3: the D largest counts of v (excluding v), descending, zero-padded."""
        out = np.empty(D, dtype=np.uint32)
        self._lib.po_theta(self.n, self.L, _p(self.paths), _p(self.off), _p(self.pid), int(v), D,
                           _p(self._work), _p(out))
        return out

    def theta_all(self, D: int, threads: int = 1) -> np.ndarray:
        out = np.empty((self.n, D), dtype=np.uint32)
        if threads > 1:
            if self._lib.po_mt_theta_many(self.n, self.L, _p(self.paths), _p(self.off), _p(self.pid), None,
                                          self.n, D, _p(out), threads) != 0:
                raise MemoryError("po_mt_theta_many failed")
            return out
        for v in range(self.n):
            out[v] = self.theta(v, D)
        return out


def dist2(a: np.ndarray, b: np.ndarray) -> int:
    a = np.ascontiguousarray(a, dtype=np.uint32)
    b = np.ascontiguousarray(b, dtype=np.uint32)
    out = np.zeros(1, dtype=np.uint64)
    if _load().po_dist2(_p(a), _p(b), a.shape[0], _p(out)) != 0:
        raise OverflowError("squared distance exceeds 64 bits")
    return int(out[0])


def knn_cross(theta_q: np.ndarray, theta_c: np.ndarray, v: int, k: int):
    """Panther++ across two graphs (Sec. 3.3's S_RP++ between theta(v) of one
    network and every theta(u) of another): the k vertices u of the second by
    (squared L2 asc, id asc); no vertex is excluded. Plain definition in
    integers (numpy), padded with (-1, UINT64_MAX)."""
    a = np.asarray(theta_q, dtype=np.int64)[v]
    b = np.asarray(theta_c, dtype=np.int64)
    d2 = ((b - a) ** 2).astype(np.uint64).sum(axis=1, dtype=np.uint64)
    order = np.lexsort((np.arange(b.shape[0]), d2))[:k]
    ids = np.full(k, -1, dtype=np.int32)
    dist = np.full(k, np.iinfo(np.uint64).max, dtype=np.uint64)
    ids[:order.size] = order
    dist[:order.size] = d2[order]
    return ids, dist


def knn_many(theta: np.ndarray, queries, k: int, threads: int = 1):
    """knn for every query: (ids int32[q][k], d2 uint64[q][k]); threads > 1 splits the queries."""
    theta = np.ascontiguousarray(theta, dtype=np.uint32)
    q = np.ascontiguousarray(queries, dtype=np.int32)
    n, D = theta.shape
    ids = np.empty((q.shape[0], k), dtype=np.int32)
    d2 = np.empty((q.shape[0], k), dtype=np.uint64)
    if _load().po_mt_knn_many(n, D, _p(theta), _p(q), q.shape[0], k, _p(ids), _p(d2), max(1, threads)) != 0:
        raise OverflowError("squared distance exceeds 64 bits")
    return ids, d2


def knn(theta: np.ndarray, v: int, k: int):
    """Sec. 3.3 / Algorithm 2: k nearest u != v by (squared L2 asc, id asc)."""
    theta = np.ascontiguousarray(theta, dtype=np.uint32)
    n, D = theta.shape
    ids = np.empty(k, dtype=np.int32)
    d2 = np.empty(k, dtype=np.uint64)
    if _load().po_knn(n, D, _p(theta), int(v), k, _p(ids), _p(d2)) != 0:
        raise OverflowError("squared distance exceeds 64 bits")
    return ids, d2
