"""Seeded synthetic inputs: Chung-Lu power-law graphs and query mixes.

This module writes inputs only. It carries none of the method's arithmetic and
is shared, read-only, by the CUDA path, the CPU oracle, the tests and the
benchmark. The recipe (ball-dropping Chung-Lu, first E distinct edges in draw
order, endpoint-keyed weights) is documented in ``chunglu.c``.

The named workloads mirror the shapes of the paper's social networks (Tencent
sub-networks: power-law degree, mean degree between about 1.5 and 38, up to
51.6M vertices; Section 5.1, Table 2), which are not available here.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chunglu.c")
_LIB = os.path.join(_HERE, "_libsynth.so")
_lock = threading.Lock()
_lib = None


def build() -> str:
    """Compile the generator (gcc, OpenMP, no FP contraction)."""
    if os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, u64, u32, dbl, vp = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                      ctypes.c_double, ctypes.c_void_p)
            lib.synth_chung_lu.argtypes = [i64, i64, dbl, u64, ctypes.c_int, u32, u32, vp, vp, vp, vp]
            lib.synth_chung_lu.restype = ctypes.c_int
            lib.synth_query_mix.argtypes = [i64, i64, vp, i64, i64, u64, vp]
            lib.synth_query_mix.restype = None
            lib.synth_uniform_ints.argtypes = [i64, i64, u64, u64, vp]
            lib.synth_uniform_ints.restype = None
            lib.synth_det_pow.argtypes = [dbl, dbl]
            lib.synth_det_pow.restype = dbl
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Graph:
    """Symmetric CSR: row_ptr int64[n+1], col int32[m] (ascending per row), w uint32[m]."""
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    draws: int
    max_degree: int
    isolated: int

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def chung_lu(n: int, mean_deg: float, gamma: float, weights=("uniform", 1, 1), seed: int = 1) -> Graph:
    """Chung-Lu graph with exactly E = round(n*mean_deg/2) distinct undirected edges.

    ``weights`` is ("uniform", lo, hi) or ("loguniform", 1, hi).
    """
    lib = _load()
    E = int(round(n * mean_deg / 2))
    kind = {"uniform": 0, "loguniform": 1}[weights[0]]
    lo, hi = int(weights[1]), int(weights[2])
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(2 * E, dtype=np.int32)
    w = np.empty(2 * E, dtype=np.uint32)
    stats = np.zeros(4, dtype=np.int64)
    rc = lib.synth_chung_lu(n, E, float(gamma), seed, kind, lo, hi,
                            _ptr(row_ptr), _ptr(col), _ptr(w), _ptr(stats))
    if rc != 0:
        raise ValueError(f"synth_chung_lu failed with code {rc}")
    return Graph(n, row_ptr, col, w, int(stats[0]), int(stats[1]), int(stats[2]))


def hub_set(g: Graph, frac: float = 0.01) -> np.ndarray:
    """The first ceil(frac*n) vertices ordered by (degree desc, id asc)."""
    deg = g.degrees()
    order = np.lexsort((np.arange(g.n), -deg))
    return np.ascontiguousarray(order[: int(math.ceil(frac * g.n))].astype(np.int32))


def query_mix(g: Graph, n_uniform: int, n_hub: int, seed: int = 1, frac: float = 0.01) -> np.ndarray:
    """n_uniform uniform queries plus n_hub queries from the top-degree set, shuffled."""
    lib = _load()
    hubs = hub_set(g, frac)
    out = np.empty(n_uniform + n_hub, dtype=np.int32)
    lib.synth_query_mix(g.n, n_uniform, _ptr(hubs), hubs.shape[0], n_hub, seed, _ptr(out))
    return out


def uniform_ints(count: int, n: int, seed: int = 1, stream: int = 0x61) -> np.ndarray:
    lib = _load()
    out = np.empty(count, dtype=np.int32)
    lib.synth_uniform_ints(count, n, seed, stream, _ptr(out))
    return out


def det_pow(b: float, e: float) -> float:
    return _load().synth_det_pow(b, e)


def graph_from_edges(n: int, edges, weights) -> Graph:
    """Symmetric CSR from an explicit undirected edge list (tiny hand-made test graphs)."""
    adj = [dict() for _ in range(n)]
    for (a, b), wt in zip(edges, weights):
        if a == b:
            raise ValueError("self-loop")
        adj[a][b] = wt
        adj[b][a] = wt
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    cols, ws = [], []
    for v in range(n):
        for u in sorted(adj[v]):
            cols.append(u)
            ws.append(adj[v][u])
        row_ptr[v + 1] = len(cols)
    col = np.array(cols, dtype=np.int32)
    w = np.array(ws, dtype=np.uint32)
    deg = np.diff(row_ptr)
    return Graph(n, row_ptr, col, w, 0, int(deg.max()) if n else 0, int((deg == 0).sum()))


# Named workloads (sizes of the four benchmark configurations).
WORKLOADS = {
    "small": dict(n=2_000, mean_deg=10, gamma=2.5, weights=("uniform", 1, 16), T=5, R=200_000, k=10),
    "batched": dict(n=1_000_000, mean_deg=20, gamma=2.3, weights=("loguniform", 1, 1024), T=5,
                    eps=0.01, delta=0.1, c=0.5, q_uniform=8192, q_hub=8192, k=5),
    "scale": dict(n=50_000_000, mean_deg=16, gamma=2.1, weights=("uniform", 1, 255), T=5,
                  R=100_000_000, k=10),
    "knn": dict(n=10_000_000, mean_deg=20, gamma=2.3, weights=("loguniform", 1, 1024), T=5,
                R=50_000_000, D=50, k=10),
}


def workload_graph(name: str, seed: int = 1, n: int | None = None) -> Graph:
    p = WORKLOADS[name]
    return chung_lu(n or p["n"], p["mean_deg"], p["gamma"], p["weights"], seed)
