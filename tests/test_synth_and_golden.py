"""The seeded input generator and the stored oracle fixtures (no GPU)."""
import os

import numpy as np

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_chung_lu_shape_and_determinism():
    g = synth.chung_lu(3000, 8, 2.4, ("uniform", 1, 9), seed=4)
    h = synth.chung_lu(3000, 8, 2.4, ("uniform", 1, 9), seed=4)
    assert g.m == 3000 * 8 and (g.col == h.col).all() and (g.w == h.w).all()
    assert g.row_ptr[0] == 0 and g.row_ptr[-1] == g.m
    deg = g.degrees()
    assert deg.max() == g.max_degree and (deg == 0).sum() == g.isolated
    # symmetric, sorted columns, no self-loop, weights in range and symmetric
    edges = {}
    for v in range(g.n):
        c = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
        assert (np.diff(c) > 0).all() and (c != v).all()
        for u, wt in zip(c.tolist(), g.w[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()):
            edges[(v, u)] = wt
    for (v, u), wt in edges.items():
        assert edges[(u, v)] == wt and 1 <= wt <= 9
    # power law: the low ids carry the high degrees
    assert deg[:30].mean() > 4 * deg.mean()


def test_loguniform_weights_and_query_mix():
    g = synth.chung_lu(5000, 10, 2.3, ("loguniform", 1, 1024), seed=2)
    assert g.w.min() >= 1 and g.w.max() <= 1024
    # log-uniform: about as many weights in [1,32) as in [32,1024]
    lo = (g.w < 32).mean()
    assert 0.4 < lo < 0.6
    q = synth.query_mix(g, 100, 100, seed=1)
    hubs = set(synth.hub_set(g).tolist())
    assert q.shape == (200,) and sum(int(x) in hubs for x in q) >= 100
    assert ((q >= 0) & (q < g.n)).all()
    assert abs(synth.det_pow(2.0, 10.0) - 1024.0) < 1e-9


def test_small_topk_fixture():
    g = synth.workload_graph("small")
    P = oracle.sample_paths(g, 1, 200_000, 5, oracle.ALIAS)
    o = oracle.Oracle(g.n, P)
    with open(os.path.join(GOLDEN, "small_topk.txt")) as f:
        lines = [ln for ln in f if not ln.startswith("#")]
    for ln in lines:
        v, rest = ln.split(":", 1)
        pairs = [tuple(map(int, x.split(":"))) for x in rest.split()]
        ids, cnt = o.topk(int(v), 10)
        assert list(zip(ids.tolist(), cnt.tolist())) == pairs


def test_sample_size_fixture():
    import math
    with open(os.path.join(GOLDEN, "sample_size.txt")) as f:
        for ln in f:
            if ln.startswith("#"):
                continue
            E, R = map(int, ln.split())
            assert oracle.sample_size(math.sqrt(1.0 / E), 0.1, 0.5, 5) == R
            # eps^2 = 1/|E| makes R ~ 3.3123 |E|
            assert abs(R / E - 3.3122566) < 1e-3
