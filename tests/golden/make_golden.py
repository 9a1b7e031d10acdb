"""Writes the stored expected values under tests/golden/ (calls only oracle/ and synth/).

    python tests/golden/make_golden.py

small_topk.txt: the 'small' workload (Chung-Lu N=2000, mean degree 10,
gamma 2.5, weights U[1,16], seed 1; T=5, R=200,000 alias-mode paths, seed 1),
top-10 (ids and counts) of vertices 0..63, one line per vertex.
sample_size.txt: R of Sec. 3.2 for the eps = sqrt(1/|E|) rule of the
Implementation Notes (c=0.5, delta=0.1, T=5) at the |E| of Table 2's Tencent
sub-networks.
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

TENCENT_E = [10_000, 50_000, 100_000, 500_000, 1_000_000, 5_000_000, 10_000_000,
             50_000_000, 100_000_000, 500_000_000, 1_000_000_000]


def main():
    g = synth.workload_graph("small")
    P = oracle.sample_paths(g, 1, 200_000, 5, oracle.ALIAS)
    o = oracle.Oracle(g.n, P)
    with open(os.path.join(HERE, "small_topk.txt"), "w") as f:
        f.write("# vertex: id:count x10  (small workload, alias mode, seed 1)\n")
        for v in range(64):
            ids, cnt = o.topk(v, 10)
            f.write(f"{v}: " + " ".join(f"{i}:{c}" for i, c in zip(ids, cnt)) + "\n")
    with open(os.path.join(HERE, "sample_size.txt"), "w") as f:
        f.write("# |E| R  (Sec. 3.2 bound, c=0.5 delta=0.1 T=5, eps=sqrt(1/|E|); |E| from Table 2)\n")
        for E in TENCENT_E:
            f.write(f"{E} {oracle.sample_size(math.sqrt(1.0 / E), 0.1, 0.5, 5)}\n")


if __name__ == "__main__":
    main()
