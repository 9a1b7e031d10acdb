"""bench.py's command-line contract on the CPU (no GPU needed).

The reference arm times the oracle on the host cores; its JSON line must carry
the keys the benchmark contract names, and under torchrun only rank 0 prints.
The GPU arm must fail loudly (non-zero exit, no JSON line) when no CUDA device
is present: there is no CPU fallback.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, timeout=600, env=None):
    return subprocess.run([sys.executable] + args, cwd=ROOT, capture_output=True, text=True, timeout=timeout,
                          env=env)


def _json_lines(text):
    return [json.loads(line) for line in text.splitlines() if line.startswith("{")]


def test_reference_arm_json_line():
    out = _run(["bench.py", "--impl", "reference", "--workload", "small", "--steps", "1", "--warmup", "3"])
    assert out.returncode == 0, out.stderr[-2000:]
    lines = _json_lines(out.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "queries/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] >= 3 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "small"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_under_torchrun_prints_once():
    out = _run(["-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
                "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference", "--workload",
                "small", "--gpus", "2", "--steps", "1", "--warmup", "3"])
    assert out.returncode == 0, out.stderr[-2000:]
    lines = _json_lines(out.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference"


def test_gpu_arm_fails_loudly_without_cuda():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    out = _run(["bench.py", "--workload", "small", "--steps", "1", "--warmup", "3"])
    assert out.returncode != 0
    assert not _json_lines(out.stdout)


def test_oracle_run_parity_check_logic():
    # the benchmark's parity block: the GPU's results stand in here as the
    # oracle's own (all identical), then one changed path entry, index entry
    # and top-k count are each caught
    import numpy as np
    import bench
    import oracle
    import synth
    g = synth.workload_graph("small")
    R, T, k = 20_000, 5, 10
    q = np.arange(g.n, dtype=np.int32)
    run = bench.OracleRun(g, R, T, k, threads=2, queries=q, keep_rows=True)
    run.step(seed=3, n_mid=300, n_light=300)
    ids, cnt = run.o.topk_many(q, k, threads=2)
    gpu = {"paths": run.paths.copy(), "off": run.o.off.copy(), "pid": run.o.pid[: run.nnz].copy(),
           "ids": ids.copy(), "cnt": cnt.copy()}
    res = run.check(gpu, q)
    assert res["paths_identical"] and res["index_identical"] and res["topk_identical"]
    assert res["topk_rows_compared"] >= 256 and res["index_pairs_compared"] == run.nnz
    bad = dict(gpu, paths=gpu["paths"].copy())
    bad["paths"][7, 3] ^= 1
    assert not run.check(bad, q)["paths_identical"]
    bad = dict(gpu, pid=gpu["pid"].copy())
    bad["pid"][11] += 1
    assert not run.check(bad, q)["index_identical"]
    bad = dict(gpu, cnt=gpu["cnt"].copy())
    heavy = int(run.heavy[0])
    bad["cnt"][heavy, 0] += 1
    assert not run.check(bad, q)["topk_identical"]
