"""CPU checks of the benchmark's host side: the reference arm (the oracle,
timed on the host cores) prints one JSON line with the keys the benchmark
contract fixes, and the adjusted Rand index the clustering legs report
agrees with the oracle's."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "sbm1k",
                          "--steps", "2", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "sbm1k"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_bench_adjusted_rand_matches_oracle(oracle_mod):
    sys.path.insert(0, ROOT)
    import bench

    rng = np.random.default_rng(11)
    for n, ka, kb in ((500, 3, 5), (4000, 20, 20), (50, 1, 3)):
        a = rng.integers(0, ka, n).astype(np.int32)
        b = np.where(rng.random(n) < 0.6, a % kb, rng.integers(0, kb, n)).astype(np.int32)
        assert abs(bench.adjusted_rand_index(a, b) - oracle_mod.adjusted_rand(a, b)) < 1e-12
    perm = rng.permutation(7)
    a = rng.integers(0, 7, 300).astype(np.int32)
    assert bench.adjusted_rand_index(a, perm[a]) == 1.0  # a relabelling is the same clustering
