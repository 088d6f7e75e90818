"""The benchmark's JSON contract (CPU only): the oracle arm prints one line with the keys the
harness reads, and the algorithmic flop model of the roofline sums to Table 1's CWY and MGS
counts."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "uniform1000", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
                "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference" and out["metric"] == "eigvecs_per_s"
    assert out["value"] > 0 and out["higher_is_better"] is True
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in out["config"]


def test_algorithmic_flops_sum_to_table1():
    # one cluster of m members (head 0) in an order-n problem, one sweep per vector: members
    # k = 1..m-1 each cost 8nk - 3k^2 (CWY) or 4nk (MGS)
    n, m = 1000, 40
    head = np.zeros(m, dtype=np.int64)
    iters = np.ones(m, dtype=np.int32)
    cwy = bench.algorithmic_flops(n, head, iters, "cwy")
    mgs = bench.algorithmic_flops(n, head, iters, "mgs")
    k = np.arange(1, m)
    assert cwy == float(np.sum(8.0 * n * k - 3.0 * k * k))
    assert mgs == float(np.sum(4.0 * n * k))
    # the closed sums: 4nm(m-1) - (m-1)m(2m-1)/2 and 2nm(m-1), i.e. 4m^2n - m^3 and 2m^2n to
    # leading order (Table 1)
    assert cwy == 4.0 * n * m * (m - 1) - (m - 1) * m * (2 * m - 1) / 2.0
    assert mgs == 2.0 * n * m * (m - 1)
    # sweep counts multiply; non-converged vectors (negative counts) count their sweeps too;
    # singletons and heads cost nothing
    iters3 = np.full(m, 3, dtype=np.int32)
    iters3[5] = -5
    expect = 3 * cwy + 2 * (8.0 * n * 5 - 3.0 * 25)
    assert bench.algorithmic_flops(n, head, iters3, "cwy") == expect
    assert bench.algorithmic_flops(n, np.arange(m), iters, "cwy") == 0.0
