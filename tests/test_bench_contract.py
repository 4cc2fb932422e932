"""bench.py's measurement arithmetic and its reference arm, without a GPU: the algorithmic
operation and byte counts the roofline fractions divide by, restated from their definitions
(Philox4x32-10 per call of four normals, Box-Muller per pair, the recursion of Eq. (state_space),
a radix-4 C2R FFT; the tables A and B read once per (mode, ring)), and the JSON line of
`bench.py --impl reference` (the oracle's Alg. 2 recursion on the host)."""
import importlib.util
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_algorithmic_operation_counts():
    b = _bench()
    # p = 1, 16384 complex points: Philox 40 x 2/4 = 20, Box-Muller 12, recursion 2 x (1 + 1) = 4,
    # FFT 10 + 3.5 x 14 = 59: 95 per item; without the integer Philox part (FP64 pipe) 75
    assert b.alg_ops_per_item(1, 16384) == pytest.approx(20 + 12 + 4 + 59)
    assert b.alg_ops_per_item(1, 16384, fp64=True) == pytest.approx(12 + 4 + 59)
    # p = 2, 1024 points: Philox 40, Box-Muller 24, recursion 2 x (4 + 3) = 14, FFT 45: 123
    assert b.alg_ops_per_item(2, 1024) == pytest.approx(123)
    # p = 3: Philox 60, Box-Muller 36, recursion 2 x (9 + 6) = 30
    assert b.alg_ops_per_item(3, 1024) == pytest.approx(60 + 36 + 30 + 45)
    assert b.sfu_ops_per_item(2) == 8


def test_algorithmic_table_bytes():
    b = _bench()
    # 16384 x 32768, p = 1, FP32: (16385 modes) x 16384 rings x (1 + 1) values x 4 bytes
    assert b.alg_table_bytes(1, 16384, 32768, False) == 16385 * 16384 * 8
    # 1024 x 2048, p = 2, FP32: 7 values per (mode, ring), 28 bytes
    assert b.alg_table_bytes(2, 1024, 2048, False) == 1025 * 1024 * 28
    assert b.alg_table_bytes(2, 1024, 2048, True) == 1025 * 1024 * 56


def test_alu_peak():
    b = _bench()
    assert b.alu_peak(False, 2070.0) == pytest.approx(152 * 128 * 2070e6)


@pytest.mark.timeout(600)
def test_reference_arm_json_line():
    """The reference arm runs the oracle on the host and prints one JSON line with the contract's
    keys; its end-to-end entry is its own value, with no host-device copies."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "plain-64x128-p1-fp64", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "points/s"
    assert d["cpu_baseline"]["kind"].startswith("oracle") and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["name"] == "plain-64x128-p1-fp64"
