"""bench.py's host-side contract, without a GPU: the default workload label, the
algorithmic flop count behind the roofline, and the reference arm's JSON line (the CPU
oracle on a tiny sample)."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_default_workload_label_is_the_headline_configuration():
    assert bench.workload_label(1_000_000, 60, "maxmin", False) == bench.WORKLOAD
    assert bench.workload_label(30_000, 150, "random", True) == "vecchia-matern-gmm30000-random-m150-nu1.0-fwd"


def test_la_flops_counts_each_location_block():
    # per location: Cholesky k^3/3 + k^2/2 + k/6 plus two solves k^2, k = min(i, m) + 1;
    # the adjoint adds 2 m_i^2 (LAPACK's dpotrf count, by hand for n = 4, m = 2)
    def f(k):
        return k ** 3 / 3 + k ** 2 / 2 + k / 6 + k ** 2
    ks = [1, 2, 3, 3]
    assert abs(bench.la_flops(4, 2, False) - sum(f(k) for k in ks)) < 1e-9
    assert abs(bench.la_flops(4, 2, True) - sum(f(k) + 2 * (k - 1) ** 2 for k in ks)) < 1e-9
    # m = 60 at 1M: about 81.3 kflop per location forward, 88.4 kflop with the gradient
    assert abs(bench.la_flops(1_000_000, 60, False) / 1e6 - 81.3e3) < 0.1e3
    assert abs(bench.la_flops(1_000_000, 60, True) / 1e6 - 88.4e3) < 0.1e3


def test_kernel_source_hash_is_stable():
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    assert h == bench.kernel_source_hash()


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "2000",
                          "--steps", "1", "--warmup", "3", "--ref-budget", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "locations/s"
    assert d["value"] > 0 and np.isfinite(d["value"]) and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == bench.workload_label(2000, 60, "maxmin", False)
