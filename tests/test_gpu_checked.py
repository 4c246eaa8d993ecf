"""The bounds-checked build (-DVECCHIA_CHECKED) on the GPU.

compute-sanitizer is not available on the GPUs these tests run on, so the library has
a build in which every index the kernels read through (conditioning sets, the location
itself, the batched work items) is checked against its range before use; a bad one is
recorded in the error slot (status EINVAL from vecchia_last_error_location) and the
affected outputs become NaN, without any out-of-bounds access, trap or fault.  Here the
checked library (selected by VECCHIA_CHECKED=1) runs a cross-section of the parity
tests in a child process: every kernel family must give the oracle's results with the
checks on, and no check may fire on valid plans.
"""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SELECTION = [
    "tests/test_gpu_parity.py::test_small_exact_workload_full_parity",
    "tests/test_gpu_parity.py::test_gradient_terms_parity",
    "tests/test_gpu_parity.py::test_lanes_per_location_shapes_match_oracle",
    "tests/test_gpu_parity.py::test_large_conditioning_sets_match_oracle",
    "tests/test_gpu_parity.py::test_not_positive_definite_reports_location",
    "tests/test_gpu_range.py",
    "tests/test_gpu_batched.py",
    "tests/test_gpu_predict.py",
    "tests/test_gpu_sphere.py",
]


def test_checked_build_runs_the_parity_cross_section():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_07412_gb300 import build

    lib = build.build(checked=True)
    assert lib.endswith("libvecchia_checked.so")
    env = dict(os.environ, VECCHIA_CHECKED="1")
    probe = subprocess.run([sys.executable, "-c", "from paper_2403_07412_gb300 import vecchia as V; "
                            "print(V.LIB_PATH)"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert probe.returncode == 0 and probe.stdout.strip().endswith("libvecchia_checked.so"), probe.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + SELECTION,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
