"""The packed FP32 sweeps in thread-block clusters against the oracle. For a few
directions the library keeps one CTA per direction by default (faster than a
cluster, whose CTAs wait on a cluster barrier at every exchange), so the cluster
kernels run only for grids too large for one CTA or under SC4DVAR_FEW_CLUSTER.
Here the few-direction parity cases of test_gpu_burgers.py rerun in a child
process with the knob at 8 (the variable is read once per process)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = ["8192-20-3-fp32", "1024-20-1-fp32"]


def test_cluster_sweeps_match_oracle():
    ids = [f"tests/test_gpu_burgers.py::test_register_resident_sweeps_match_oracle[{c}]" for c in CASES]
    env = dict(os.environ, SC4DVAR_FEW_CLUSTER="8")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", *ids], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert f"{len(CASES)} passed" in r.stdout
