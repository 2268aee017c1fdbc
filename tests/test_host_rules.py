"""Host-side rules (no GPU): the interpolated route's sample count chosen
from a pseudo-C_l error budget, and bench.py's --gpus N outside torchrun
refusing to run fewer ranks than asked for."""
import json
import os
import subprocess
import sys

import pytest

from paper_2312_12285_gb300 import ops


def _model_err(lmax, n):
    # the rule's own error model: 4.3e-6 (16 lmax / N)^4 (cubic Hermite spline, h^4)
    return 4.3e-6 * (16.0 * lmax / n) ** 4


@pytest.mark.parametrize("lmax", [1, 32, 128, 1024, 1536, 2048, 4096])
@pytest.mark.parametrize("tol", [1e-6, 1e-5, 1e-4, 1e-3])
def test_ntheta_meets_its_budget_and_is_smallest(lmax, tol):
    n = ops.ntheta_for_tolerance(lmax, tol)
    assert n % 2 == 0 and 2 <= n <= 32768
    if n < 32768:
        assert _model_err(lmax, n) <= tol / 4.0 * (1 + 1e-12)
        if n > 2:  # the next even count down no longer meets it
            assert _model_err(lmax, n - 2) > tol / 4.0 * (1 - 1e-9)


def test_ntheta_monotone():
    for tol in (1e-5, 1e-4):
        ns = [ops.ntheta_for_tolerance(l, tol) for l in range(16, 4097, 240)]
        assert ns == sorted(ns)
    for lmax in (512, 2048):
        ns = [ops.ntheta_for_tolerance(lmax, t) for t in (1e-6, 1e-5, 1e-4, 1e-3)]
        assert ns == sorted(ns, reverse=True)


def test_ntheta_benchmark_value():
    # the sample count the bench's interpolated lines use at lmax 2048 and 1536
    assert ops.ntheta_for_tolerance(2048, 1e-4) == 21104
    assert ops.ntheta_for_tolerance(1536, 1e-4) == 15828


def test_bench_gpus_refuses_missing_gpus():
    """--gpus N > 1 without WORLD_SIZE starts N ranks itself; on a node with
    fewer than N GPUs it prints one JSON error line and exits 2 instead of
    running (and reporting) fewer ranks."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--steps", "1"],
                       capture_output=True, text=True, env=env, timeout=300, cwd=root)
    assert r.returncode == 2, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert "--gpus 2" in line["error"]
