"""Host-side rules (no GPU): the interpolated route's sample count chosen
from a pseudo-C_l error budget; bench.py's --gpus N outside torchrun
refusing to run fewer ranks than asked for; and the JSON line of bench.py's
reference arm (the oracle on the host cores)."""
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


def _bench(args, extra_env=None):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(root, "bench.py"), *args], capture_output=True, text=True,
                          env=env, timeout=600, cwd=root)


def test_bench_reference_arm_line():
    """--impl reference (the FP64 oracle timed on the host cores, on a bounded
    sample of the workload) prints one JSON line with the contract's keys: the
    same metric, unit and direction as the library's line, a cpu_baseline of
    kind "oracle" naming its cores and sample, and an e2e block with no
    host-device bytes; a rank other than 0 prints nothing and exits 0."""
    args = ["--impl", "reference", "--steps", "1", "--warmup", "1", "--scale", "0.01", "--lmax", "256"]
    r = _bench(args)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["higher_is_better"] is True
    assert line["unit"] == "points*modes/s" and line["value"] > 0 and line["steps"] == 1
    assert line["config"]["lmax"] == 256 and "lognormal_cap" in line["config"]["workload"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    r1 = _bench(args, {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r1.returncode == 0 and r1.stdout.strip() == "", (r1.stdout[-500:], r1.stderr[-2000:])
