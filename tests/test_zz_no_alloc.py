"""pointsht_alm_noalloc: the transform for callers that cannot allocate device
memory (for example a host framework that owns every device allocation, so no
workspace can be handed in).  Its scratch is a fixed array inside the library
that keeps whatever the previous call left in it.  So before each compared
call the array is filled with other data (a larger catalog with other
weights, two fields), and the compared call's results must match
pointsht_alm, which uses a caller workspace, on two calls in a row: nothing
stale may leak into the result, including from regions the smaller call does
not use.

This file is collected last on purpose; the last test runs it again, alone,
in a fresh process, where the first no-allocation call of the process is the
one that looks up the array."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_12285_gb300 import _lib, catalogs, ops  # noqa: E402

pytestmark = pytest.mark.gpu

NOALLOC_BYTES = 64 * 1024 * 1024  # POINTSHT_NOALLOC_SCRATCH_BYTES in include/pointsht.h


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def _noalloc(plan, cats, nfield, precision, out):
    arr, n = _lib.catalog_array(ops._entries(cats, precision, plan.device))
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return plan.lib.pointsht_alm_noalloc(plan.handle, arr, n, nfield, _lib.PRECISIONS[precision],
                                         ctypes.c_void_p(out.data_ptr()), st)


def _cats(wl, dev):
    return [ops.Cat(torch.from_numpy(c.x).to(dev), torch.from_numpy(c.phi).to(dev), torch.from_numpy(c.w).to(dev),
                    c.field, c.coeff) for c in wl.catalogs]


@pytest.mark.parametrize("precision,lmax,ng,nr", [("fp32", 256, 20_000, 60_000), ("fp64", 96, 3_000, 9_000)])
def test_noalloc_matches_workspace_path_twice(dev, precision, lmax, ng, nr):
    dt = np.float64 if precision == "fp64" else np.float32
    wl = catalogs.uniform_fullsky(ng, nr, 0.25, lmax, dt, config_id=21, precision=precision)
    cats = _cats(wl, dev)
    # a larger catalog with other weights over two fields, to leave other data
    # in every part of the array the compared call uses (and in parts it does not)
    big = catalogs.uniform_fullsky(2 * ng, 2 * nr, 0.4, lmax, dt, config_id=23, precision=precision)
    big.catalogs[1].field = 1
    bcats = _cats(big, dev)
    for c in bcats:
        c.w.mul_(3.0)
    plan = ops.get_plan(lmax, dev)
    assert ops.workspace_bytes(plan, bcats, 2, precision) <= NOALLOC_BYTES
    assert ops.workspace_bytes(plan, bcats, 2, precision) > ops.workspace_bytes(plan, cats, 1, precision)
    ref = ops.alm_raw(plan, cats, 1, precision).cpu().numpy()
    tol = 1e-12 if precision == "fp64" else 1e-6  # tolerances of the parity tests (FP64 / FP32 paths)
    scale = np.max(np.abs(ref))
    for _ in range(2):
        junk = torch.empty((2, plan.nmodes), dtype=torch.complex128, device=dev)
        _lib.check(_noalloc(plan, bcats, 2, precision, junk), "alm_noalloc (other data)")
        out = torch.full((1, plan.nmodes), complex("nan"), dtype=torch.complex128, device=dev)
        _lib.check(_noalloc(plan, cats, 1, precision, out), "alm_noalloc")
        torch.cuda.synchronize()
        plan.check()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= tol * scale


def test_noalloc_rejects_oversized_request(dev):
    lmax = 2048  # one accumulation slot alone is 33.6 MB; several slots exceed the fixed array
    wl = catalogs.uniform_fullsky(100_000, 900_000, 0.1, lmax, np.float32, config_id=22, precision="fp32")
    cats = [ops.Cat(torch.from_numpy(c.x).to(dev), torch.from_numpy(c.phi).to(dev), torch.from_numpy(c.w).to(dev),
                    c.field, c.coeff) for c in wl.catalogs]
    plan = ops.get_plan(lmax, dev)
    assert ops.workspace_bytes(plan, cats, 1, "fp32") > NOALLOC_BYTES
    out = torch.zeros((1, plan.nmodes), dtype=torch.complex128, device=dev)
    assert _noalloc(plan, cats, 1, "fp32", out) == _lib.ENOMEM
    assert "scratch" in _lib.last_error()


@pytest.mark.skipif(os.environ.get("POINTSHT_NOALLOC_CHILD") == "1", reason="already the fresh process")
def test_noalloc_in_a_fresh_process(dev):
    """This file's tests, alone in a new process (first use of the array there)."""
    env = dict(os.environ, POINTSHT_NOALLOC_CHILD="1")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                        os.path.abspath(__file__)], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
