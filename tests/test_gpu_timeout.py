"""The bounded waits' give-up path, exercised without faulting or hanging a
GPU: with the plan's wait probe on, the first CTA of the analysis launch waits
on a shared-memory barrier that no copy and no thread ever arrives at, gives
up, records the timeout and leaves before it takes a work unit or issues a
copy (nothing is left in flight).  pointsht_plan_check then reports
POINTSHT_ETIMEOUT; the other CTAs have taken every unit, so the a_lm are
complete; with the probe off the next call reports no error and gives the
same a_lm bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2312_12285_gb300 import _lib, catalogs, ops  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_wait_probe_reports_timeout_then_recovers(dev, prec):
    L = 96
    dt = np.float32 if prec == "fp32" else np.float64
    wl = catalogs.uniform_fullsky(20_000, 60_000, 0.25, L, dt, config_id=12, precision=prec)
    cats = [ops.Cat(*(torch.from_numpy(v).to(dev) for v in (c.x, c.phi, c.w)), c.field, c.coeff)
            for c in wl.catalogs]
    plan = ops.Plan(L, dev)
    plan.check()
    plan.set_wait_probe(True)
    a1 = ops.alm_raw(plan, cats, 1, prec).cpu().numpy()[0]
    torch.cuda.synchronize()
    with pytest.raises(_lib.PointSHTError) as err:
        plan.check()
    assert err.value.status == _lib.ETIMEOUT
    plan.set_wait_probe(False)
    a2 = ops.alm_raw(plan, cats, 1, prec).cpu().numpy()[0]
    plan.check()  # the error word was cleared by the previous check; nothing new
    assert np.array_equal(a1.view(np.uint64), a2.view(np.uint64))
    ref = oracle.field_alm([(c.x, c.phi, c.w, c.coeff) for c in wl.catalogs], L)
    assert oracle.rel_err_per_l(a2, ref, L) <= (1e-10 if prec == "fp64" else 1e-5)
