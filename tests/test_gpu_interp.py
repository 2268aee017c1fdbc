"""The interpolated transform (pointsht_alm_interp, App. "Interpolation" with
samples in theta) on the GPU.

Two comparisons:
  * against the oracle's interpolated transform (same algorithm, FP64): the
    difference is the GPU's rounding only (FP32 binning and recurrence,
    fp16 hi + lo products): a_lm rows and C_l within 1e-5;
  * against the exact transform (oracle.alm): the interpolation error, h^4
    small: C_l within 1e-4 (the mixed-path target) at 16 samples per
    multipole, a_lm rows within 1e-4.
"""
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


def _cats(wl, dev):
    return [ops.Cat(torch.from_numpy(np.ascontiguousarray(c.x, np.float32)).to(dev),
                    torch.from_numpy(np.ascontiguousarray(c.phi, np.float32)).to(dev),
                    torch.from_numpy(np.ascontiguousarray(c.w, np.float32)).to(dev), c.field, c.coeff)
            for c in wl.catalogs]


def _run(dev, wl, ntheta, nfield=1):
    plan = ops.get_plan(wl.lmax, dev)
    a = ops.alm_interp(plan, _cats(wl, dev), nfield, ntheta)
    torch.cuda.synchronize()
    plan.check()
    return a.cpu().numpy()


def _field(wl, f=0):
    sel = [c for c in wl.catalogs if c.field == f]
    x = np.concatenate([c.x for c in sel]).astype(np.float64)
    phi = np.concatenate([c.phi for c in sel]).astype(np.float64)
    w = np.concatenate([c.w.astype(np.float64) * c.coeff for c in sel])
    return x, phi, w


def _cl_err(a, ref, L):
    c, r = oracle.cl(a, a, L), oracle.cl(ref, ref, L)
    return float(np.max(np.abs(c[1:] - r[1:]) / r[1:]))


@pytest.fixture(scope="module")
def cap(dev):
    L = 96
    wl = catalogs.lognormal_cap(3_000, 27_000, L, config_id=41, nwaves=64, grid=(128, 256))
    return wl, _field(wl)


@pytest.mark.parametrize("per_l", [8, 16])
def test_matches_interpolation_oracle(dev, cap, per_l):
    wl, (x, phi, w) = cap
    L = wl.lmax
    got = _run(dev, wl, per_l * L)[0]
    ref = oracle.alm_interp(x, phi, w, L, per_l * L)
    assert oracle.rel_err_per_l(got, ref, L) <= 1e-5
    assert _cl_err(got, ref, L) <= 1e-5


def test_interpolation_error_against_exact_transform(dev, cap):
    wl, (x, phi, w) = cap
    L = wl.lmax
    got = _run(dev, wl, 16 * L)[0]
    ref = oracle.alm(x, phi, w, L)
    assert oracle.rel_err_per_l(got, ref, L) <= 1e-4
    assert _cl_err(got, ref, L) <= 1e-4


def test_run_to_run_bitwise(dev, cap):
    wl, _ = cap
    a = _run(dev, wl, 16 * wl.lmax)
    b = _run(dev, wl, 16 * wl.lmax)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("L,ntheta,n", [(37, 592, 4_001), (1, 2, 300), (64, 1024, 70_000), (20, 320, 7)])
def test_ragged_sizes(dev, L, ntheta, n):
    """Samples not a multiple of the 1024-sample tile (padding), odd lmax,
    the smallest grid, more points than one sort range (65536), tiny sets."""
    rng = catalogs.rng_for(42, n)
    x = rng.uniform(-1, 1, n).astype(np.float32)
    phi = rng.uniform(0, 2 * np.pi, n).astype(np.float32)
    w = rng.uniform(0.5, 1.5, n).astype(np.float32)
    wl = catalogs.Workload("t", L, "fp32", 1, [catalogs.Catalog(x, phi, w, 1.0, 0)])
    got = _run(dev, wl, ntheta)[0]
    ref = oracle.alm_interp(x.astype(np.float64), phi.astype(np.float64), w.astype(np.float64), L, ntheta)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_pole_points(dev):
    """Points at and next to both poles use the ghost samples; the sample
    positions next to the pole run the near-pole (difference) form of the
    FP32 recurrence, so the values there hold the FP32 level: 1e-5 of the
    largest value against the interpolation oracle."""
    L = 48
    x = np.array([1.0, -1.0, 1.0 - 1e-7, -1.0 + 3e-6, 0.99999], np.float32)
    phi = np.array([0.1, 1.2, 2.3, 3.4, 4.5], np.float32)
    w = np.array([1.0, 0.7, 1.3, 0.9, 1.1], np.float32)
    wl = catalogs.Workload("poles", L, "fp32", 1, [catalogs.Catalog(x, phi, w, 1.0, 0)])
    got = _run(dev, wl, 16 * L)[0]
    ref = oracle.alm_interp(x.astype(np.float64), phi.astype(np.float64), w.astype(np.float64), L, 16 * L)
    exact = oracle.alm(x.astype(np.float64), phi.astype(np.float64), w.astype(np.float64), L)
    scale = np.max(np.abs(exact))
    assert np.max(np.abs(got - ref)) <= 1e-5 * scale
    assert np.max(np.abs(got - exact)) <= 1e-4 * scale


def test_two_fields_and_an_empty_one(dev):
    L = 40
    wl = catalogs.uniform_fullsky(2_000, 6_000, 0.3, L, np.float32, config_id=43, precision="fp32")
    wl.catalogs[1].field = 1
    wl.nfield = 3  # field 2 has no catalog
    got = _run(dev, wl, 16 * L, nfield=3)
    for f in (0, 1):
        x, phi, w = _field(wl, f)
        ref = oracle.alm_interp(x, phi, w, L, 16 * L)
        assert oracle.rel_err_per_l(got[f], ref, L) <= 1e-5
    assert np.all(got[2] == 0)


def test_six_fields_span_groups_and_passes(dev):
    """Six fields (transform groups of 4 + 2; passes of 8 columns that span
    fields), uneven sizes and an empty fifth field: each field against the
    oracle, and against the same field transformed alone."""
    L = 48
    rng = np.random.default_rng(4406)
    sizes = [5_000, 300, 2_500, 40, 0, 1_200]
    cats_np = []
    for f, n in enumerate(sizes):
        if n == 0:
            continue
        x, phi = catalogs.uniform_sphere(rng, n)
        w = rng.uniform(0.5, 1.5, n).astype(np.float32)
        cats_np.append((x, phi, w, f, 1.0 - 0.3 * f))
    cats = [ops.Cat(*(torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (x, phi, w)), f, co)
            for (x, phi, w, f, co) in cats_np]
    plan = ops.get_plan(L, dev)
    nt = 16 * L
    got = ops.alm_interp(plan, cats, 6, nt).cpu().numpy()
    plan.check()
    assert np.all(got[4] == 0)
    for (x, phi, w, f, co), c in zip(cats_np, cats):
        ref = oracle.alm_interp(x.astype(np.float64), phi.astype(np.float64), w.astype(np.float64) * co, L, nt)
        assert oracle.rel_err_per_l(got[f], ref, L) <= 1e-5, f
        alone = ops.alm_interp(plan, [ops.Cat(c.x, c.phi, c.w, 0, co)], 1, nt).cpu().numpy()[0]
        assert np.max(np.abs(got[f] - alone)) <= 1e-6 * np.max(np.abs(alone)), f


def test_argument_errors(dev):
    wl = catalogs.uniform_fullsky(10, 10, 0.3, 8, np.float32, config_id=44, precision="fp32")
    plan = ops.get_plan(8, dev)
    for nt in (15, 0, 32770):
        with pytest.raises(_lib.PointSHTError) as ei:
            ops.alm_interp(plan, _cats(wl, dev), 1, nt)
        assert ei.value.status == _lib.EINVAL


def test_field_of_2_31_points_is_refused(dev):
    """The route's binning counts are 32-bit, so a field of 2^31 points or
    more is refused on the host before anything is enqueued: two catalogs of
    2^30 points on one field give EINVAL naming the limit and a zero
    workspace size, while 2^31 - 1 points pass the size query.  The call is
    made with NULL output and workspace (and catalogs whose arrays are far
    shorter than their counts), so no kernel could run even past the check."""
    plan = ops.get_plan(8, dev)
    t = torch.zeros(32, dtype=torch.float32, device=dev)
    p = t.data_ptr()
    arr, n = _lib.catalog_array([(p, p, p, 1 << 30, 0, 1.0)] * 2)
    assert plan.lib.pointsht_workspace_size_interp(plan.handle, arr, n, 1, 64) == 0
    assert plan.lib.pointsht_alm_interp(plan.handle, arr, n, 1, 64, None, None, 0, None) == _lib.EINVAL
    assert "2^31 or more points" in _lib.last_error()
    arr, n = _lib.catalog_array([(p, p, p, 1 << 30, 0, 1.0), (p, p, p, (1 << 30) - 1, 0, 1.0)])
    assert plan.lib.pointsht_workspace_size_interp(plan.handle, arr, n, 1, 64) > 0


# ------------------------------------------------------------------ full size --
@pytest.fixture(scope="module")
def full(dev):
    wl = catalogs.config(3)
    assert wl.npoints == 10_000_000 and wl.lmax == 2048
    return wl, _run(dev, wl, 32768)[0]


def test_fullsize_sampled_columns(full):
    """Columns m = 0 (largest values near the poles) and the short columns
    m = 1900, 2047, 2048 over all 1e7 points against the exact transform;
    m = 0 carries the FP32 recurrence's near-pole error (3e-4, as for the
    direct FP32 path at this size)."""
    wl, got = full
    L = wl.lmax
    x, phi, w = _field(wl)
    tol = {0: 3e-4, 1900: 1e-4, 2047: 1e-4, 2048: 1e-4}
    ref = oracle.alm(x, phi, w, L, mlist=list(tol))
    for m, col in ref.items():
        g = got[oracle.index(m, m, L):oracle.index(L, m, L) + 1]
        assert np.linalg.norm(g - col) <= tol[m] * np.linalg.norm(col), m


def test_fullsize_low_l_pseudo_cl(full):
    wl, got = full
    L, Ls = wl.lmax, 32
    x, phi, w = _field(wl)
    ref = oracle.alm(x, phi, w, Ls)
    sub = np.concatenate([got[oracle.index(m, m, L):oracle.index(Ls, m, L) + 1] for m in range(Ls + 1)])
    assert _cl_err(sub, ref, Ls) <= 1e-4


def test_fullsize_matches_direct_fp32_path(full, dev):
    """Whole triangle against the direct FP32 path (itself held to 1e-5 of
    the oracle): C_l within 1e-4 at every l."""
    wl, got = full
    plan = ops.get_plan(wl.lmax, dev)
    direct = ops.alm_raw(plan, _cats(wl, dev), 1, "fp32").cpu().numpy()[0]
    assert _cl_err(got, direct, wl.lmax) <= 1e-4
