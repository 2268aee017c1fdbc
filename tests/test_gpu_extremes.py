"""Extremes of size, against the FP64 oracle: the smallest lmax (1, 2, 3:
columns of one or two steps, order pairs that are a single column) through
every path; the largest lmax each path supports (FP32 recurrence 4096; FP64
the largest whose accumulator rows fit in shared memory, 2970 on a GB300) on
single points and small catalogs; and one field of more than 2^31 points (a
seeded pattern repeated on the device, so that the oracle's values for the
pattern give the expected ones) through the FP32 path and its adjoint, both
weight-column kernels, and the FP64 path and its adjoint.

Tolerances: FP64 path 1e-10 relative per multipole row (1e-13 on single-point
identities); FP32 path 1e-5 relative per row at low lmax, and at lmax 4096 the
single-point addition theorem C_l = w^2/4pi within 4e-5 (the FP32 recurrence
carries ~l eps per value); mixed path and interpolated route 1e-4 / 1e-5 as in
their own test files.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2312_12285_gb300 import catalogs, ops  # noqa: E402

pytestmark = pytest.mark.gpu

FOUR_PI = 4.0 * np.pi


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def _points(n, seed, dtype=np.float32):
    rng = np.random.default_rng(seed)
    x, phi = catalogs.uniform_sphere(rng, n, dtype)
    w = rng.uniform(0.5, 1.5, n).astype(dtype)
    return x, phi, w


def _cat(dev, x, phi, w, field=0, coeff=1.0):
    return ops.Cat(*(torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (x, phi, w)), field, coeff)


def _alm(dev, cats, L, prec, nfield=1):
    plan = ops.get_plan(L, dev)
    a = ops.alm_raw(plan, cats, nfield, prec)
    torch.cuda.synchronize()
    plan.check()
    return a.cpu().numpy()


@pytest.mark.parametrize("L", [1, 2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tiny_lmax_transform_and_adjoint(dev, L, prec):
    dt = np.float64 if prec == "fp64" else np.float32
    x, phi, w = _points(3001, 700 + L, dt)
    ref = oracle.alm(x.astype(np.float64), phi.astype(np.float64), w.astype(np.float64) * -0.7, L)
    got = _alm(dev, [_cat(dev, x, phi, w, 0, -0.7)], L, prec)[0]
    assert got.shape == ref.shape == (oracle.nmodes(L),)
    assert oracle.rel_err_per_l(got, ref, L) <= (1e-10 if prec == "fp64" else 1e-5)
    # adjoint with a random cotangent
    rng = np.random.default_rng(L)
    M = oracle.nmodes(L)
    g = rng.standard_normal((1, M)) + 1j * rng.standard_normal((1, M))
    plan = ops.get_plan(L, dev)
    (gw,) = ops.alm_backward_raw(plan, [_cat(dev, x, phi, w, 0, -0.7)], 1, prec, torch.from_numpy(g).to(dev))
    torch.cuda.synchronize()
    plan.check()
    r = -0.7 * oracle.adjoint(x.astype(np.float64), phi.astype(np.float64), g[0], L)
    got_g = gw.double().cpu().numpy()
    assert np.max(np.abs(got_g - r)) <= (1e-11 if prec == "fp64" else 2e-5) * np.max(np.abs(r))


@pytest.mark.parametrize("L", [1, 2, 3])
def test_tiny_lmax_mixed_and_interpolated(dev, L):
    x, phi, w = _points(2500, 800 + L)
    rng = np.random.default_rng(900 + L)
    W = np.stack([w, rng.uniform(0.8, 1.2, x.size).astype(np.float32), rng.standard_normal(x.size).astype(np.float32)])
    plan = ops.get_plan(L, dev)
    x64, p64 = x.astype(np.float64), phi.astype(np.float64)
    for kernel in ("mma.sync", "tcgen05"):
        plan.set_mixed_kernel(kernel)
        try:
            got = ops.alm_columns(plan, torch.from_numpy(x).to(dev), torch.from_numpy(phi).to(dev),
                                  torch.from_numpy(np.ascontiguousarray(W)).to(dev), "mixed").cpu().numpy()
            plan.check()
        finally:
            plan.set_mixed_kernel("mma.sync")
        for f in range(3):
            ref = oracle.alm(x64, p64, W[f].astype(np.float64), L)
            assert oracle.rel_err_per_l(got[f], ref, L) <= 1e-4, (kernel, f)
    nt = 16 * L
    gi = ops.alm_interp(plan, [_cat(dev, x, phi, w)], 1, nt).cpu().numpy()[0]
    plan.check()
    ri = oracle.alm_interp(x64, p64, w.astype(np.float64), L, nt)
    assert oracle.rel_err_per_l(gi, ri, L) <= 1e-5


def test_fp32_max_lmax_single_points_and_catalog(dev):
    """lmax 4096, the FP32 recurrence's limit: single points at x = 0.31, 0,
    0.97 and 1 obey the addition theorem C_l = w^2/4pi at every l, and 200
    random points match the oracle row by row."""
    L = 4096
    for xv in (0.31, 0.0, 0.97, 1.0):
        c = _cat(dev, np.array([xv], np.float32), np.array([1.3], np.float32), np.array([1.7], np.float32))
        a = _alm(dev, [c], L, "fp32")[0]
        cl = oracle.cl(a, a, L)
        assert np.max(np.abs(cl / (1.7 ** 2 / FOUR_PI) - 1.0)) <= 4e-5, xv
    x, phi, w = _points(200, 4096)
    got = _alm(dev, [_cat(dev, x, phi, w)], L, "fp32")[0]
    ref = oracle.alm(x.astype(np.float64), phi.astype(np.float64), w.astype(np.float64), L)
    assert oracle.rel_err_per_l(got, ref, L) <= 1e-4


def test_weight_columns_at_fp32_max_lmax(dev):
    """Weight columns at lmax 4096 through both contraction kernels (the
    tcgen05 kernel's coefficient copies grow with lmax: ~207 KB of shared
    memory there): 1 500 points, two columns, against the oracle."""
    L = 4096
    x, phi, w = _points(1500, 4097)
    W = np.stack([w, np.random.default_rng(4098).standard_normal(x.size).astype(np.float32)])
    plan = ops.get_plan(L, dev)
    x64, p64 = x.astype(np.float64), phi.astype(np.float64)
    ref = [oracle.alm(x64, p64, W[f].astype(np.float64), L) for f in range(2)]
    for kernel in ("mma.sync", "tcgen05"):
        plan.set_mixed_kernel(kernel)
        try:
            got = ops.alm_columns(plan, torch.from_numpy(x).to(dev), torch.from_numpy(phi).to(dev),
                                  torch.from_numpy(np.ascontiguousarray(W)).to(dev), "mixed").cpu().numpy()
            plan.check()
        finally:
            plan.set_mixed_kernel("mma.sync")
        for f in range(2):
            assert oracle.rel_err_per_l(got[f], ref[f], L) <= 1e-4, (kernel, f)


def test_fp64_max_lmax(dev):
    """The FP64 analysis keeps a CTA's per-warp accumulator rows in shared
    memory, so its lmax is bounded by the device (2970 on a GB300, below the
    plan's 8192): a larger plan is refused with EINVAL naming the bound, and at
    the bound a single point at x = -0.42 obeys the addition theorem to 1e-12
    and 60 random points match the oracle row by row to 1e-10."""
    import re
    from paper_2312_12285_gb300 import _lib
    c = _cat(dev, np.array([-0.42]), np.array([0.4]), np.array([0.9]))
    with pytest.raises(_lib.PointSHTError) as err:
        _alm(dev, [c], 8192, "fp64")
    assert err.value.status == _lib.EINVAL
    L = int(re.search(r"lmax <= (\d+)", str(err.value)).group(1))
    assert 2048 <= L < 8192
    a = _alm(dev, [c], L, "fp64")[0]
    cl = oracle.cl(a, a, L)
    assert np.max(np.abs(cl / (0.9 ** 2 / FOUR_PI) - 1.0)) <= 1e-12
    x, phi, w = _points(60, 8192, np.float64)
    got = _alm(dev, [_cat(dev, x, phi, w)], L, "fp64")[0]
    ref = oracle.alm(x, phi, w, L)
    assert oracle.rel_err_per_l(got, ref, L) <= 1e-10


def test_more_than_2_31_points_in_one_field(dev):
    """One field of 2 147 975 181 points (> 2^31; a 65 549-point seeded
    pattern repeated 32 769 times on the device, so the field also ends in a
    ragged, padded tail), lmax 64, FP32 path and its adjoint: every point
    index, sort range, chunk and point id past 2^31 is in use.  Expected
    values from the oracle on the pattern alone: a_lm = R x the pattern's a_lm
    (1e-4 per multipole row, the FP32 path's bound; a_00 to 1e-5), and the
    gradient of every copy equals the oracle gradient of its pattern point
    (2e-5 of the largest, as at small sizes), checked on 200 000 random copies
    and on the copies around index 2^31 and at the end."""
    torch.cuda.empty_cache()  # blocks cached by earlier tests count as used
    free, _ = torch.cuda.mem_get_info()
    if free < 110e9:
        pytest.skip("needs ~100 GB of free device memory")
    L, npat, R = 64, 65_549, 32_769
    n = npat * R
    assert n > 2**31
    x, phi, w = _points(npat, 2**31)
    xt, pt, wt = (torch.from_numpy(v).to(dev).repeat(R) for v in (x, phi, w))
    cat = ops.Cat(xt, pt, wt, 0, 1.0)
    x64, p64, w64 = x.astype(np.float64), phi.astype(np.float64), w.astype(np.float64)
    a = _alm(dev, [cat], L, "fp32")[0]
    ref = R * oracle.alm(x64, p64, w64, L)
    assert oracle.rel_err_per_l(a, ref, L) <= 1e-4
    a00 = R * np.sum(w64) / np.sqrt(FOUR_PI)
    assert abs(a[0] - a00) <= 1e-5 * a00
    rng = np.random.default_rng(2**31 + 1)
    M = oracle.nmodes(L)
    g = rng.standard_normal((1, M)) + 1j * rng.standard_normal((1, M))
    plan = ops.get_plan(L, dev)
    (gw,) = ops.alm_backward_raw(plan, [cat], 1, "fp32", torch.from_numpy(g).to(dev))
    torch.cuda.synchronize()
    plan.check()
    idx = np.concatenate([rng.integers(0, n, 200_000), np.arange(2**31 - 1000, 2**31 + 1000),
                          np.arange(n - 1000, n)]).astype(np.int64)
    got = gw[torch.from_numpy(idx).to(dev)].double().cpu().numpy()
    r = oracle.adjoint(x64, p64, g[0], L)[idx % npat]
    assert np.max(np.abs(got - r)) <= 2e-5 * np.max(np.abs(r))
    del xt, pt, wt, cat, gw
    torch.cuda.empty_cache()


def test_weight_columns_more_than_2_31_points(dev):
    """Two weight columns on 2 147 975 181 points (the 65 549-point pattern
    repeated 32 769 times), lmax 64, through both contraction kernels:
    alm = R x the oracle's a_lm of the pattern, column by column, at the
    mixed path's 1e-4 per multipole row."""
    torch.cuda.empty_cache()  # blocks cached by earlier tests count as used
    free, _ = torch.cuda.mem_get_info()
    if free < 110e9:
        pytest.skip("needs ~100 GB of free device memory")
    L, npat, R = 64, 65_549, 32_769
    x, phi, w = _points(npat, 2**31)
    w2 = np.random.default_rng(2**31 + 2).standard_normal(npat).astype(np.float32)
    xt, pt = (torch.from_numpy(v).to(dev).repeat(R) for v in (x, phi))
    W = torch.from_numpy(np.stack([w, w2])).to(dev).repeat(1, R)
    assert W.is_contiguous() and W.shape == (2, npat * R)
    x64, p64 = x.astype(np.float64), phi.astype(np.float64)
    ref = [R * oracle.alm(x64, p64, c.astype(np.float64), L) for c in (w, w2)]
    plan = ops.get_plan(L, dev)
    for kernel in ("mma.sync", "tcgen05"):
        plan.set_mixed_kernel(kernel)
        try:
            got = ops.alm_columns(plan, xt, pt, W, "mixed").cpu().numpy()
            plan.check()
        finally:
            plan.set_mixed_kernel("mma.sync")
        for f in range(2):
            assert oracle.rel_err_per_l(got[f], ref[f], L) <= 1e-4, (kernel, f)
    del xt, pt, W
    torch.cuda.empty_cache()


def test_fp64_more_than_2_31_points(dev):
    """The FP64 path and its catalog-order adjoint on one field of
    2 147 975 181 points (the 65 549-point pattern, in float64, repeated
    32 769 times), lmax 16: a_lm = R x the oracle's a_lm of the pattern
    (1e-10 per multipole row) and the gradient of every copy equals the
    oracle's gradient of its pattern point (1e-11 of the largest), sampled
    around index 2^31 and at the end."""
    torch.cuda.empty_cache()  # blocks cached by earlier tests count as used
    free, _ = torch.cuda.mem_get_info()
    if free < 150e9:
        pytest.skip("needs ~140 GB of free device memory")
    L, npat, R = 16, 65_549, 32_769
    n = npat * R
    x, phi, w = _points(npat, 2**31 + 3, np.float64)
    cat = ops.Cat(*(torch.from_numpy(v).to(dev).repeat(R) for v in (x, phi, w)), 0, 1.0)
    a = _alm(dev, [cat], L, "fp64")[0]
    assert oracle.rel_err_per_l(a, R * oracle.alm(x, phi, w, L), L) <= 1e-10
    rng = np.random.default_rng(2**31 + 4)
    M = oracle.nmodes(L)
    g = rng.standard_normal((1, M)) + 1j * rng.standard_normal((1, M))
    plan = ops.get_plan(L, dev)
    (gw,) = ops.alm_backward_raw(plan, [cat], 1, "fp64", torch.from_numpy(g).to(dev))
    torch.cuda.synchronize()
    plan.check()
    idx = np.concatenate([rng.integers(0, n, 200_000), np.arange(2**31 - 1000, 2**31 + 1000),
                          np.arange(n - 1000, n)]).astype(np.int64)
    got = gw[torch.from_numpy(idx).to(dev)].cpu().numpy()
    r = oracle.adjoint(x, phi, g[0], L)[idx % npat]
    assert np.max(np.abs(got - r)) <= 1e-11 * np.max(np.abs(r))
    del cat, gw
    torch.cuda.empty_cache()


def test_adjoint_and_spin2_at_fp32_max_lmax(dev):
    """lmax 4096 through the FP32 adjoint (1 500 points, random cotangent)
    and the spin-2 transform (800 points) against the oracle.  The FP32
    recurrence carries ~l eps per value, so the bounds are those of lmax
    4096: 3e-4 of the largest gradient, 1e-4 per multipole row of E and B."""
    L = 4096
    x, phi, w = _points(1500, 4099)
    rng = np.random.default_rng(4100)
    M = oracle.nmodes(L)
    g = rng.standard_normal((1, M)) + 1j * rng.standard_normal((1, M))
    plan = ops.get_plan(L, dev)
    (gw,) = ops.alm_backward_raw(plan, [_cat(dev, x, phi, w)], 1, "fp32", torch.from_numpy(g).to(dev))
    torch.cuda.synchronize()
    plan.check()
    r = oracle.adjoint(x.astype(np.float64), phi.astype(np.float64), g[0], L)
    err = np.max(np.abs(gw.double().cpu().numpy() - r)) / np.max(np.abs(r))
    print(f"adjoint lmax {L}: {err:.2e}")
    assert err <= 3e-4
    n = 800
    xs, ps = rng.uniform(-1, 1, n), rng.uniform(0, 2 * np.pi, n)
    ws, g1, g2 = rng.uniform(0.5, 1.5, n), 0.3 * rng.standard_normal(n), 0.3 * rng.standard_normal(n)
    arrs = [v.astype(np.float32) for v in (xs, ps, ws, g1, g2)]
    cat = ops.ShearCat(*(torch.from_numpy(a).to(dev) for a in arrs), 0, 1.0)
    E, B = ops.alm_spin2(plan, [cat], 1)
    torch.cuda.synchronize()
    plan.check()
    Er, Br = oracle.alm_spin2(*(a.astype(np.float64) for a in arrs), L)
    lidx = np.concatenate([np.arange(m, L + 1) for m in range(L + 1)])  # l of each packed mode
    for name, got, ref in (("E", E.cpu().numpy()[0], Er), ("B", B.cpu().numpy()[0], Br)):
        num = np.bincount(lidx, np.abs(got - ref) ** 2, L + 1)
        den = np.bincount(lidx, np.abs(ref) ** 2, L + 1)
        worst = float(np.sqrt(np.max(num[2:] / den[2:])))
        print(f"spin-2 {name} lmax {L}: {worst:.2e}")
        assert worst <= 1e-4
