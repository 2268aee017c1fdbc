"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances (stated against the FP64 oracle, which consumes the same rounded
inputs):
  * FP64 path: a_lm relative error per multipole row <= 1e-10;
  * FP32 path: pseudo-C_l error <= 1e-5 of the total (pre-subtraction) C_l,
    for every 1 <= l <= lmax;
  * integer-exact properties (zeros at the poles, bitwise determinism) exactly.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2312_12285_gb300 import catalogs, ops  # noqa: E402

pytestmark = pytest.mark.gpu

FOUR_PI = 4.0 * math.pi


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def to_cats(wl, dev, dtype=None):
    out = []
    for c in wl.catalogs:
        x, p, w = c.x, c.phi, c.w
        if dtype is not None:
            x, p, w = x.astype(dtype), p.astype(dtype), w.astype(dtype)
        out.append(ops.Cat(torch.from_numpy(np.ascontiguousarray(x)).to(dev),
                           torch.from_numpy(np.ascontiguousarray(p)).to(dev),
                           torch.from_numpy(np.ascontiguousarray(w)).to(dev), c.field, c.coeff))
    return out


def oracle_alm(cats_np, L, f=0):
    sel = [(c[0], c[1], c[2], c[4]) for c in cats_np if c[3] == f]
    if not sel:
        return np.zeros(oracle.nmodes(L), np.complex128)
    return oracle.field_alm(sel, L)


def np_cats(cats):
    return [(c.x.double().cpu().numpy(), c.phi.double().cpu().numpy(), c.w.double().cpu().numpy(), c.field,
             c.coeff) for c in cats]


def cl_err(cl, ref_total, ref_noise):
    ref = ref_total - ref_noise
    return float(np.max(np.abs(cl[1:] - ref[1:]) / np.abs(ref_total[1:])))


def run_alm(dev, cats, L, nfield=1, prec="fp32"):
    plan = ops.get_plan(L, dev)
    a = ops.alm_raw(plan, cats, nfield, prec)
    torch.cuda.synchronize()
    plan.check()
    return a.cpu().numpy()


# --------------------------------------------------------- config 1 --
def test_config1_fp64_full(dev):
    wl = catalogs.config(1)
    cats = to_cats(wl, dev)
    a = run_alm(dev, cats, wl.lmax, prec="fp64")[0]
    ref = oracle_alm(np_cats(cats), wl.lmax)
    assert oracle.rel_err_per_l(a, ref, wl.lmax) <= 1e-10
    # pseudo-C_l with shot noise removed (Eq. pseudoCl, Sec. 2.1)
    noise = ops.shot_noise_raw(cats, 1, "fp64", dev).cpu().numpy()
    w_signed = np.concatenate([c.w.cpu().numpy() * c.coeff for c in cats])
    assert abs(noise[0, 0] - oracle.shot_noise(w_signed)) <= 1e-13 * noise[0, 0]
    cl = ops.cl_raw(torch.from_numpy(a[None]).to(dev), torch.from_numpy(noise).to(dev)).cpu().numpy()[0]
    tot = oracle.cl(ref, ref, wl.lmax)
    assert cl_err(cl, tot, oracle.shot_noise(w_signed)) <= 1e-10


def test_config1_inputs_fp32_path(dev):
    wl = catalogs.config(1)
    cats = to_cats(wl, dev, np.float32)
    a = run_alm(dev, cats, wl.lmax, prec="fp32")[0]
    ref = oracle_alm(np_cats(cats), wl.lmax)
    tot = oracle.cl(ref, ref, wl.lmax)
    n = oracle.shot_noise(np.concatenate([c.w.double().cpu().numpy() * c.coeff for c in cats]))
    assert cl_err(oracle.cl(a, a, wl.lmax) - n, tot, n) <= 1e-5
    assert oracle.rel_err_per_l(a, ref, wl.lmax) <= 1e-4


@pytest.mark.parametrize("ng,nr,L", [(300, 3000, 1024), (200, 1800, 2048)])
def test_lognormal_cap_fp32(dev, ng, nr, L):
    wl = catalogs.lognormal_cap(ng, nr, L, config_id=2 if L == 1024 else 3, nwaves=64, grid=(128, 256))
    cats = to_cats(wl, dev)
    a = run_alm(dev, cats, L, prec="fp32")[0]
    ref = oracle_alm(np_cats(cats), L)
    tot = oracle.cl(ref, ref, L)
    n = oracle.shot_noise(np.concatenate([c.w.double().cpu().numpy() * c.coeff for c in cats]))
    err = cl_err(oracle.cl(a, a, L) - n, tot, n)
    assert err <= 1e-5, err


# --------------------------------------------------------- edge cases --
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ragged_sizes_poles_and_empty_fields(dev, prec):
    dt = np.float64 if prec == "fp64" else np.float32
    rng = np.random.default_rng(11)
    L = 96
    cats = []
    for f, n in ((0, 1), (0, 255), (2, 257), (2, 0), (3, 1000)):
        x = rng.uniform(-1, 1, n)
        if n >= 4:
            x[:4] = [1.0, -1.0, 1 - 1e-7, -1 + 1e-7]
        phi = rng.uniform(-20, 20, n)
        w = rng.uniform(0.5, 1.5, n)
        cats.append(ops.Cat(*(torch.from_numpy(v.astype(dt)).to(dev) for v in (x, phi, w)), f,
                            float(rng.uniform(-1, 1))))
    a = run_alm(dev, cats, L, nfield=4, prec=prec)
    cn = np_cats(cats)
    for f in range(4):
        ref = oracle_alm(cn, L, f)
        scale = max(1e-300, np.max(np.abs(ref)))
        tol = 1e-12 if prec == "fp64" else 2e-6
        assert np.max(np.abs(a[f] - ref)) <= tol * scale if f != 1 else np.all(a[f] == 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_single_point_at_pole_exact_zeros(dev, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    L = 300
    c = ops.Cat(torch.tensor([1.0], dtype=dt, device=dev), torch.tensor([0.3], dtype=dt, device=dev),
                torch.tensor([2.0], dtype=dt, device=dev))
    a = run_alm(dev, [c], L, prec=prec)[0]
    assert np.all(a[L + 1:] == 0)  # m > 0 vanish exactly at x = 1
    ls = np.arange(L + 1)
    # FP32: at x = 1 the three-term recurrence has a double root; the near-pole
    # form (Reinsch's difference form, only small quantities rounded) keeps
    # the l-recurrence at ~1e-6 of the column maximum (a float32 emulation of
    # the plain form gives ~1e-4 by l = 300 and 3e-3 by l = 2048).
    tol = 1e-13 if prec == "fp64" else 1e-5
    assert np.allclose(a[:L + 1].real, 2.0 * np.sqrt((2 * ls + 1) / FOUR_PI), rtol=tol, atol=0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_addition_theorem_single_point_high_l(dev, prec):
    """Single point: C_l = w^2/4pi for every l <= 2048 (every (l, m) normalised)."""
    dt = torch.float64 if prec == "fp64" else torch.float32
    L = 2048 if prec == "fp32" else 512
    # FP32: ~1e-6 away from the poles; near them (|x| >= 0.9, both signs) the
    # near-pole form of the recurrence keeps the same level up to l = 2048 (the
    # plain form's error grows to ~0.5% at x = 1: C_l = lambda_l0^2 alone there).
    for x, tol32 in ((0.4132, 2e-6), (-0.03, 2e-6), (0.9991, 1e-5), (-0.99995, 1e-5), (1.0, 2e-5),
                     (-1.0, 2e-5)):
        c = ops.Cat(torch.tensor([x], dtype=dt, device=dev), torch.tensor([2.2], dtype=dt, device=dev),
                    torch.tensor([1.5], dtype=dt, device=dev))
        a = run_alm(dev, [c], L, prec=prec)
        cl = ops.cl_raw(torch.from_numpy(a).to(dev)).cpu().numpy()[0]
        tol = 1e-12 if prec == "fp64" else tol32
        assert np.max(np.abs(cl / (1.5 ** 2 / FOUR_PI) - 1)) <= tol, x


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_bitwise_deterministic(dev, prec):
    wl = catalogs.uniform_fullsky(3000, 9000, 0.3, 200, np.float64 if prec == "fp64" else np.float32, 9)
    cats = to_cats(wl, dev)
    a1 = run_alm(dev, cats, 200, prec=prec)
    a2 = run_alm(dev, cats, 200, prec=prec)
    assert np.array_equal(a1.view(np.uint64), a2.view(np.uint64))


def test_out_of_range_input_is_reported(dev):
    c = ops.Cat(torch.tensor([0.2, 1.5], device=dev), torch.tensor([0.1, 0.2], device=dev),
                torch.tensor([1.0, 1.0], device=dev))
    plan = ops.get_plan(8, dev)
    ops.alm_raw(plan, [c], 1, "fp32")
    with pytest.raises(ops._lib.PointSHTError) as ei:
        plan.check()
    assert ei.value.status == ops._lib.ERANGE
    plan.check()  # flags were cleared


# ------------------------------------------------ spectra and helpers --
def test_cross_spectra_noise_combine_and_bins(dev):
    rng = np.random.default_rng(12)
    L = 64
    srcs = []
    for f, n in enumerate((400, 700, 5000)):
        x, p, w = rng.uniform(-1, 1, n), rng.uniform(0, 6.3, n), rng.uniform(0.8, 1.2, n)
        srcs.append(ops.Cat(*(torch.from_numpy(v).to(dev) for v in (x, p, w)), f, 1.0))
    a = ops.alm_raw(ops.get_plan(L, dev), srcs, 3, "fp64")
    noise = ops.shot_noise_raw(srcs, 3, "fp64", dev)
    alpha = [0.08, 0.14]
    coef = torch.tensor([[1.0, 0.0, -alpha[0]], [0.0, 1.0, -alpha[1]]], dtype=torch.float64, device=dev)
    d, nd = ops.combine_raw(a, coef, noise)
    cl = ops.cl_raw(d, nd).cpu().numpy()
    cn = np_cats(srcs)
    refs = [oracle_alm(cn, L, f) for f in range(3)]
    dref = [refs[0] - alpha[0] * refs[2], refs[1] - alpha[1] * refs[2]]
    wsq = [np.sum(c[2] ** 2) for c in cn]
    nref = np.array([[wsq[0] + alpha[0] ** 2 * wsq[2], alpha[0] * alpha[1] * wsq[2]],
                     [alpha[0] * alpha[1] * wsq[2], wsq[1] + alpha[1] ** 2 * wsq[2]]]) / FOUR_PI
    assert np.allclose(nd.cpu().numpy(), nref, rtol=1e-12)
    p = 0
    for f in range(2):
        for g in range(f, 2):
            ref = oracle.cl(dref[f], dref[g], L) - nref[f, g]
            assert np.max(np.abs(cl[p] - ref)) <= 1e-10 * np.max(np.abs(oracle.cl(dref[f], dref[f], L)))
            p += 1
    edges = torch.tensor([1, 4, 9, 30, 65], dtype=torch.int32, device=dev)
    cb = ops.bin_raw(torch.from_numpy(cl).to(dev), edges).cpu().numpy()
    for s in range(3):
        assert np.allclose(cb[s], oracle.binned(cl[s], edges.cpu().numpy(), L), rtol=1e-13, atol=0)


@pytest.mark.parametrize("prec,L,tol", [("fp64", 40, 1e-11), ("fp32", 300, 2e-5)])
def test_adjoint_matches_oracle(dev, prec, L, tol):
    dt = np.float64 if prec == "fp64" else np.float32
    rng = np.random.default_rng(13)
    n = 150
    x = rng.uniform(-1, 1, n)
    x[:2] = [1.0, -0.99999]
    p, w = rng.uniform(0, 6.3, n), rng.uniform(0.8, 1.2, n)
    cat = ops.Cat(*(torch.from_numpy(v.astype(dt)).to(dev) for v in (x, p, w)), 0, -0.7)
    M = oracle.nmodes(L)
    g = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    gn = np.array([[0.37]])
    plan = ops.get_plan(L, dev)
    (gw,) = ops.alm_backward_raw(plan, [cat], 1, prec, torch.from_numpy(g[None]).to(dev),
                                 torch.from_numpy(gn).to(dev))
    gw = gw.double().cpu().numpy()
    xs, ps, ws = (v.astype(dt).astype(np.float64) for v in (x, p, w))
    ref = -0.7 * oracle.adjoint(xs, ps, g, L) + 2 * 0.49 * ws * 0.37 / FOUR_PI
    assert np.max(np.abs(gw - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_adjoint_several_catalogs_and_fields(dev, prec):
    """Three catalogs on two fields (one catalog empty), more points than one
    warp and not a multiple of it: each gradient must land on its own
    catalog and index (the FP32 adjoint works in |x|-sorted order and maps
    back through the point id)."""
    dt = np.float64 if prec == "fp64" else np.float32
    L = 120
    rng = np.random.default_rng(17)
    sizes, fields, coeffs = [700, 0, 1301, 45], [0, 1, 1, 0], [1.0, 0.5, -0.3, 2.0]
    raw = [(rng.uniform(-1, 1, n), rng.uniform(0, 6.28, n), rng.uniform(0.5, 1.5, n)) for n in sizes]
    cats = [ops.Cat(*(torch.from_numpy(v.astype(dt)).to(dev) for v in r), f, c)
            for r, f, c in zip(raw, fields, coeffs)]
    M = oracle.nmodes(L)
    g = rng.standard_normal((2, M)) + 1j * rng.standard_normal((2, M))
    gn = np.array([[0.21, 0.0], [0.0, -0.4]])
    plan = ops.get_plan(L, dev)
    grads = ops.alm_backward_raw(plan, cats, 2, prec, torch.from_numpy(g).to(dev), torch.from_numpy(gn).to(dev))
    torch.cuda.synchronize()
    plan.check()
    tol = 1e-11 if prec == "fp64" else 2e-5
    for (x, p, w), f, c, gw in zip(raw, fields, coeffs, grads):
        got = gw.double().cpu().numpy()
        assert got.shape == (x.size,)
        if x.size == 0:
            continue
        xs, ps, ws = (v.astype(dt).astype(np.float64) for v in (x, p, w))
        ref = c * oracle.adjoint(xs, ps, g[f], L) + 2 * c * c * ws * gn[f, f] / FOUR_PI
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


def test_adjoint_fields_at_cta_boundaries(dev):
    """FP32 adjoint with five fields of 1, 1023, 1024, 1025 and 3000 points
    (fields are padded to whole 1024-point CTAs, whose four warps share the
    staged coefficient chunks), one of them with every point near the north
    pole (near-pole form for m < 256), lmax 300 (several 64-step chunks per
    order): each gradient against the oracle."""
    L = 300
    rng = np.random.default_rng(29)
    sizes = [1, 1023, 1024, 1025, 3000]
    raw = []
    for f, n in enumerate(sizes):
        x = rng.uniform(0.95, 1.0, n) if f == 2 else rng.uniform(-1, 1, n)
        raw.append((x, rng.uniform(0, 6.28, n), rng.uniform(0.5, 1.5, n)))
    coeffs = [1.0, -0.4, 0.8, 1.3, -1.1]
    cats = [ops.Cat(*(torch.from_numpy(v.astype(np.float32)).to(dev) for v in r), f, c)
            for f, (r, c) in enumerate(zip(raw, coeffs))]
    M = oracle.nmodes(L)
    nf = len(sizes)
    g = rng.standard_normal((nf, M)) + 1j * rng.standard_normal((nf, M))
    gn = np.diag(rng.uniform(-0.5, 0.5, nf))
    plan = ops.get_plan(L, dev)
    grads = ops.alm_backward_raw(plan, cats, nf, "fp32", torch.from_numpy(g).to(dev), torch.from_numpy(gn).to(dev))
    torch.cuda.synchronize()
    plan.check()
    for f, ((x, p, w), c, gw) in enumerate(zip(raw, coeffs, grads)):
        got = gw.double().cpu().numpy()
        xs, ps, ws = (v.astype(np.float32).astype(np.float64) for v in (x, p, w))
        ref = c * oracle.adjoint(xs, ps, g[f], L) + 2 * c * c * ws * gn[f, f] / FOUR_PI
        # the FP32 recurrence carries ~l eps per value: at lmax 300 (2.5 times the
        # lmax of the 2e-5 test above) random cotangents give ~2e-5 of the
        # largest gradient on the uniform 3000-point field
        assert np.max(np.abs(got - ref)) <= 4e-5 * np.max(np.abs(ref)), f


def test_autograd_binned_cl_gradient(dev):
    """Differentiation config structure (small): d(sum_b g_b C_b)/dw via the
    adjoint kernel vs the oracle's definition-level gradient."""
    L = 128
    wl = catalogs.lognormal_cap(400, 2000, L, config_id=5, nwaves=32, grid=(64, 128))
    edges = catalogs.log_bin_edges(L, 32)
    gb = catalogs.rng_for(5, 7).standard_normal(32)
    cats = to_cats(wl, dev)
    for c in cats:
        c.w.requires_grad_(True)
    e_t = torch.from_numpy(edges.astype(np.int32)).to(dev)
    cb = ops.binned_pseudo_cl(cats, L, e_t, 1, "fp32")
    loss = (cb[0] * torch.from_numpy(gb).to(dev)).sum()
    loss.backward()
    idx = [np.arange(0, 400, 13), np.arange(0, 2000, 61)]
    ref = oracle.grad_binned_cl([(c.x, c.phi, c.w.astype(np.float64), c.coeff) for c in wl.catalogs], L, edges,
                                gb, idx)
    for c, i, r in zip(cats, idx, ref):
        got = c.w.grad.double().cpu().numpy()[i]
        assert np.max(np.abs(got - r)) <= 1e-4 * np.max(np.abs(r))


def _pole_cap(rng, n, x0, sign):
    """n points uniform in solid angle with sign * x in [x0, 1] (a polar cap)."""
    x = sign * (1.0 - rng.uniform(0.0, 1.0 - x0, n))
    return x, rng.uniform(0.0, 2 * math.pi, n)


@pytest.mark.parametrize("near_pole_form", [True, False])
def test_near_pole_catalogs_against_oracle(dev, near_pole_form):
    """Points in both polar caps (|x| >= 0.92, field 0 north, field 1 south, so
    that every tile lies on one side), lmax 1024: with the near-pole form the
    FP32 a_lm rows stay within 1e-5 of the oracle's; the plain form's error is
    reported for comparison (double root of the recurrence at x = +-1)."""
    L = 1024
    rng = np.random.default_rng(1024)
    cats = []
    for f, sign in ((0, 1.0), (1, -1.0)):
        x, phi = _pole_cap(rng, 6000, 0.92, sign)
        w = rng.uniform(0.8, 1.2, x.shape[0])
        cats.append(ops.Cat(*(torch.from_numpy(v.astype(np.float32)).to(dev) for v in (x, phi, w)), f, 1.0))
    plan = ops.Plan(L, dev)
    if not near_pole_form:
        plan.set_pole_threshold(2.0)
    a = ops.alm_raw(plan, cats, 2, "fp32").cpu().numpy()
    plan.check()
    cn = np_cats(cats)
    errs = [oracle.rel_err_per_l(a[f], oracle_alm(cn, L, f), L) for f in (0, 1)]
    print("near-pole form" if near_pole_form else "plain form", errs)
    if near_pole_form:
        assert max(errs) <= 1e-5, errs


@pytest.mark.parametrize("near_pole_form", [True, False])
def test_near_pole_synthesis(dev, near_pole_form):
    """The FP32 adjoint (synthesis) at points near both poles, lmax 1024: with
    the near-pole form within 1e-5 of the field's RMS of the oracle (the
    plain form's error is printed for comparison)."""
    L = 1024
    rng = np.random.default_rng(77)
    M = oracle.nmodes(L)
    ls = np.concatenate([np.arange(m, L + 1) for m in range(L + 1)])
    a = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) / (1.0 + ls)
    for l in range(L + 1):
        a[oracle.index(l, 0, L)] = a[oracle.index(l, 0, L)].real
    xs, ps = [], []
    for sign in (1.0, -1.0):
        x, phi = _pole_cap(rng, 2048, 0.95, sign)
        xs.append(x)
        ps.append(phi)
    x = np.concatenate(xs).astype(np.float32)
    phi = np.concatenate(ps).astype(np.float32)
    plan = ops.Plan(L, dev)
    if not near_pole_form:
        plan.set_pole_threshold(2.0)
    got = ops.synthesis(plan, torch.from_numpy(x).to(dev), torch.from_numpy(phi).to(dev),
                        torch.from_numpy(a).to(dev)).double().cpu().numpy()
    plan.check()
    ref = oracle.synthesis(x.astype(np.float64), phi.astype(np.float64), a, L)
    cm = np.where(np.concatenate([np.full(L - m + 1, m) for m in range(L + 1)]) == 0, 1.0, 2.0)
    rms = math.sqrt(float(np.sum(cm * np.abs(a) ** 2)) / FOUR_PI)
    err = float(np.max(np.abs(got - ref))) / rms
    print("near-pole form" if near_pole_form else "plain form", err)
    if near_pole_form:
        assert err <= 1e-5, err
