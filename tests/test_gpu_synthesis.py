"""Point-evaluation synthesis (pointsht_synthesis) and the golden-spiral
workload (Sec. "Golden spiral") on the GPU, against the oracle.

Synthesis runs the adjoint kernels with unit weights and table factor c_m
(1 at m = 0, 2 above), so its FP32 tolerance is the adjoint's: 2e-5 of the
largest value for moderate lmax."""
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


def _real_field_alm(L, seed, slope=1.0):
    rng = np.random.default_rng(seed)
    M = oracle.nmodes(L)
    a = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    ls = np.concatenate([np.arange(m, L + 1) for m in range(L + 1)])
    a /= (1.0 + ls) ** slope
    for l in range(L + 1):
        a[oracle.index(l, 0, L)] = a[oracle.index(l, 0, L)].real
    return a


def _rms(a, L):
    """RMS of the field over the sphere (Parseval: mean f^2 = sum_{l,|m|} |a_lm|^2 / 4pi):
    the error scale for a handful of points, where the value itself may
    cancel far below it (one point at the pole sums only the m = 0 terms)."""
    cm = np.concatenate([np.full(L - m + 1, 1.0 if m == 0 else 2.0) for m in range(L + 1)])
    return float(np.sqrt(np.sum(cm * np.abs(a) ** 2) / (4 * np.pi)))


def _synth(dev, x, phi, a, L, prec):
    dt = np.float64 if prec == "fp64" else np.float32
    plan = ops.get_plan(L, dev)
    out = ops.synthesis(plan, torch.from_numpy(x.astype(dt)).to(dev), torch.from_numpy(phi.astype(dt)).to(dev),
                        torch.from_numpy(a).to(dev), prec)
    torch.cuda.synchronize()
    plan.check()
    return out.double().cpu().numpy()


@pytest.mark.parametrize("prec,L,n,tol", [("fp64", 48, 1000, 1e-11), ("fp32", 300, 3001, 2e-5),
                                          ("fp32", 64, 1, 2e-5), ("fp32", 64, 257, 2e-5), ("fp64", 31, 5, 1e-11)])
def test_synthesis_matches_oracle(dev, prec, L, n, tol):
    dt = np.float64 if prec == "fp64" else np.float32
    rng = np.random.default_rng(L + n)
    x = rng.uniform(-1, 1, n)
    x[: min(n, 2)] = [1.0, -1.0][: min(n, 2)]
    phi = rng.uniform(0, 2 * np.pi, n)
    a = _real_field_alm(L, n)
    got = _synth(dev, x, phi, a, L, prec)
    ref = oracle.synthesis(x.astype(dt).astype(np.float64), phi.astype(dt).astype(np.float64), a, L)
    assert np.max(np.abs(got - ref)) <= tol * max(np.max(np.abs(ref)), _rms(a, L))


def test_synthesis_empty_and_errors(dev):
    plan = ops.get_plan(16, dev)
    e = torch.empty(0, dtype=torch.float32, device=dev)
    a = torch.zeros(plan.nmodes, dtype=torch.complex128, device=dev)
    assert ops.synthesis(plan, e, e, a, "fp32").numel() == 0
    lib = _lib.load()
    assert lib.pointsht_workspace_size_synthesis(plan.handle, -1, _lib.PRECISIONS["fp32"]) == 0
    assert lib.pointsht_workspace_size_synthesis(plan.handle, 10, _lib.PRECISIONS["mixed"]) == 0
    with pytest.raises(ValueError):
        ops.synthesis(plan, e, e, torch.zeros(3, dtype=torch.complex128, device=dev), "fp32")


def test_synthesis_out_of_range_flagged(dev):
    plan = ops.get_plan(8, dev)
    x = torch.tensor([0.5, 1.5], dtype=torch.float32, device=dev)
    phi = torch.tensor([0.1, 0.2], dtype=torch.float32, device=dev)
    a = torch.zeros(plan.nmodes, dtype=torch.complex128, device=dev)
    ops.synthesis(plan, x, phi, a, "fp32")
    torch.cuda.synchronize()
    with pytest.raises(_lib.PointSHTError) as ei:
        plan.check()
    assert ei.value.status == _lib.ERANGE


# ------------------------------------------------------ golden spiral --
# The spiral's spectrum is blue: at low l, and on every odd l + m (the point
# set is symmetric in x up to the jitter), its a_lm are many orders of
# magnitude below the Poisson level sqrt(N / 4pi) that sets the size of the
# FP32 path's rounding (each point's term is rounded at ~1e-7 of its own size,
# and the N terms of a mode add those errors like a random walk).  FP32 is
# therefore held to 1e-5 relative plus DELTA32 x the Poisson scale; FP64 to
# 1e-10 relative (the FP64 target).
DELTA32 = 2e-6


@pytest.fixture(scope="module")
def spiral(dev):
    wl = catalogs.config(6)
    assert wl.npoints == 163_840 and wl.lmax == 2048
    c = wl.catalogs[0]
    plan = ops.get_plan(wl.lmax, dev)
    out = {}
    for prec, dt in (("fp32", torch.float32), ("fp64", torch.float64)):
        cat = ops.Cat(*(torch.from_numpy(v).to(dev).to(dt) for v in (c.x, c.phi, c.w)), 0, 1.0)
        out[prec] = ops.alm_raw(plan, [cat], 1, prec)
    torch.cuda.synchronize()
    plan.check()
    return wl, plan, out


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_golden_spiral_sampled_columns(spiral, prec):
    """The spiral's a_lm at lmax 2048 on the columns m = 0, 1, 700, 2047,
    2048 against the oracle over all 163 840 points."""
    wl, _, a = spiral
    L = wl.lmax
    c = wl.catalogs[0]
    got = a[prec].cpu().numpy()[0]
    ms = [0, 1, 700, 2047, 2048]
    ref = oracle.alm(c.x.astype(np.float64), c.phi.astype(np.float64), c.w.astype(np.float64), L, mlist=ms)
    shot = c.n / (4 * np.pi)
    for m, col in ref.items():
        g = got[oracle.index(m, m, L):oracle.index(L, m, L) + 1]
        if prec == "fp64":
            tol = 1e-10 * np.linalg.norm(col)
        else:
            tol = 1e-5 * np.linalg.norm(col) + DELTA32 * np.sqrt((L - m + 1) * shot)
        assert np.linalg.norm(g - col) <= tol, m


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_golden_spiral_low_l_cl(spiral, prec):
    """C_l for l <= 48, where the spiral's power is far below shot noise and,
    at odd l, ~1e-10 of the even-l power."""
    wl, _, a = spiral
    L, Ls = wl.lmax, 48
    c = wl.catalogs[0]
    got = a[prec].cpu().numpy()[0]
    ref = oracle.alm(c.x.astype(np.float64), c.phi.astype(np.float64), c.w.astype(np.float64), Ls)
    sub = np.concatenate([got[oracle.index(m, m, L):oracle.index(Ls, m, L) + 1] for m in range(Ls + 1)])
    cg, cr = oracle.cl(sub, sub, Ls), oracle.cl(ref, ref, Ls)
    if prec == "fp64":
        assert np.max(np.abs(cg - cr) / cr) <= 1e-10
    else:
        shot = c.n / (4 * np.pi)
        assert np.all(np.abs(cg - cr) <= 1e-5 * cr + 2 * DELTA32 * np.sqrt(cr * shot) + DELTA32 ** 2 * shot)


def test_golden_spiral_synthesis_sampled_points(spiral, dev):
    """Synthesis of the spiral's own a_lm (lmax 2048) on all 163 840 points,
    checked at 48 sampled points against the oracle's synthesis of the same
    coefficients, and the duality sum_i w_i f(n_i) = sum_lm c_m Re(a conj(a))
    over all points (GPU against GPU: a property at full size)."""
    wl, plan, alm = spiral
    a = alm["fp32"]
    L = wl.lmax
    c = wl.catalogs[0]
    f = ops.synthesis(plan, torch.from_numpy(c.x).to(dev), torch.from_numpy(c.phi).to(dev), a[0], "fp32")
    torch.cuda.synchronize()
    plan.check()
    f = f.double().cpu().numpy()
    idx = np.sort(np.random.default_rng(3).choice(c.n, 48, replace=False))
    an = a[0].cpu().numpy()
    ref = oracle.synthesis(c.x[idx].astype(np.float64), c.phi[idx].astype(np.float64), an, L)
    assert np.max(np.abs(f[idx] - ref)) <= 1e-4 * np.max(np.abs(ref))
    cm = np.concatenate([np.full(L - m + 1, 1.0 if m == 0 else 2.0) for m in range(L + 1)])
    rhs = np.sum(cm * np.abs(an) ** 2)
    assert abs(np.sum(f) - rhs) <= 1e-5 * rhs
