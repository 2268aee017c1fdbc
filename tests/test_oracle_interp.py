"""Pins of the oracle's interpolated transform (App. "Interpolation"), with
the samples equispaced in theta and continued across the poles.

Each pin is chosen so that a plausible mistake fails it: a wrong Hermite
basis function (cubic reproduction), a dropped or mis-scaled derivative term
(fourth-order convergence; exactness at the samples), a wrong ghost-sample
sign at the poles (pole and near-pole points), a misplaced interval
(points on the samples, monopole)."""
import numpy as np
import pytest

import oracle


def test_hermite_basis_reproduces_cubics():
    """S(t) = c0 p(0) + c1 h p'(0) + c2 p(h) + c3 h p'(h) equals p(t h) for every
    cubic p: the defining property of the cubic Hermite spline."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        a = rng.standard_normal(4)
        h = rng.uniform(0.01, 2.0)
        p = np.polynomial.Polynomial(a)
        dp = p.deriv()
        for t in np.linspace(0.0, 1.0, 11):
            c = oracle.hermite_basis(t)
            s = c[0] * p(0.0) + c[1] * h * dp(0.0) + c[2] * p(h) + c[3] * h * dp(h)
            assert abs(s - p(t * h)) <= 1e-12 * (1 + abs(p(t * h)))


def test_basis_end_values():
    assert np.array_equal(oracle.hermite_basis(0.0), [1.0, 0.0, 0.0, 0.0])
    assert np.allclose(oracle.hermite_basis(1.0), [0.0, 0.0, 1.0, 0.0], atol=0)


def _points(n, seed, lo=-1.0, hi=1.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, n), rng.uniform(0, 2 * np.pi, n), rng.uniform(0.5, 1.5, n)


def test_points_on_the_samples_are_exact():
    """A point at a sample theta_k = (k + 1/2) pi / N gets y_lm(theta_k) itself."""
    L, N = 40, 160
    k = np.arange(0, N, 3)
    x = np.cos((k + 0.5) * np.pi / N)
    rng = np.random.default_rng(4)
    phi = rng.uniform(0, 2 * np.pi, x.size)
    w = rng.uniform(0.5, 1.5, x.size)
    a = oracle.alm_interp(x, phi, w, L, N)
    ref = oracle.alm(x, phi, w, L)
    assert np.max(np.abs(a - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_fourth_order_convergence():
    """The error of the interpolated a_lm against the exact transform falls as
    h^4: doubling the samples divides its RMS over all modes by ~16."""
    L = 48
    x, phi, w = _points(3000, 5)
    ref = oracle.alm(x, phi, w, L)
    errs = [np.sqrt(np.mean(np.abs(oracle.alm_interp(x, phi, w, L, f * L) - ref) ** 2)) for f in (8, 16, 32)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13.0 < r1 < 19.0 and 13.0 < r2 < 19.0, (errs, r1, r2)
    assert oracle.rel_err_per_l(oracle.alm_interp(x, phi, w, L, 16 * L), ref, L) <= 5e-6


@pytest.mark.parametrize("xs", [[1.0], [-1.0], [1.0 - 1e-9, -1.0 + 1e-7], [0.9999, -0.99995]])
def test_pole_and_near_pole_points(xs):
    """Points at or next to the poles interpolate across the ghost samples;
    a wrong continuation sign would make odd or even m wrong by O(1)."""
    L, N = 32, 32 * 16
    x = np.asarray(xs, np.float64)
    phi = np.linspace(0.3, 2.0, x.size)
    w = np.full(x.size, 1.25)
    a = oracle.alm_interp(x, phi, w, L, N)
    ref = oracle.alm(x, phi, w, L)
    scale = 1.25 * x.size * np.sqrt((2 * L + 1) / (4 * np.pi))
    assert np.max(np.abs(a - ref)) <= 2e-6 * scale


def test_monopole_is_exact():
    """y_00 is constant (derivative 0), which the spline reproduces exactly:
    a_00 = sum w / sqrt(4 pi) for any N."""
    x, phi, w = _points(2000, 6)
    for N in (7, 64):
        a = oracle.alm_interp(x, phi, w, 8, N)
        assert abs(a[0] - np.sum(w) / np.sqrt(4 * np.pi)) <= 1e-12 * np.sum(w)


def test_order_coupled_derivative_identity():
    """The GPU's interpolated route takes dlambda_lm/dtheta in the order-coupled
    form 1/2 [sqrt((l-m)(l+m+1)) lambda_{l,m+1} - sqrt((l+m)(l-m+1)) lambda_{l,m-1}]
    (lambda_{l,-1} = -lambda_{l,1}); pin it against App. A's derivative
    [l x Pbar_l - (l+m) sqrt((l-m)/(l+m)) Pbar_{l-1}] / sin(theta) (times the
    normalisation), with the oracle's Pbar."""
    L = 40

    def lam(x, m):
        return oracle.pbar(x, L, m) * np.sqrt((2 * np.arange(m, L + 1) + 1) / (4 * np.pi))

    for th in (1e-2, 0.05, 0.7, 1.3, 2.9, np.pi - 1e-2):
        x, s = np.cos(th), np.sin(th)
        cols = [lam(x, m) for m in range(L + 1)]
        for m in range(L + 1):
            l = np.arange(m, L + 1)
            pb = oracle.pbar(x, L, m)
            prev = np.concatenate([[0.0], pb[:-1]])
            coef = (l + m) * np.sqrt(np.where(l > m, (l - m) / np.maximum(l + m, 1), 0.0))
            d_paper = np.sqrt((2 * l + 1) / (4 * np.pi)) * (l * x * pb - coef * prev) / s
            up = np.zeros_like(cols[m])
            if m + 1 <= L:
                up[1:] = cols[m + 1]
            dn = cols[m - 1][1:] if m >= 1 else -np.concatenate([[0.0], cols[1]])
            d_id = 0.5 * (np.sqrt((l - m) * (l + m + 1)) * up - np.sqrt((l + m) * (l - m + 1)) * dn)
            assert np.max(np.abs(d_id - d_paper)) <= 1e-11 * max(1.0, np.max(np.abs(d_paper)))
