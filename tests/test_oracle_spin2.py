"""Pins of the oracle's spin-2 (shear) transform.

* lambda^(n)_lm = sqrt((2l+1)/4pi) d^l_{m,n}(theta) against sympy's Wigner
  small-d (a library's closed form) for n = -2, 0, +2;
* n = 0 reduces to the scalar lambda_lm of App. A;
* _{2}Y_lm = sqrt((l-2)!/(l+2)!) eth eth Y_lm, with eth the spin-raising
  operator -(sin theta)^s [d/dtheta + (i/sin theta) d/dphi] (sin theta)^-s
  by finite differences of the scalar Y_lm: fixes the sign convention that
  ties the d-function form to the spin-raising one;
* orthonormality of _{2}Y_lm by Gauss-Legendre x Fourier quadrature;
* E/B: a shear field synthesised from E_lm alone (B = 0), analysed on a
  quadrature grid, gives back E and B = 0; and from B alone gives back B and
  E = 0 (checks the E/B combination and the _{-2}Y branch);
* high m: the column for m = 2048 near the pole against the same column in
  long-double-free log space (values far below the FP64 range stay finite)."""
import numpy as np
import pytest

import oracle

FOUR_PI = 4.0 * np.pi


@pytest.mark.parametrize("n", [-2, 0, 2])
def test_against_sympy_small_d(n):
    sp = pytest.importorskip("sympy")
    from sympy.physics.quantum.spin import Rotation
    L = 6
    for th in (0.3, 1.1, 2.0, 2.9):
        x = np.cos(th)
        for m in range(L + 1):
            got = oracle.spin_lambda(x, L, m, n)
            for l in range(L + 1):
                if l < max(m, abs(n)):
                    assert got[l] == 0.0
                    continue
                d = complex(sp.N(Rotation.d(l, m, n, sp.Float(th, 30)).doit(), 30)).real
                ref = np.sqrt((2 * l + 1) / FOUR_PI) * d
                assert abs(got[l] - ref) <= 1e-13, (th, m, l, n)


def test_spin0_is_scalar_lambda():
    L = 80
    for x in (-0.97, -0.2, 0.4, 0.999):
        for m in (0, 1, 7, 40, 80):
            lam = oracle.pbar(x, L, m) * np.sqrt((2 * np.arange(m, L + 1) + 1) / FOUR_PI)
            got = oracle.spin_lambda(x, L, m, 0)[m:]
            assert np.max(np.abs(got - lam)) <= 1e-12 * max(1.0, np.max(np.abs(lam)))


def _ylm_theta(l, m, th):
    return oracle.ylm(np.cos(th), 0.0, l, m)[l - m].real  # Y_lm at phi = 0 (real for m >= 0)


def test_eth_eth_convention():
    """_{2}Y_lm(theta, 0) = sqrt((l-2)!/(l+2)!) (eth eth Y_lm)(theta, 0), with
    eth_s f = -(sin^s)(d/dtheta - m / sin)(sin^-s f) for f ~ e^{i m phi}
    ((i / sin) d/dphi gives -m / sin), by 4th-order central differences."""
    from math import factorial
    h = 1e-3

    def d1(f, t):
        return (-f(t + 2 * h) + 8 * f(t + h) - 8 * f(t - h) + f(t - 2 * h)) / (12 * h)

    for l in (2, 3, 5):
        for m in range(0, l + 1):
            for th in (0.6, 1.3, 2.2):
                def f0(t):
                    return _ylm_theta(l, m, t)

                def eth0(t):  # s = 0: -(d/dtheta - m / sin) Y
                    return -(d1(f0, t) - m / np.sin(t) * f0(t))

                # s = 1: -sin (d/dtheta - m / sin)(sin^-1 g)
                def g(t):
                    return eth0(t) / np.sin(t)

                eth1 = -np.sin(th) * (d1(g, th) - m / np.sin(th) * g(th))
                ref = np.sqrt(factorial(l - 2) / factorial(l + 2)) * eth1
                # _{2}Y_lm(theta, 0) = lambda^(-2)_lm (the conjugate of _{2}Y* at phi = 0)
                got = oracle.spin_lambda(np.cos(th), l, m, -2)[l]
                assert abs(got - ref) <= 1e-7, (l, m, th)


def _grid(n):
    x, wx = np.polynomial.legendre.leggauss(n)
    phi = np.arange(2 * n) * (np.pi / n)
    return x, wx, phi


def test_orthonormality_by_quadrature():
    L = 12
    n = 2 * L + 4
    x, wx, _ = _grid(n)
    for m in (0, 1, 3, 7):
        cols = np.array([oracle.spin_lambda(xi, L, m, -2) for xi in x])  # [node, l]
        G = 2 * np.pi * (cols * wx[:, None]).T @ cols  # int over phi of |e^{im phi}|^2 = 2 pi
        l0 = max(m, 2)
        assert np.max(np.abs(G[l0:, l0:] - np.eye(L + 1 - l0))) <= 1e-12


def _spin2_Y(L, x, phi):
    """_{2}Y_lm for -l <= m <= l at every grid point: dict (l, m) -> array."""
    out = {}
    for m in range(L + 1):
        lp = np.array([oracle.spin_lambda(xi, L, m, -2) for xi in x])  # _{2}Y_lm(theta, 0), m >= 0
        lq = np.array([oracle.spin_lambda(xi, L, m, 2) for xi in x])   # d^l_{m,2}
        for l in range(max(m, 2), L + 1):
            out[(l, m)] = lp[:, l][:, None] * np.exp(1j * m * phi)[None, :]
            if m > 0:
                # _{2}Y_{l,-m} = sqrt((2l+1)/4pi) d^l_{-m,-2} e^{-i m phi}, d^l_{-m,-2} = (-1)^m d^l_{m,2}
                out[(l, -m)] = (-1) ** m * lq[:, l][:, None] * np.exp(-1j * m * phi)[None, :]
    return out


@pytest.mark.parametrize("mode", ["E", "B"])
def test_pure_E_or_B_field_roundtrip(mode):
    """g1 + i g2 = -sum_{l,|m|} (E_lm + i B_lm) _{2}Y_lm on a quadrature grid
    (real-field coefficients: X_{l,-m} = (-1)^m conj(X_lm)); the weighted
    analysis (w = quadrature weight) must return E and B, the other one 0."""
    L = 6
    n = 2 * L + 6
    xg, wx, phig = _grid(n)
    Y = _spin2_Y(L, xg, phig)
    rng = np.random.default_rng(5 if mode == "E" else 6)
    X = {}
    for l in range(2, L + 1):
        X[(l, 0)] = rng.standard_normal()
        for m in range(1, l + 1):
            X[(l, m)] = rng.standard_normal() + 1j * rng.standard_normal()
            X[(l, -m)] = (-1) ** m * np.conj(X[(l, m)])
    field = np.zeros((n, 2 * n), np.complex128)
    for (l, m), c in X.items():
        coef = c if mode == "E" else 1j * c
        field -= coef * Y[(l, m)]
    g1, g2 = field.real, field.imag
    xx = np.repeat(xg, 2 * n)
    pp = np.tile(phig, n)
    ww = np.repeat(wx * (np.pi / n), 2 * n)
    E, B = oracle.alm_spin2(xx, pp, ww, g1.ravel(), g2.ravel(), L)
    want, zero = (E, B) if mode == "E" else (B, E)
    for l in range(L + 1):
        for m in range(0, l + 1):
            ref = X.get((l, m), 0.0) if l >= 2 else 0.0
            assert abs(want[oracle.index(l, m, L)] - ref) <= 1e-12, (l, m)
            assert abs(zero[oracle.index(l, m, L)]) <= 1e-12, (l, m)


def test_high_m_near_pole_stays_finite_and_matches_log_form():
    """m = l = 2048 at x = 0.99: the seed is ~2^-(m+2)*... far below the FP64
    range, carried by the exponent; the top-row value in log form must agree."""
    from math import lgamma, log
    L, m = 2048, 2048
    x = 0.99
    got = oracle.spin_lambda(x, L, m, -2)[L]
    th = np.arccos(x)
    logv = (0.5 * np.log((2 * L + 1) / FOUR_PI) + 0.5 * (lgamma(2 * L + 1) - lgamma(L - 1) - lgamma(L + 3))
            + (L - 2) * np.log(np.cos(th / 2)) + (L + 2) * np.log(np.sin(th / 2)))
    if logv < log(np.finfo(float).tiny):
        assert got == 0.0 or abs(got) < 1e-300
    else:
        assert abs(abs(got) / np.exp(logv) - 1.0) <= 1e-10
    mid = oracle.spin_lambda(0.3, L, 1500, -2)
    assert np.all(np.isfinite(mid)) and np.max(np.abs(mid)) > 0.1


def test_column_form_matches_full_transform():
    rng = np.random.default_rng(11)
    n, L = 500, 24
    x, phi = rng.uniform(-1, 1, n), rng.uniform(0, 2 * np.pi, n)
    w, g1, g2 = rng.uniform(0.5, 1.5, n), rng.standard_normal(n), rng.standard_normal(n)
    E, B = oracle.alm_spin2(x, phi, w, g1, g2, L)
    cols = oracle.alm_spin2_cols(x, phi, w, g1, g2, L, [0, 1, 5, 24])
    for m, (ec, bc) in cols.items():
        sl = slice(oracle.index(m, m, L), oracle.index(L, m, L) + 1)
        assert np.allclose(ec[m:], E[sl], rtol=1e-12, atol=1e-12)
        assert np.allclose(bc[m:], B[sl], rtol=1e-12, atol=1e-12)
