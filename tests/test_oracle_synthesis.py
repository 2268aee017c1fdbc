"""Pins of the oracle's point-evaluation synthesis f(n) = sum_{l,|m|<=l} a_lm Y_lm(n)
of a real field from its m >= 0 coefficients: textbook closed forms, scipy's
Y_lm with explicit negative orders, the addition theorem (scipy's Legendre
polynomials), a vanishing imaginary part, and duality with the analysis
(Eq. alm_def): sum_i w_i f(n_i) = sum_lm b_lm conj(a_lm)."""
import numpy as np
import pytest

import oracle

FOUR_PI = 4.0 * np.pi


def _points(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, n)
    x[:2] = [1.0, -1.0]
    return x, rng.uniform(0, 2 * np.pi, n)


def _real_field_alm(L, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(oracle.nmodes(L)) + 1j * rng.standard_normal(oracle.nmodes(L))
    for l in range(L + 1):
        a[oracle.index(l, 0, L)] = a[oracle.index(l, 0, L)].real  # a_l0 real for a real field
    return a


def test_closed_forms_low_l():
    x, phi = _points(50, 1)
    s = np.sqrt((1 - x) * (1 + x))
    L = 1
    a = np.zeros(oracle.nmodes(L), np.complex128)
    a[oracle.index(0, 0, L)] = 0.7
    assert np.allclose(oracle.synthesis(x, phi, a, L), 0.7 / np.sqrt(FOUR_PI), rtol=1e-15, atol=0)
    a[:] = 0
    a[oracle.index(1, 0, L)] = -1.3
    assert np.allclose(oracle.synthesis(x, phi, a, L), -1.3 * np.sqrt(3 / FOUR_PI) * x, rtol=1e-14, atol=1e-16)
    a[:] = 0
    c = 0.4 - 0.9j
    a[oracle.index(1, 1, L)] = c
    y11 = -np.sqrt(3 / (8 * np.pi)) * s * np.exp(1j * phi)
    assert np.allclose(oracle.synthesis(x, phi, a, L), 2 * (c * y11).real, rtol=1e-13, atol=1e-15)


def test_against_scipy_with_negative_orders():
    sp = pytest.importorskip("scipy.special")
    L = 12
    a = _real_field_alm(L, 2)
    x, phi = _points(40, 3)
    th = np.arccos(x)
    ref = np.zeros(x.size, np.complex128)
    for l in range(L + 1):
        for m in range(-l, l + 1):
            alm = a[oracle.index(l, abs(m), L)]
            if m < 0:
                alm = (-1) ** m * np.conj(alm)
            ref += alm * sp.sph_harm_y(l, m, th, phi)
    re, im = oracle.synthesis(x, phi, a, L, return_imag=True)
    assert np.max(np.abs(re - ref.real)) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(im)) <= 1e-12 * np.max(np.abs(ref))


def test_addition_theorem():
    """a_lm = conj(Y_lm(n0)) gives f(n) = sum_l (2l+1)/4pi P_l(n . n0)."""
    sp = pytest.importorskip("scipy.special")
    L = 40
    x0, phi0 = 0.3, 1.1
    a = np.zeros(oracle.nmodes(L), np.complex128)
    for m in range(L + 1):
        a[oracle.index(m, m, L):oracle.index(L, m, L) + 1] = np.conj(oracle.ylm(x0, phi0, L, m))
    x, phi = _points(30, 4)
    cosg = x * x0 + np.sqrt((1 - x * x) * (1 - x0 * x0)) * np.cos(phi - phi0)
    ref = sum((2 * l + 1) / FOUR_PI * sp.eval_legendre(l, cosg) for l in range(L + 1))
    assert np.max(np.abs(oracle.synthesis(x, phi, a, L) - ref)) <= 1e-12 * (L + 1) ** 2 / FOUR_PI


def test_duality_with_analysis():
    L = 24
    x, phi = _points(300, 5)
    w = np.random.default_rng(6).uniform(0.5, 1.5, x.size)
    b = _real_field_alm(L, 7)
    lhs = np.sum(w * oracle.synthesis(x, phi, b, L))
    a = oracle.alm(x, phi, w, L)
    cm = np.array([1.0 if m == 0 else 2.0 for m in range(L + 1) for _ in range(m, L + 1)])
    rhs = np.sum(cm * (b * np.conj(a)).real)
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(w)) * np.max(np.abs(b)) * L
