"""Pins of the FP64 oracle against things other than itself: textbook closed
forms, an independent library (scipy), arbitrary precision (mpmath, Rodrigues'
formula), Gauss-Legendre quadrature exactness, exact symmetries, the addition
theorem and brute-force finite differences.  CPU only."""
import math

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")
scipy_special = pytest.importorskip("scipy.special")

FOUR_PI = 4.0 * math.pi


# ------------------------------------------------------------ closed forms --
def _ylm_textbook(l, m, th, ph):
    s, c = math.sin(th), math.cos(th)
    e = complex(math.cos(m * ph), math.sin(m * ph))
    table = {
        (0, 0): 0.5 * math.sqrt(1 / math.pi),
        (1, 0): math.sqrt(3 / FOUR_PI) * c,
        (1, 1): -math.sqrt(3 / (8 * math.pi)) * s,
        (2, 0): math.sqrt(5 / (16 * math.pi)) * (3 * c * c - 1),
        (2, 1): -math.sqrt(15 / (8 * math.pi)) * s * c,
        (2, 2): 0.25 * math.sqrt(15 / (2 * math.pi)) * s * s,
    }
    return table[(l, m)] * e


def test_low_l_closed_forms(oracle_mod):
    rng = np.random.default_rng(0)
    for th, ph in zip(rng.uniform(0, math.pi, 7), rng.uniform(0, 2 * math.pi, 7)):
        for m in range(3):
            y = oracle_mod.ylm(math.cos(th), ph, 2, m)
            for l in range(m, 3):
                assert abs(y[l - m] - _ylm_textbook(l, m, th, ph)) < 1e-15


def test_matches_scipy_sph_harm_y(oracle_mod):
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.uniform(-1, 1, 6), [0.0, 0.999999, -0.999999, 1.0, -1.0]])
    L = 50
    for x in xs:
        ph = rng.uniform(0, 2 * math.pi)
        th = math.acos(x)
        for m in range(L + 1):
            ref = sph_harm_y(np.arange(m, L + 1), m, th, ph)
            got = oracle_mod.ylm(x, ph, L, m)
            assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) < 2e-14, (x, m)


def _pbar_rodrigues(l, m, x):
    """Pbar_l^m from Rodrigues' formula as an exact finite sum, in mpmath:
    P_l^m = (-1)^m/(2^l l!) (1-x^2)^{m/2} d^{l+m}/dx^{l+m} (x^2-1)^l."""
    with mpmath.workdps(int(1.5 * l) + 60):
        x = mpmath.mpf(x)
        s = mpmath.sqrt((1 - x) * (1 + x))
        tot = mpmath.mpf(0)
        for j in range((l + m + 1) // 2, l + 1):
            p = 2 * j - l - m
            tot += (mpmath.binomial(l, j) * (-1) ** (l - j) * mpmath.factorial(2 * j)
                    / mpmath.factorial(p) * x ** p)
        P = (-1) ** m / (mpmath.mpf(2) ** l * mpmath.factorial(l)) * s ** m * tot
        return +(mpmath.sqrt(mpmath.factorial(l - m) / mpmath.factorial(l + m)) * P)


@pytest.mark.parametrize("l,m,x,tol", [
    (2048, 2048, 0.9999, 1e-12),     # sectoral far below the FP64 range (exponent tracking)
    (2048, 2047, -0.999999, 1e-12),  # x < 0, 2^-19000
    (2000, 1990, 0.99, 1e-12),
    (2048, 1800, 0.95, 1e-12),
    (1024, 0, 0.77, 1e-12),
    (1500, 700, -0.62, 1e-12),
    (2048, 3, 0.999, 1e-11),
])
def test_high_degree_vs_arbitrary_precision(oracle_mod, l, m, x, tol):
    ref = _pbar_rodrigues(l, m, x)
    mant, expo = oracle_mod.pbar_scaled(x, l, m)
    got = mpmath.mpf(float(mant[-1])) * mpmath.mpf(2) ** int(expo[-1])
    assert abs(got / ref - 1) < tol


def test_normalisation_gauss_legendre(oracle_mod):
    """2 pi int lambda_lm(x)^2 dx = 1 (orthonormal Y_lm), exact with n > l GL nodes."""
    L = 160
    xg, wg = np.polynomial.legendre.leggauss(L + 2)
    for m in (0, 1, 7, 80, 159, 160):
        vals = np.array([oracle_mod.ylm(x, 0.0, L, m).real for x in xg])  # (n, L-m+1)
        norms = 2 * math.pi * (wg[:, None] * vals ** 2).sum(axis=0)
        assert np.max(np.abs(norms - 1.0)) < 1e-12, m
        if L - m >= 2:  # orthogonality between degrees at fixed m
            assert abs(2 * math.pi * np.sum(wg * vals[:, 0] * vals[:, 2])) < 1e-12


# --------------------------------------------------- whole transform (a_lm) --
def test_quadrature_exactness_recovers_band_limited_coefficients(oracle_mod):
    """Points on a Gauss-Legendre x Fourier grid, weighted by a band-limited
    field f = sum b_lm Y_lm (synthesised with scipy) times the quadrature
    weight: a_lm = sum_i w_i Y*_lm(n_i) = int f Y*_lm = b_lm exactly."""
    from scipy.special import sph_harm_y
    L = 20
    rng = np.random.default_rng(3)
    b = {}
    for l in range(L + 1):
        b[(l, 0)] = complex(rng.standard_normal(), 0.0)
        for m in range(1, l + 1):
            b[(l, m)] = complex(rng.standard_normal(), rng.standard_normal())
    xg, wg = np.polynomial.legendre.leggauss(L + 1)
    nphi = 2 * L + 2
    ph = np.arange(nphi) * 2 * math.pi / nphi
    X, PH = np.meshgrid(xg, ph, indexing="ij")
    W = np.repeat(wg, nphi).reshape(X.shape) * (2 * math.pi / nphi)
    th = np.arccos(X)
    f = np.zeros(X.shape)
    for (l, m), v in b.items():
        y = sph_harm_y(l, m, th, PH)
        # real field: b_{l,-m} = (-1)^m conj(b_lm), Y_{l,-m} = (-1)^m conj(Y_lm)
        f += (v * y).real if m == 0 else 2.0 * (v * y).real
    a = oracle_mod.alm(X.ravel(), PH.ravel(), (f * W).ravel(), L)
    for (l, m), v in b.items():
        assert abs(a[oracle_mod.index(l, m, L)] - v) < 1e-12


def test_full_vs_listed_orders(oracle_mod):
    rng = np.random.default_rng(4)
    n, L = 300, 40
    x, ph, w = rng.uniform(-1, 1, n), rng.uniform(0, 2 * math.pi, n), rng.uniform(0.5, 1.5, n)
    full = oracle_mod.alm(x, ph, w, L)
    cols = oracle_mod.alm(x, ph, w, L, mlist=[0, 13, 40])
    for m, c in cols.items():
        i0 = oracle_mod.index(m, m, L)
        assert np.array_equal(c, full[i0:i0 + L - m + 1])


def test_pole_points(oracle_mod):
    L = 300
    ls = np.arange(L + 1)
    for x, sign in ((1.0, 1.0), (-1.0, -1.0)):
        a = oracle_mod.alm([x], [0.7], [1.3], L)
        a0 = a[:L + 1]
        assert np.allclose(a0.real, 1.3 * np.sqrt((2 * ls + 1) / FOUR_PI) * sign ** ls, rtol=1e-13, atol=0)
        assert np.all(a0.imag == 0)
        assert np.all(a[L + 1:] == 0)  # m > 0 vanish at the poles


def test_mirror_rotation_monopole(oracle_mod):
    rng = np.random.default_rng(5)
    n, L = 500, 64
    x, ph, w = rng.uniform(-1, 1, n), rng.uniform(0, 2 * math.pi, n), rng.uniform(0.5, 1.5, n)
    a = oracle_mod.alm(x, ph, w, L)
    am = oracle_mod.alm(-x, ph, w, L)
    d = 0.37
    ar = oracle_mod.alm(x, ph + d, w, L)
    for m in range(L + 1):
        sl = slice(oracle_mod.index(m, m, L), oracle_mod.index(L, m, L) + 1)
        l = np.arange(m, L + 1)
        assert np.allclose(am[sl], (-1.0) ** (l + m) * a[sl], rtol=0, atol=1e-11)
        assert np.allclose(ar[sl], np.exp(-1j * m * d) * a[sl], rtol=0, atol=1e-11)
    assert abs(a[0] - np.sum(w) / math.sqrt(FOUR_PI)) < 1e-12


def test_addition_theorem_single_point_to_lmax_2048(oracle_mod):
    """Single point of weight w: C_l = w^2/4pi at every l (P_l(1) = 1), i.e.
    zero after shot-noise subtraction; pins the normalisation of every (l, m)."""
    L = 2048
    w = 1.7
    a = oracle_mod.alm([0.4132], [2.2], [w], L)
    c = oracle_mod.cl(a, a, L)
    assert np.max(np.abs(c / (w * w / FOUR_PI) - 1)) < 1e-11
    assert np.max(np.abs(c - oracle_mod.shot_noise([w]))) < 1e-11 * w * w / FOUR_PI


def test_cross_noise_of_fields_sharing_randoms(oracle_mod):
    """Fields a = D_a - alpha_a R and b = D_b - alpha_b R with distinct data
    points but one random catalog R (Sec. 2.1, cross-spectra of tracers
    sharing randoms): the only coincident (i = j) pairs of the cross-spectrum
    are R's, so its noise is alpha_a alpha_b sum w_R^2 / 4pi, the off-diagonal
    entry of the noise matrix the GPU test compares with.  With R alone (no
    data) the cross-spectrum is exactly that at every l (addition theorem);
    a wrong sign, a missing alpha or a data term in the cross entry fails."""
    L = 300
    xr, pr, wr = np.array([0.21, 0.21]), np.array([1.1, 1.1]), np.array([0.8, 1.3])  # coincident randoms
    al_a, al_b = 0.08, 0.14
    ra = oracle_mod.alm(xr, pr, -al_a * wr, L)
    rb = oracle_mod.alm(xr, pr, -al_b * wr, L)
    cross = oracle_mod.cl(ra, rb, L)
    n_ab = al_a * al_b * np.sum(wr) ** 2 / FOUR_PI  # two coincident points: (sum w)^2
    assert np.max(np.abs(cross / n_ab - 1)) < 1e-12
    # one random point: the noise-matrix entry alpha_a alpha_b w^2 / 4pi itself
    r1a = oracle_mod.alm(xr[:1], pr[:1], -al_a * wr[:1], L)
    r1b = oracle_mod.alm(xr[:1], pr[:1], -al_b * wr[:1], L)
    assert np.max(np.abs(oracle_mod.cl(r1a, r1b, L) - al_a * al_b * wr[0] ** 2 / FOUR_PI)) < 1e-13
    # distinct data points in each field add no flat term to the cross-spectrum:
    # its mean over l matches the noise entry only through R (random data positions)
    rng = np.random.default_rng(5)
    n = 4000
    xa, pa = rng.uniform(-1, 1, n), rng.uniform(0, 2 * np.pi, n)
    xb, pb = rng.uniform(-1, 1, n), rng.uniform(0, 2 * np.pi, n)
    xs, ps = rng.uniform(-1, 1, 3 * n), rng.uniform(0, 2 * np.pi, 3 * n)
    ws = rng.uniform(0.8, 1.2, 3 * n)
    fa = oracle_mod.field_alm([(xa, pa, np.ones(n), 1.0), (xs, ps, ws, -al_a)], 64)
    fb = oracle_mod.field_alm([(xb, pb, np.ones(n), 1.0), (xs, ps, ws, -al_b)], 64)
    mean_cross = np.mean(oracle_mod.cl(fa, fb, 64)[1:])
    n_ab = al_a * al_b * np.sum(ws * ws) / FOUR_PI
    n_aa = (n + al_a ** 2 * np.sum(ws * ws)) / FOUR_PI
    assert abs(mean_cross - n_ab) < 0.1 * n_aa  # unclustered: cross power is the shared noise, up to scatter


def test_coincident_points(oracle_mod):
    L, n, w = 200, 5, 0.9
    a = oracle_mod.alm(np.full(n, -0.3), np.full(n, 4.0), np.full(n, w), L)
    c = oracle_mod.cl(a, a, L)
    assert np.max(np.abs(c / (n * n * w * w / FOUR_PI) - 1)) < 1e-12


def test_cross_spectrum_symmetry_and_auto(oracle_mod):
    rng = np.random.default_rng(6)
    L = 30
    a = oracle_mod.alm(rng.uniform(-1, 1, 50), rng.uniform(0, 6, 50), np.ones(50), L)
    b = oracle_mod.alm(rng.uniform(-1, 1, 70), rng.uniform(0, 6, 70), np.ones(70), L)
    assert np.allclose(oracle_mod.cl(a, b, L), oracle_mod.cl(b, a, L), rtol=1e-14, atol=1e-14)
    # |a+b|^2 = |a|^2 + |b|^2 + 2 Re(a b*)
    lhs = oracle_mod.cl(a + b, a + b, L)
    rhs = oracle_mod.cl(a, a, L) + oracle_mod.cl(b, b, L) + 2 * oracle_mod.cl(a, b, L)
    assert np.allclose(lhs, rhs, rtol=1e-12)


def test_adjoint_dot_product(oracle_mod):
    """<g, A w> = <A^T g, w> for the linear map w -> a_lm."""
    rng = np.random.default_rng(7)
    n, L = 40, 24
    x, ph, w = rng.uniform(-1, 1, n), rng.uniform(0, 2 * math.pi, n), rng.standard_normal(n)
    g = rng.standard_normal(oracle_mod.nmodes(L)) + 1j * rng.standard_normal(oracle_mod.nmodes(L))
    a = oracle_mod.alm(x, ph, w, L)
    lhs = np.sum((np.conj(g) * a).real)
    rhs = np.dot(oracle_mod.adjoint(x, ph, g, L), w)
    assert abs(lhs - rhs) < 1e-10 * (abs(lhs) + 1)


def test_binning_matrix(oracle_mod):
    L = 100
    e = np.array([2, 5, 9, 30, 101])
    th = oracle_mod.bin_matrix(e, L)
    assert np.allclose(th.sum(axis=1), 1.0)
    assert np.allclose(oracle_mod.binned(np.full(L + 1, 3.5), e, L), 3.5)


def test_gradient_vs_full_recompute_finite_differences(oracle_mod):
    """dL/dw_i for L = sum_b g_b C_b (shot noise removed) against central
    differences of the whole pipeline recomputed from scratch."""
    rng = np.random.default_rng(8)
    L = 32
    xg, pg = rng.uniform(-1, 1, 120), rng.uniform(0, 2 * math.pi, 120)
    xr, pr = rng.uniform(-1, 1, 200), rng.uniform(0, 2 * math.pi, 200)
    wg, wr = rng.uniform(0.8, 1.2, 120), rng.uniform(0.8, 1.2, 200)
    alpha = 0.55
    edges = np.array([2, 4, 8, 16, 33])
    gb = rng.standard_normal(4)

    def loss(wg_, wr_):
        cats = [(xg, pg, wg_, 1.0), (xr, pr, wr_, -alpha)]
        a = oracle_mod.field_alm(cats, L)
        n = oracle_mod.shot_noise(np.concatenate([wg_, -alpha * wr_]))
        return float(np.dot(gb, oracle_mod.binned(oracle_mod.cl(a, a, L) - n, edges, L)))

    idx = [np.array([0, 17, 119]), np.array([3, 150])]
    grads = oracle_mod.grad_binned_cl([(xg, pg, wg, 1.0), (xr, pr, wr, -alpha)], L, edges, gb, idx)
    for ci, (ws, gr) in enumerate(zip((wg, wr), grads)):
        for k, i in enumerate(idx[ci]):
            h = 1e-4
            wp, wm = ws.copy(), ws.copy()
            wp[i] += h
            wm[i] -= h
            if ci == 0:
                fd = (loss(wp, wr) - loss(wm, wr)) / (2 * h)
            else:
                fd = (loss(wg, wp) - loss(wg, wm)) / (2 * h)
            assert abs(fd - gr[k]) < 1e-6 * (abs(fd) + 1e-3), (ci, i, fd, gr[k])


def test_single_point_gradient_closed_form(oracle_mod):
    """One point of weight w: C_l = w^2/4pi so dC_l/dw = 2w/4pi before the
    shot-noise subtraction and 0 after it."""
    L = 40
    w = 1.3
    edges = np.array([1, 10, 41])
    gb = np.array([0.7, -1.1])
    (g,) = oracle_mod.grad_binned_cl([([0.2], [1.0], [w], 1.0)], L, edges, gb, [np.array([0])])
    assert abs(g[0]) < 1e-12


def test_gradient_euler_identity(oracle_mod):
    """L = sum_b g_b C_b is homogeneous of degree 2 in the weights (a_lm is
    linear in them, C_l and the shot noise quadratic), so the oracle gradient
    over every object obeys sum_i w_i dL/dw_i = 2 L exactly: a whole-sum check
    that a dropped factor 2, a wrong c_m = 2 weight for m > 0 or a wrong sign
    of the noise term fails (the identity the full-size GPU gradient is also
    held to)."""
    L = 48
    rng = np.random.default_rng(31)
    xg, pg, wg = rng.uniform(-1, 1, 300), rng.uniform(0, 2 * math.pi, 300), rng.uniform(0.8, 1.2, 300)
    xr, pr, wr = rng.uniform(-1, 1, 900), rng.uniform(0, 2 * math.pi, 900), rng.uniform(0.8, 1.2, 900)
    alpha = 0.31
    edges = np.array([1, 3, 7, 15, 31, 49])
    gb = rng.standard_normal(5)
    cats = [(xg, pg, wg, 1.0), (xr, pr, wr, -alpha)]
    a = oracle_mod.field_alm(cats, L)
    n = oracle_mod.shot_noise(np.concatenate([wg, -alpha * wr]))
    cb = oracle_mod.binned(oracle_mod.cl(a, a, L) - n, edges, L)
    loss = float(np.dot(gb, cb))
    gg, gr = oracle_mod.grad_binned_cl(cats, L, edges, gb, [np.arange(300), np.arange(900)])
    s = float(np.dot(wg, gg) + np.dot(wr, gr))
    scale = float(np.dot(np.abs(gb), np.abs(oracle_mod.binned(oracle_mod.cl(a, a, L), edges, L))))
    assert abs(s - 2.0 * loss) <= 1e-12 * scale
