"""Pins of the oracle's mode-coupling matrix (Eq. chat), its 3j symbols with
zero orders (App. "Wigner 3j symbols"), the binned coupling, the decoupling
(Eq. mode_coupling, Eq. expectation_value) and the FKP-like normalisation.

Each pin is independent of the oracle's own closed form and chosen so that a
plausible mistake fails it: exact rational 3j values from a library (sign,
parity, factorial placement), the paper's recurrence and terminal case, the
3j orthogonality sum, M = I on the full sky (prefactor 2l'+1 and 1/4pi), row
sums against the Parseval identity, and M itself against the ensemble average
of a masked field computed by quadrature of products of library Y_lm (the
derivation behind Eq. chat, done numerically)."""
import numpy as np
import pytest

import oracle

FOUR_PI = 4.0 * np.pi


@pytest.mark.parametrize("l1,l2,l3", [(0, 0, 0), (1, 1, 0), (1, 1, 2), (2, 2, 2), (3, 2, 1), (4, 6, 8),
                                      (5, 7, 4), (10, 7, 5), (12, 12, 12), (9, 4, 5), (3, 3, 1), (6, 2, 3)])
def test_threej_exact_values(l1, l2, l3):
    """Against sympy's exact Wigner 3j (Racah's formula in rational
    arithmetic); odd l1 + l2 + l3 must give 0."""
    wigner = pytest.importorskip("sympy.physics.wigner")
    ref = float(wigner.wigner_3j(l1, l2, l3, 0, 0, 0))
    got = oracle.threej000(l1, l2, l3)
    assert abs(got - ref) <= 1e-15 * max(1.0, abs(ref))


def test_threej_triangle_and_parity_zero():
    assert oracle.threej000(1, 1, 3) == 0.0
    assert oracle.threej000(2, 5, 2) == 0.0
    assert oracle.threej000(4, 4, 1) == 0.0


def test_threej_paper_recurrence_and_terminal_case():
    """(l1 l2 l3) = sqrt[(L-2l2-1)(L-2l3+2) / ((L-2l2)(L-2l3+1))] (l1 l2+1 l3-1)
    with L = l1 + l2 + l3, down to the terminal (l l 0) = (-1)^l / sqrt(2l+1):
    the paper's route, which reaches every symbol with l2 + l3 = l1."""
    for l1 in (1, 5, 17, 60, 301, 1200):
        for l2 in sorted({0, 1, l1 // 3, l1 // 2, l1 - 1, l1}):
            l3 = l1 - l2
            L = l1 + l2 + l3
            v = (-1.0) ** l1 / np.sqrt(2 * l1 + 1)  # (l1, l1, 0)
            for k2 in range(l1 - 1, l2 - 1, -1):  # walk (l1, k2 + 1, L - l1 - k2 - 1) -> (l1, k2, L - l1 - k2)
                k3 = L - l1 - k2
                v *= np.sqrt((L - 2 * k2 - 1) * (L - 2 * k3 + 2) / ((L - 2 * k2) * (L - 2 * k3 + 1)))
            assert abs(oracle.threej000(l1, l2, l3) - v) <= 1e-12 * abs(v), (l1, l2, l3)


@pytest.mark.parametrize("l1,l2", [(0, 0), (3, 5), (40, 40), (100, 37), (1000, 1500), (2048, 2048)])
def test_threej_orthogonality(l1, l2):
    """sum_l3 (2 l3 + 1) (l1 l2 l3; 0 0 0)^2 = 1."""
    s = sum((2 * l3 + 1) * oracle.threej000(l1, l2, l3) ** 2 for l3 in range(abs(l1 - l2), l1 + l2 + 1))
    assert abs(s - 1.0) <= 1e-12


def test_full_sky_coupling_is_identity():
    """w = 1 on the whole sphere: w_00 = sqrt(4 pi), W_0 = 4 pi, W_l>0 = 0,
    so Eq. chat must give M = I."""
    L = 60
    W = np.zeros(L + 1)
    W[0] = FOUR_PI
    M = oracle.coupling(W, L)
    assert np.max(np.abs(M - np.eye(L + 1))) <= 1e-13


def test_row_sums_parseval():
    """A constant C_l (shot noise) is coupled into [sum_l' (2l'+1) W_l' / 4pi] C
    at every l whose row sees all the window's multipoles (l + lmax_w <= lmax)."""
    rng = np.random.default_rng(3)
    L, Lw = 80, 30
    W = rng.uniform(0.1, 1.0, Lw + 1) / (1 + np.arange(Lw + 1)) ** 2
    M = oracle.coupling(W, L)
    target = np.sum((2 * np.arange(Lw + 1) + 1) * W) / FOUR_PI
    rows = M[: L - Lw + 1].sum(axis=1)
    assert np.max(np.abs(rows - target)) <= 1e-13 * target
    assert abs(oracle.fkp_norm(W) * target - 1.0) <= 1e-15


def _sph_grid(n):
    """Gauss-Legendre in x times 2n equispaced phi: exact for band limit < n."""
    x, wx = np.polynomial.legendre.leggauss(n)
    phi = np.arange(2 * n) * (np.pi / n)
    return x, wx, phi


def _ylm_all(lmax, x, phi):
    """Y_lm(x, phi) for -l <= m <= l from scipy (a library independent of the
    oracle): dict (l, m) -> array over the grid."""
    sp = pytest.importorskip("scipy.special")
    th = np.arccos(x)[:, None]
    ph = phi[None, :]
    return {(l, m): sp.sph_harm_y(l, m, th, ph) for l in range(lmax + 1) for m in range(-l, l + 1)}


def test_coupling_equals_masked_ensemble_average():
    """The derivation of Eq. chat done numerically: for a real window w with
    multipoles up to Lw and an isotropic field whose only power is C_l0 = 1,
    <C^_l> = (1/(2l+1)) sum_m sum_m0 |int w Y_l0m0 Y*_lm dOmega|^2 must equal
    M_l l0.  The integrals are exact Gauss-Legendre x phi quadratures of
    scipy's Y_lm; W_l comes from w's own coefficients (Eq. wldef)."""
    Lw, L = 3, 6
    n = Lw + 2 * L + 2
    x, wx, phi = _sph_grid(n)
    Y = _ylm_all(L + Lw, x, phi)
    rng = np.random.default_rng(8)
    wlm = {}
    for l in range(Lw + 1):
        wlm[(l, 0)] = rng.standard_normal()
        for m in range(1, l + 1):
            wlm[(l, m)] = rng.standard_normal() + 1j * rng.standard_normal()
            wlm[(l, -m)] = (-1) ** m * np.conj(wlm[(l, m)])
    wlm[(0, 0)] += 4.0  # mostly positive window
    w = sum(c * Y[k] for k, c in wlm.items()).real
    W = np.array([sum(abs(wlm[(l, m)]) ** 2 for m in range(-l, l + 1)) / (2 * l + 1) for l in range(Lw + 1)])
    quad = wx[:, None] * (np.pi / n)  # dOmega weights: dx dphi
    M = oracle.coupling(W, L)
    for l0 in range(L + 1):
        for l in range(L + 1):
            tot = 0.0
            for m0 in range(-l0, l0 + 1):
                prod = w * Y[(l0, m0)]
                for m in range(-l, l + 1):
                    tot += abs(np.sum(quad * prod * np.conj(Y[(l, m)]))) ** 2
            assert abs(tot / (2 * l + 1) - M[l, l0]) <= 1e-12 * np.max(np.abs(M)), (l, l0)


def test_fkp_norm_parseval():
    """sum_l (2l+1) W_l / 4pi = int w^2 dOmega / 4pi for a band-limited window."""
    Lw = 5
    n = 2 * Lw + 2
    x, wx, phi = _sph_grid(n)
    Y = _ylm_all(Lw, x, phi)
    rng = np.random.default_rng(9)
    wlm = {}
    for l in range(Lw + 1):
        wlm[(l, 0)] = rng.standard_normal()
        for m in range(1, l + 1):
            wlm[(l, m)] = rng.standard_normal() + 1j * rng.standard_normal()
            wlm[(l, -m)] = (-1) ** m * np.conj(wlm[(l, m)])
    w = sum(c * Y[k] for k, c in wlm.items()).real
    W = np.array([sum(abs(wlm[(l, m)]) ** 2 for m in range(-l, l + 1)) / (2 * l + 1) for l in range(Lw + 1)])
    integral = np.sum(wx[:, None] * (np.pi / n) * w ** 2)
    assert abs(1.0 / oracle.fkp_norm(W) - integral / FOUR_PI) <= 1e-13 * integral


def test_binned_full_sky_and_piecewise_constant_recovery():
    """On the full sky M_bb' = I.  With a cut sky, a true C_l that is constant
    on each bin (zero outside the binned range) is recovered exactly by the
    window matrix: cal M C = C_b (Eq. expectation_value)."""
    L = 64
    edges = np.array([2, 5, 9, 17, 30, 50, 65])
    W0 = np.zeros(L + 1)
    W0[0] = FOUR_PI
    R0, Mbb0 = oracle.binned_coupling(oracle.coupling(W0, L), edges)
    assert np.max(np.abs(Mbb0 - np.eye(edges.size - 1))) <= 1e-13
    rng = np.random.default_rng(4)
    W = np.zeros(L + 1)
    W[:20] = rng.uniform(0.2, 1.0, 20) / (1 + np.arange(20)) ** 1.5
    M = oracle.coupling(W, L)
    R, Mbb = oracle.binned_coupling(M, edges)
    Cb = rng.uniform(0.5, 2.0, edges.size - 1)
    C = np.zeros(L + 1)
    for b in range(edges.size - 1):
        C[edges[b]:edges[b + 1]] = Cb[b]
    Minv, Mcal, dec = oracle.decouple(Mbb, R, (oracle.bin_matrix(edges, L) @ (M @ C))[None])
    assert np.max(np.abs(Mcal @ C - Cb)) <= 1e-12 * np.max(Cb)
    assert np.max(np.abs(dec[0] - Cb)) <= 1e-12 * np.max(Cb)


@pytest.mark.parametrize("L,lw", [(0, 0), (1, 5), (7, 3), (40, 80), (40, 100), (25, 10)])
def test_coupling_row_matches_matrix(L, lw):
    """oracle.coupling_row (one row, for the large-lmax GPU comparisons) is
    row l of the pinned matrix: M_ll' carries (2l'+1), so it is not
    symmetric and a transposed or shifted row fails."""
    W = np.random.default_rng(L * 1000 + lw).uniform(0.1, 2.0, lw + 1)
    M = oracle.coupling(W, L)
    if L > 2:
        assert not np.allclose(M, M.T)
    for l in range(L + 1):
        row = oracle.coupling_row(W, L, l)
        assert np.max(np.abs(row - M[l])) <= 1e-13 * max(1.0, np.max(np.abs(M[l]))), l


def test_window_cl_single_point_and_noise():
    """W_l of one point of weight w is w^2/4pi at every l (addition theorem);
    subtracting the shot-noise constant w^2/4pi (the footnote to Eq. wldef)
    leaves zero, and two coincident points give 4 w^2/4pi against a noise
    of 2 w^2/4pi."""
    L, w = 60, 1.7
    x, phi = np.array([0.37]), np.array([2.1])
    a = oracle.alm(x, phi, np.array([w]), L)
    n1 = w * w / FOUR_PI
    assert np.max(np.abs(oracle.window_cl(a, L) - n1)) <= 1e-13 * n1
    assert np.max(np.abs(oracle.window_cl(a, L, n1))) <= 1e-13 * n1
    a2 = oracle.alm(np.repeat(x, 2), np.repeat(phi, 2), np.array([w, w]), L)
    assert np.max(np.abs(oracle.window_cl(a2, L, 2 * n1) - 2 * n1)) <= 1e-13 * n1
