"""The seeded input generators: deterministic, with the requested sizes and structure."""
import math

import numpy as np

from paper_2312_12285_gb300 import catalogs


def test_uniform_fullsky_config1_shape_and_determinism():
    a = catalogs.config(1)
    b = catalogs.config(1)
    assert a.lmax == 128 and a.nfield == 1
    assert [c.n for c in a.catalogs] == [10_000, 50_000]
    assert a.catalogs[1].coeff == -0.2
    for ca, cb in zip(a.catalogs, b.catalogs):
        assert ca.x.dtype == np.float64
        assert np.array_equal(ca.x, cb.x) and np.array_equal(ca.phi, cb.phi)
        assert np.all(np.abs(ca.x) <= 1) and np.all((ca.phi >= 0) & (ca.phi < 2 * math.pi))


def test_lognormal_cap_small():
    wl = catalogs.lognormal_cap(2000, 20000, 256, config_id=2, nwaves=64, grid=(128, 256))
    g, r = wl.catalogs
    assert g.n == 2000 and r.n == 20000 and g.x.dtype == np.float32
    mask = wl.extra["mask"]
    assert mask.contains(g.x, g.phi).all() and mask.contains(r.x, r.phi).all()
    assert np.all((g.w >= 0.8) & (g.w <= 1.2))
    alpha = wl.extra["alpha"]
    assert abs(r.coeff + alpha) < 1e-15
    assert abs(alpha - np.sum(g.w, dtype=np.float64) / np.sum(r.w, dtype=np.float64)) < 1e-12


def test_cap_mask_sky_fraction():
    rng = catalogs.rng_for(99)
    mask = catalogs.make_cap_mask(rng, nholes=0)
    x, phi = catalogs.uniform_sphere(rng, 400_000, np.float64)
    frac = mask.contains(x, phi).mean()
    assert abs(frac - 0.4) < 0.005


def test_golden_spiral_range():
    x, phi = catalogs.golden_spiral(163_840, catalogs.rng_for(6))
    assert x.shape == (163_840,)
    assert np.all(np.abs(x) <= 0.5 + 1e-5)


def test_log_bin_edges():
    e = catalogs.log_bin_edges(1024, 32)
    assert len(e) == 33 and e[-1] == 1025 and np.all(np.diff(e) > 0) and e[0] >= 1


def test_golden_spiral_layout():
    """Sec. 3.1: N points, cos(theta) on [1 - (2k+1)/N]/2 up to the jitter,
    azimuths advancing by 2 pi / varphi (varphi the golden ratio), seeded."""
    wl = catalogs.golden_spiral_workload(4096, 64, jitter=1e-6)
    c = wl.catalogs[0]
    assert c.n == 4096 and wl.lmax == 64 and wl.nfield == 1
    k = np.arange(4096)
    assert np.max(np.abs(c.x - 0.5 * (1 - (2 * k + 1) / 4096))) <= 1e-5
    step = 2 * np.pi * np.mod(2 / (1 + np.sqrt(5)), 1.0)
    dphi = np.mod(np.diff(c.phi.astype(np.float64)) - step + np.pi, 2 * np.pi) - np.pi
    assert np.max(np.abs(dphi)) <= 1e-5
    assert np.array_equal(c.x, catalogs.golden_spiral_workload(4096, 64).catalogs[0].x)
    assert np.all(c.w == 1)


def test_coupling_term_count_matches_brute_force():
    """bench.coupling_terms (the algorithmic work count of the mode-coupling
    row) against a direct count of the non-zero 3j terms of Eq. chat over
    pairs l <= l'."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "bench_mod", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    for L, Lw in ((0, 0), (3, 3), (9, 4), (12, 30), (20, 20)):
        n = sum(1 for l in range(L + 1) for lp in range(l, L + 1)
                for lam in range(lp - l, min(l + lp, Lw) + 1) if (l + lp + lam) % 2 == 0)
        assert bench.coupling_terms(L, Lw) == n, (L, Lw)
