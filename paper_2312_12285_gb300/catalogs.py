"""Seeded synthetic point catalogs with the structure of the paper's workloads.

This module only draws inputs: positions (x = cos theta, phi), weights and the
per-catalog field coefficients.  It contains none of the transform's
arithmetic (no Legendre functions, no harmonic sums) and is shared by the
tests, the benchmark and the oracle comparisons, which all consume the same
arrays.

Workloads (arXiv:2312.12285, Sec. 3 and the direct-SHT timing of Sec. 2.2):

* ``uniform_fullsky``: galaxies and randoms uniform on the sphere, unit
  weights, fixed alpha (the FKP field n_g - alpha n_r, Sec. 2.1).
* ``lognormal_cap``: a lognormal density exp(G - sigma^2/2) of a Gaussian
  random field G, Poisson-sampled into galaxies inside a spherical-cap survey
  mask with small circular holes (the "bright star" mask of Sec. 3.2), plus
  randoms thrown uniformly in the same mask; weights uniform in [0.8, 1.2];
  alpha = sum w_D / sum w_R (normalising a_00 of randoms to data, Sec. 2.3).
* ``tomographic``: several galaxy bins of log-uniform sizes sampled from the
  same G (so their cross-spectra are non-zero) sharing one random catalog.
* ``golden_spiral``: the Fibonacci-spiral point set of Sec. 3.1, between
  cos theta = -1/2 and +1/2, perturbed by a tiny random jitter.

The Gaussian field G is a random-wave field (``WaveField``): a sum of K plane
waves cos(kappa_j khat_j . n + psi_j) on the unit sphere with isotropic
directions, uniform phases and wavenumbers of density (kappa + 10)^(-1/2) on
[1, lmax], which gives C_l^G proportional to (l + 10)^(-3/2) up to lmax.  It is
evaluated at the cell centres of an equiangular grid with one cell per half
wavelength of kappa = lmax, and points are drawn cell by cell (multinomial
counts over the cell weights, uniform positions inside a cell), so the
density carries structure up to lmax.  The field is built from correctly
rounded arithmetic only, so every machine draws the same catalog.
"""
from __future__ import annotations

import hashlib
import math
import os
import pickle
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field as dc_field

import numpy as np

BASE_SEED = 2312_12285


@dataclass
class Catalog:
    """One point catalog: x = cos(theta), phi (radians), weights, and its
    coefficient in one output field (+1 for data, -alpha for randoms)."""
    x: np.ndarray
    phi: np.ndarray
    w: np.ndarray
    coeff: float
    field: int
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


@dataclass
class Workload:
    name: str
    lmax: int
    precision: str  # "fp64" | "fp32" | "mixed"
    nfield: int
    catalogs: list
    extra: dict = dc_field(default_factory=dict)

    @property
    def npoints(self) -> int:
        return sum(c.n for c in self.catalogs)

    @property
    def nmodes(self) -> int:
        return (self.lmax + 1) * (self.lmax + 2) // 2


def rng_for(config_id: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([BASE_SEED + config_id, stream]))


# ------------------------------------------------------------------ masks --
@dataclass
class CapMask:
    """Spherical cap of angular radius rho around (theta0, phi0), minus small
    circular holes.  cos_rho = 0.2 gives a cap of 40% of the sky."""
    theta0: float = math.radians(60.0)
    phi0: float = 1.0
    cos_rho: float = 0.2
    hole_centers: np.ndarray | None = None  # (k, 3) unit vectors
    hole_cos: float = math.cos(math.radians(2.5))

    def contains(self, x: np.ndarray, phi: np.ndarray) -> np.ndarray:
        x = x.astype(np.float64)
        phi = phi.astype(np.float64)
        s = np.sqrt(np.maximum(0.0, (1.0 - x) * (1.0 + x)))
        ux, uy, uz = s * np.cos(phi), s * np.sin(phi), x
        c0 = np.array([math.sin(self.theta0) * math.cos(self.phi0),
                       math.sin(self.theta0) * math.sin(self.phi0), math.cos(self.theta0)])
        inside = ux * c0[0] + uy * c0[1] + uz * c0[2] >= self.cos_rho
        if self.hole_centers is not None:
            for h in self.hole_centers:
                inside &= ux * h[0] + uy * h[1] + uz * h[2] < self.hole_cos
        return inside


def make_cap_mask(rng: np.random.Generator, nholes: int = 10) -> CapMask:
    mask = CapMask()
    centers = []
    while len(centers) < nholes:
        x, phi = _uniform_raw(rng, 64)
        ok = mask.contains(x, phi)
        for xi, pi in zip(x[ok], phi[ok]):
            s = math.sqrt(max(0.0, 1.0 - xi * xi))
            centers.append((s * math.cos(pi), s * math.sin(pi), xi))
            if len(centers) == nholes:
                break
    mask.hole_centers = np.asarray(centers)
    return mask


# ------------------------------------------------------------ primitives --
def _uniform_raw(rng: np.random.Generator, n: int):
    """Uniform on the sphere in float64: x ~ U[-1, 1], phi ~ U[0, 2pi)."""
    x = 2.0 * rng.random(n) - 1.0
    phi = 2.0 * math.pi * rng.random(n)
    return x, phi


def uniform_sphere(rng: np.random.Generator, n: int, dtype=np.float32):
    x, phi = _uniform_raw(rng, n)
    return x.astype(dtype), phi.astype(dtype)


# ------------------------------------------------------ Gaussian field --
# Reproducible trigonometry.  The field below feeds an accept/reject of
# millions of candidates, so a last-bit difference in a library cosine
# between two machines would change which galaxies are drawn.  Every step of
# the field is therefore made of correctly rounded IEEE operations only
# (multiply, add, rint): reduction of the argument to [-pi, pi] in float64 and
# the Taylor series of the cosine, sum_k (-1)^k r^(2k) / (2k)!, to k = 9 by
# Horner's rule in float32 (truncation error pi^20/20! < 4e-9, float32
# rounding ~1e-7): the same bits on any machine.
_TWO_PI = 2.0 * math.pi
_COS_TAYLOR = [np.float32((-1) ** k / math.factorial(2 * k)) for k in range(10)]


def _det_cos(arg: np.ndarray) -> np.ndarray:
    r = arg - _TWO_PI * np.rint(arg * (1.0 / _TWO_PI))
    z32 = r.astype(np.float32)
    z32 *= z32
    p = np.full_like(z32, _COS_TAYLOR[9])
    for k in range(8, -1, -1):
        p *= z32
        p += _COS_TAYLOR[k]
    return p


def _f32(v):
    """Round float64 values to float32 and back, so that a last-bit difference
    in a library sqrt/sin/cos upstream does not reach the field."""
    return np.asarray(v, np.float64).astype(np.float32).astype(np.float64)


@dataclass
class WaveField:
    """Random-wave Gaussian field on the sphere: G(n) = sigma sqrt(2/K) sum_j
    cos(kappa_j khat_j . n + psi_j) with isotropic khat_j, uniform psi_j and
    wavenumbers of density proportional to (kappa + 10)^(-1/2) on [1, lmax].
    One wave restricted to the unit sphere has the angular spectrum
    (2l+1) j_l(kappa)^2 (addition theorem of spherical Bessel functions), which
    for kappa > l averages to ~1/(kappa sqrt(kappa^2 - l^2)) and vanishes for
    kappa < l, so this density gives C_l^G proportional to (l + 10)^(-3/2)
    below lmax (the red spectrum of Sec. 3.2) and no power above lmax
    (band-limited).  Var G = sigma^2.

    G is evaluated at the centres of an equiangular grid of ntheta x nphi cells
    (cell edges theta_j = j pi / ntheta, phi_k = 2 pi k / nphi) with ntheta =
    lmax and nphi = 2 lmax by default: one cell per half wavelength of the
    highest wavenumber."""
    kappa: np.ndarray
    khat: np.ndarray   # (K, 3)
    psi: np.ndarray
    sigma: float
    ntheta: int
    nphi: int
    grid: np.ndarray | None = None  # (ntheta, nphi) float64

    def tabulate(self, block: int = 64):
        nt, npp = self.ntheta, self.nphi
        th = (np.arange(nt) + 0.5) * (math.pi / nt)
        ph = (np.arange(npp) + 0.5) * (_TWO_PI / npp)
        st, ct = _f32(np.sin(th)), _f32(np.cos(th))
        cp, sp = _f32(np.cos(ph)), _f32(np.sin(ph))
        kv = _f32(self.khat * self.kappa[:, None])
        hxy = kv[:, 0:1] * cp[None, :] + kv[:, 1:2] * sp[None, :]   # (K, nphi)
        kz, psi = kv[:, 2], _f32(self.psi)
        K = kv.shape[0]
        amp = self.sigma * math.sqrt(2.0 / K)
        grid = np.empty((nt, npp), np.float64)

        def rows(j0, j1):
            for j in range(j0, j1):
                acc = np.zeros(npp, np.float64)
                for w0 in range(0, K, block):
                    w1 = min(K, w0 + block)
                    arg = st[j] * hxy[w0:w1] + (ct[j] * kz[w0:w1] + psi[w0:w1])[:, None]
                    acc += _det_cos(arg).sum(axis=0, dtype=np.float64)
                grid[j] = amp * acc

        nthr = max(1, min(16, os.cpu_count() or 1))
        step = max(1, (nt + 4 * nthr - 1) // (4 * nthr))
        with ThreadPoolExecutor(nthr) as ex:
            list(ex.map(lambda j0: rows(j0, min(nt, j0 + step)), range(0, nt, step)))
        self.grid = grid


def make_wave_field(rng: np.random.Generator, lmax: int, nwaves: int = 256, sigma: float = 0.5,
                    grid=None) -> WaveField:
    u = rng.random(nwaves)
    a, b = math.sqrt(11.0), math.sqrt(lmax + 10.0)
    kappa = (a + u * (b - a)) ** 2 - 10.0
    dx, dphi = _uniform_raw(rng, nwaves)
    ds = np.sqrt(np.maximum(0.0, 1.0 - dx * dx))
    khat = np.stack([ds * np.cos(dphi), ds * np.sin(dphi), dx], axis=1)
    psi = _TWO_PI * rng.random(nwaves)
    nt, npp = grid if grid is not None else (max(64, lmax), 2 * max(64, lmax))
    f = WaveField(kappa, khat, psi, sigma, int(nt), int(npp))
    f.tabulate()
    return f


# --------------------------------------------------- sampling by cells --
def _cell_geometry(nt: int, npp: int):
    """cos of the theta edges (nt + 1) and the solid angle of a cell in ring j."""
    ce = _f32(np.cos(np.arange(nt + 1) * (math.pi / nt)))
    ce[0], ce[-1] = 1.0, -1.0
    area = (ce[:-1] - ce[1:]) * (_TWO_PI / npp)
    return ce, area


def _cells_near_mask(mask: CapMask, nt: int, npp: int) -> np.ndarray:
    """(nt, npp) bool: cells whose centre lies within the cap radius plus one
    cell width of the cap centre (every cell that meets the cap)."""
    th = (np.arange(nt) + 0.5) * (math.pi / nt)
    ph = (np.arange(npp) + 0.5) * (_TWO_PI / npp)
    c0 = np.array([math.sin(mask.theta0) * math.cos(mask.phi0), math.sin(mask.theta0) * math.sin(mask.phi0),
                   math.cos(mask.theta0)])
    d = np.sin(th)[:, None] * (c0[0] * np.cos(ph) + c0[1] * np.sin(ph))[None, :] + c0[2] * np.cos(th)[:, None]
    rho = math.acos(mask.cos_rho) + 1.5 * math.pi / nt
    return d >= math.cos(min(math.pi, rho))


def sample_cells(rng: np.random.Generator, n: int, weight: np.ndarray, mask: CapMask, dtype=np.float32):
    """n points drawn with a density proportional to weight[j, k] / area(j, k)
    inside cell (j, k) of an equiangular grid, restricted to the mask: cell
    counts from a multinomial over the cell weights, positions uniform in
    solid angle inside the cell (x uniform between the cell's cos theta edges,
    phi uniform between its edges), points outside the mask rejected and
    replaced by further rounds; of the accepted points a random n are kept,
    in random order (a Poisson sample conditioned on its total)."""
    nt, npp = weight.shape
    ce, _ = _cell_geometry(nt, npp)
    p = weight.ravel() / weight.sum()
    xs, ps, have, acc = [], [], 0, 0.9
    while have < n:
        ndraw = int((n - have) / acc * 1.02) + 256
        counts = rng.multinomial(ndraw, p)
        cells = np.repeat(np.arange(p.size, dtype=np.int64), counts)
        j, k = cells // npp, cells % npp
        x = ce[j + 1] + rng.random(ndraw) * (ce[j] - ce[j + 1])
        phi = (k + rng.random(ndraw)) * (_TWO_PI / npp)
        ok = mask.contains(x, phi)
        acc = max(0.05, float(ok.mean()))
        xs.append(x[ok])
        ps.append(phi[ok])
        have += int(ok.sum())
    x, phi = np.concatenate(xs), np.concatenate(ps)
    keep = rng.permutation(x.shape[0])[:n]
    return x[keep].astype(dtype), phi[keep].astype(dtype)


def field_weights(fld: WaveField, mask: CapMask) -> np.ndarray:
    """Cell weights of the lognormal density exp(G - sigma^2/2) times the cell's
    solid angle, zero for cells that do not meet the cap."""
    _, area = _cell_geometry(fld.ntheta, fld.nphi)
    near = _cells_near_mask(mask, fld.ntheta, fld.nphi)
    return np.where(near, np.exp(fld.grid - 0.5 * fld.sigma ** 2) * area[:, None], 0.0)


def uniform_weights(mask: CapMask, nt: int, npp: int) -> np.ndarray:
    _, area = _cell_geometry(nt, npp)
    near = _cells_near_mask(mask, nt, npp)
    return np.where(near, np.broadcast_to(area[:, None], (nt, npp)), 0.0)


def golden_spiral(n: int, rng: np.random.Generator, jitter: float = 1e-6, dtype=np.float32):
    """Fibonacci spiral between cos theta = -1/2 and 1/2 (Sec. 3.1), k = 0..n-1,
    each point moved by a small Gaussian jitter (radians) in theta and phi."""
    k = np.arange(n, dtype=np.float64)
    x = 0.5 * (1.0 - (2.0 * k + 1.0) / n)
    golden = (1.0 + math.sqrt(5.0)) / 2.0
    phi = np.mod(2.0 * math.pi * k / golden, 2.0 * math.pi)
    th = np.arccos(x) + jitter * rng.standard_normal(n)
    phi = np.mod(phi + jitter * rng.standard_normal(n), 2.0 * math.pi)
    return np.cos(th).astype(dtype), phi.astype(dtype)


# -------------------------------------------------------------- workloads --
def uniform_fullsky(n_gal: int = 10_000, n_ran: int = 50_000, alpha: float = 0.2, lmax: int = 128,
                    dtype=np.float64, config_id: int = 1, precision: str = "fp64") -> Workload:
    rng = rng_for(config_id)
    xg, pg = uniform_sphere(rng, n_gal, dtype)
    xr, pr = uniform_sphere(rng, n_ran, dtype)
    cats = [Catalog(xg, pg, np.ones(n_gal, dtype), 1.0, 0, "galaxies"),
            Catalog(xr, pr, np.ones(n_ran, dtype), -alpha, 0, "randoms")]
    return Workload("uniform_fullsky", lmax, precision, 1, cats, {"alpha": alpha})


def lognormal_cap(n_gal: int, n_ran: int, lmax: int, config_id: int, precision: str = "fp32",
                  dtype=np.float32, nwaves: int = 256, grid=None, nholes: int = 10,
                  name: str = "lognormal_cap") -> Workload:
    """Galaxies Poisson-sampled from the lognormal density exp(G - sigma^2/2)
    (sigma = 0.5, G band-limited to lmax) inside the cap mask, randoms uniform
    in the same mask, weights U[0.8, 1.2], alpha = sum w_D / sum w_R."""
    rng = rng_for(config_id)
    mask = make_cap_mask(rng, nholes)
    fld = make_wave_field(rng, lmax, nwaves=nwaves, grid=grid)
    xg, pg = sample_cells(rng, n_gal, field_weights(fld, mask), mask, dtype)
    xr, pr = sample_cells(rng, n_ran, uniform_weights(mask, fld.ntheta, fld.nphi), mask, dtype)
    wg = rng.uniform(0.8, 1.2, n_gal).astype(dtype)
    wr = rng.uniform(0.8, 1.2, n_ran).astype(dtype)
    alpha = float(np.sum(wg, dtype=np.float64) / np.sum(wr, dtype=np.float64))
    cats = [Catalog(xg, pg, wg, 1.0, 0, "galaxies"), Catalog(xr, pr, wr, -alpha, 0, "randoms")]
    return Workload(name, lmax, precision, 1, cats, {"alpha": alpha, "mask": mask})


def tomographic(nbins: int, n_min: float, n_max: float, n_ran: int, lmax: int, config_id: int = 4,
                precision: str = "fp32", dtype=np.float32, nwaves: int = 256, grid=None):
    """Galaxy bins of log-uniform sizes in [n_min, n_max] sampled from one
    lognormal density (so their cross-spectra are non-zero), and a shared
    random catalog.  Fields 0..nbins-1 are the bins (coeff +1) and field nbins
    is the random catalog (coeff +1); the FKP fields D_b - alpha_b R are
    linear combinations of these (extra['alpha'][b] = sum w_b / sum w_R)."""
    rng = rng_for(config_id)
    mask = make_cap_mask(rng, 10)
    fld = make_wave_field(rng, lmax, nwaves=nwaves, grid=grid)
    wgt = field_weights(fld, mask)
    sizes = np.round(10.0 ** rng.uniform(math.log10(n_min), math.log10(n_max), nbins)).astype(np.int64)
    cats = []
    for b, nb in enumerate(sizes):
        x, p = sample_cells(rng, int(nb), wgt, mask, dtype)
        w = rng.uniform(0.8, 1.2, int(nb)).astype(dtype)
        cats.append(Catalog(x, p, w, 1.0, b, f"bin{b}"))
    xr, pr = sample_cells(rng, n_ran, uniform_weights(mask, fld.ntheta, fld.nphi), mask, dtype)
    wr = rng.uniform(0.8, 1.2, n_ran).astype(dtype)
    cats.append(Catalog(xr, pr, wr, 1.0, nbins, "randoms"))
    sw_r = float(np.sum(wr, dtype=np.float64))
    alpha = [float(np.sum(c.w, dtype=np.float64)) / sw_r for c in cats[:nbins]]
    return Workload("tomographic", lmax, precision, nbins + 1, cats,
                    {"alpha": alpha, "nbins": nbins, "mask": mask})


def weight_columns(wl: Workload, ncol: int):
    """One point set (all catalogs of field 0 concatenated) carrying ``ncol``
    weight columns, as jackknife resampling of a pseudo-C_l uses them:
    column 0 is the field's signed weights coeff_c * w_i (data - alpha
    randoms); column k >= 1 is the same with the k-th of ncol - 1 equal
    azimuthal wedges removed (weights set to 0).  Returns float32 x, phi [n]
    and W [ncol, n]."""
    cats = [c for c in wl.catalogs if c.field == 0]
    x = np.concatenate([c.x for c in cats]).astype(np.float32)
    phi = np.concatenate([c.phi for c in cats]).astype(np.float32)
    w0 = np.concatenate([c.w.astype(np.float64) * c.coeff for c in cats]).astype(np.float32)
    W = np.empty((ncol, x.shape[0]), np.float32)
    W[0] = w0
    nw = max(1, ncol - 1)
    wedge = np.floor(np.mod(phi.astype(np.float64), 2.0 * math.pi) / (2.0 * math.pi) * nw).astype(np.int64)
    for k in range(1, ncol):
        W[k] = np.where(wedge == k - 1, np.float32(0.0), w0)
    return x, phi, W


def log_bin_edges(lmax: int, nbins: int = 32) -> np.ndarray:
    """Log-spaced multipole bin edges e_k = floor(2 (N_l/2)^(k/nbins)), made
    strictly increasing, with the last edge = lmax + 1."""
    nl = lmax + 1
    e = [int(math.floor(2.0 * (nl / 2.0) ** (k / nbins))) for k in range(nbins + 1)]
    e[-1] = nl
    for k in range(1, nbins + 1):
        if e[k] <= e[k - 1]:
            e[k] = e[k - 1] + 1
    for k in range(nbins - 1, -1, -1):
        if e[k] >= e[k + 1]:
            e[k] = e[k + 1] - 1
    return np.asarray(e, np.int64)


def golden_spiral_workload(n: int = 163_840, lmax: int = 2048, jitter: float = 1e-6, config_id: int = 6,
                           dtype=np.float32) -> Workload:
    """The golden-spiral example (Sec. 3.1) as a workload: ``golden_spiral``
    points with w = 1 in one field.  A blue spectrum: most of its power at
    high l."""
    x, phi = golden_spiral(n, rng_for(config_id), jitter, dtype)
    cats = [Catalog(x, phi, np.ones(n, dtype), 1.0, 0, "spiral")]
    return Workload("golden_spiral", lmax, "fp32", 1, cats, {"jitter": jitter})


def config(i: int, scale: float = 1.0, lmax: int | None = None) -> Workload:
    """The five configurations (and the spiral), optionally with point counts
    scaled by ``scale``; built once per machine and kept in the on-disk cache
    (``cached``).

    1 plain FP64: 1e4 galaxies + 5e4 randoms, full sky, w = 1, alpha = 0.2, lmax 128.
    2 plain FP32: 1e6 galaxies (lognormal, cap mask 40% sky) + 1e7 randoms, lmax 1024.
    3 precision: 1e7 points (1e6 galaxies + 9e6 randoms), same mask/field, lmax 2048.
    4 batching: 16 bins of 10^U[5,7] galaxies + 2e7 shared randoms, lmax 1536.
    5 differentiation: 2e6 galaxies + 1e7 randoms, lmax 1024, 32 log bins.
    6 golden spiral: 163 840 points with |cos theta| <= 1/2, w = 1, lmax 2048.
    """
    return cached(("config", i, scale, lmax), lambda: _config(i, scale, lmax))


def _config(i: int, scale: float, lmax: int | None) -> Workload:
    def sc(n):
        return max(1, int(round(n * scale)))
    if i == 1:
        return uniform_fullsky(sc(10_000), sc(50_000), 0.2, lmax or 128)
    if i == 2:
        return lognormal_cap(sc(1_000_000), sc(10_000_000), lmax or 1024, 2, "fp32",
                             name="lognormal_cap_l1024")
    if i == 3:
        return lognormal_cap(sc(1_000_000), sc(9_000_000), lmax or 2048, 3, "mixed",
                             name="lognormal_cap_l2048")
    if i == 4:
        return tomographic(16, 1e5 * scale, 1e7 * scale, sc(20_000_000), lmax or 1536)
    if i == 5:
        wl = lognormal_cap(sc(2_000_000), sc(10_000_000), lmax or 1024, 5, "fp32",
                           name="differentiation_l1024")
        L = wl.lmax
        wl.extra["edges"] = log_bin_edges(L, 32)
        r = rng_for(5, 7)
        wl.extra["g_b"] = r.standard_normal(32)
        ng, nr = wl.catalogs[0].n, wl.catalogs[1].n
        wl.extra["fd_idx"] = [np.sort(r.choice(ng, min(32, ng), replace=False)),
                              np.sort(r.choice(nr, min(32, nr), replace=False))]
        return wl
    if i == 6:
        return golden_spiral_workload(sc(163_840), lmax or 2048)
    raise ValueError(f"unknown config {i}")


# ------------------------------------------------------------ disk cache --
def _cache_dir() -> str:
    d = os.environ.get("POINTSHT_CACHE_DIR")
    if not d:
        d = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_cache", "catalogs")
    return d


def cached(key, build):
    """build() memoised on disk under a key made of ``key`` and this module's
    source text (a change to any generator invalidates every entry).  The
    large configurations take tens of seconds to draw; tests, the benchmark
    and the oracle's reference script then share one draw per machine."""
    with open(os.path.abspath(__file__), "rb") as fh:
        h = hashlib.sha1(fh.read())
    h.update(repr(key).encode())
    path = os.path.join(_cache_dir(), h.hexdigest()[:20] + ".pkl")
    if os.path.exists(path):
        try:
            with open(path, "rb") as fh:
                return pickle.load(fh)
        except Exception:
            pass
    wl = build()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "wb") as fh:
            pickle.dump(wl, fh, protocol=5)
        os.replace(tmp, path)
    except OSError:
        pass
    return wl


def fingerprint(wl: Workload) -> list:
    """Per catalog: point count and a SHA-1 of the x, phi and w bytes (used to
    check that a stored oracle result belongs to the catalog at hand)."""
    out = []
    for c in wl.catalogs:
        h = hashlib.sha1()
        for a in (c.x, c.phi, c.w):
            h.update(np.ascontiguousarray(a).tobytes())
        out.append([c.n, h.hexdigest()])
    return out
