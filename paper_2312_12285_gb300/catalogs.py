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
  random field G, Poisson-thinned into galaxies inside a spherical-cap survey
  mask with small circular holes (the "bright star" mask of Sec. 3.2), plus
  randoms thrown uniformly in the same mask; weights uniform in [0.8, 1.2];
  alpha = sum w_D / sum w_R (normalising a_00 of randoms to data, Sec. 2.3).
* ``tomographic``: several galaxy bins of log-uniform sizes thinned from the
  same G (so their cross-spectra are non-zero) sharing one random catalog.
* ``golden_spiral``: the Fibonacci-spiral point set of Sec. 3.1, between
  cos theta = -1/2 and +1/2, perturbed by a tiny random jitter.

The Gaussian field G is a random-wave field: a sum of K plane waves
cos(kappa_j khat_j . n + psi_j) evaluated on the unit sphere, with isotropic
directions, uniform phases and wavenumbers drawn with density proportional to
(kappa + 10)^(-1/2) on [1, kappa_max].  A plane wave of wavenumber kappa puts
angular power at l <~ kappa with weight ~ 1/(kappa sqrt(kappa^2 - l^2)), so this
density gives C_l^G roughly proportional to (l + 10)^(-3/2) (the red spectrum
of Sec. 3.2).  G is tabulated on an equiangular (theta, phi) grid and read
with bilinear interpolation.
"""
from __future__ import annotations

import math
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


def uniform_in_mask(rng: np.random.Generator, n: int, mask: CapMask, dtype=np.float32,
                    batch: int = 1 << 22):
    xs, ps, have = [], [], 0
    while have < n:
        x, phi = _uniform_raw(rng, batch)
        ok = mask.contains(x, phi)
        xs.append(x[ok])
        ps.append(phi[ok])
        have += int(ok.sum())
    x = np.concatenate(xs)[:n].astype(dtype)
    phi = np.concatenate(ps)[:n].astype(dtype)
    return x, phi


@dataclass
class RandomWaveField:
    """Gaussian-like random field on the sphere from K random plane waves."""
    kvec: np.ndarray   # (K, 3) wave vectors kappa * khat
    psi: np.ndarray    # (K,) phases
    sigma: float
    grid_theta: np.ndarray | None = None
    grid: np.ndarray | None = None     # (ntheta, nphi) tabulated G

    def evaluate(self, x: np.ndarray, phi: np.ndarray, chunk: int = 1 << 15) -> np.ndarray:
        """Direct evaluation (float64) at points; cost K per point."""
        out = np.empty(x.shape[0], np.float64)
        amp = self.sigma * math.sqrt(2.0 / self.kvec.shape[0])
        for i0 in range(0, x.shape[0], chunk):
            xx = x[i0:i0 + chunk].astype(np.float64)
            pp = phi[i0:i0 + chunk].astype(np.float64)
            s = np.sqrt(np.maximum(0.0, (1.0 - xx) * (1.0 + xx)))
            n3 = np.stack([s * np.cos(pp), s * np.sin(pp), xx], axis=1)
            arg = n3 @ self.kvec.T + self.psi[None, :]
            out[i0:i0 + chunk] = amp * np.cos(arg).sum(axis=1)
        return out

    def tabulate(self, ntheta: int, nphi: int):
        th = (np.arange(ntheta) + 0.5) * math.pi / ntheta
        ph = np.arange(nphi) * 2.0 * math.pi / nphi
        tt, pp = np.meshgrid(th, ph, indexing="ij")
        g = self.evaluate(np.cos(tt).ravel(), pp.ravel())
        self.grid_theta = th
        self.grid = g.reshape(ntheta, nphi).astype(np.float32)

    def lookup(self, x: np.ndarray, phi: np.ndarray) -> np.ndarray:
        """Bilinear interpolation of the tabulated field."""
        nt, npp = self.grid.shape
        th = np.arccos(np.clip(x.astype(np.float64), -1.0, 1.0))
        ft = th / math.pi * nt - 0.5
        fp = np.mod(phi.astype(np.float64), 2.0 * math.pi) / (2.0 * math.pi) * npp
        it = np.clip(np.floor(ft).astype(np.int64), 0, nt - 2)
        dt = np.clip(ft - it, 0.0, 1.0)
        ip = np.floor(fp).astype(np.int64) % npp
        dp = fp - np.floor(fp)
        ip1 = (ip + 1) % npp
        g = self.grid
        v = ((1 - dt) * (1 - dp) * g[it, ip] + (1 - dt) * dp * g[it, ip1]
             + dt * (1 - dp) * g[it + 1, ip] + dt * dp * g[it + 1, ip1])
        return v


def make_random_wave_field(rng: np.random.Generator, kappa_max: float, nwaves: int = 256,
                           sigma: float = 0.5, ntheta: int = 512, nphi: int = 1024) -> RandomWaveField:
    u = rng.random(nwaves)
    a, b = math.sqrt(11.0), math.sqrt(kappa_max + 10.0)
    kappa = (a + u * (b - a)) ** 2 - 10.0
    dx, dphi = _uniform_raw(rng, nwaves)
    ds = np.sqrt(np.maximum(0.0, 1.0 - dx * dx))
    khat = np.stack([ds * np.cos(dphi), ds * np.sin(dphi), dx], axis=1)
    f = RandomWaveField(kvec=khat * kappa[:, None], psi=2.0 * math.pi * rng.random(nwaves),
                        sigma=sigma)
    f.tabulate(ntheta, nphi)
    return f


def poisson_thin(rng: np.random.Generator, n: int, mask: CapMask, fld: RandomWaveField,
                 dtype=np.float32, batch: int = 1 << 21):
    """n galaxies with density proportional to exp(G - sigma^2/2) inside the mask
    (accept/reject against the maximum of the tabulated field)."""
    gmax = float(fld.grid.max())
    xs, ps, have = [], [], 0
    while have < n:
        x, phi = uniform_in_mask(rng, batch, mask, dtype=np.float64)
        g = fld.lookup(x, phi)
        keep = rng.random(x.shape[0]) < np.exp(g - gmax)
        xs.append(x[keep])
        ps.append(phi[keep])
        have += int(keep.sum())
    return np.concatenate(xs)[:n].astype(dtype), np.concatenate(ps)[:n].astype(dtype)


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
                  dtype=np.float32, nwaves: int = 256, grid=(512, 1024), nholes: int = 10,
                  name: str = "lognormal_cap") -> Workload:
    rng = rng_for(config_id)
    mask = make_cap_mask(rng, nholes)
    fld = make_random_wave_field(rng, kappa_max=float(lmax), nwaves=nwaves, ntheta=grid[0],
                                 nphi=grid[1])
    xg, pg = poisson_thin(rng, n_gal, mask, fld, dtype)
    xr, pr = uniform_in_mask(rng, n_ran, mask, dtype)
    wg = rng.uniform(0.8, 1.2, n_gal).astype(dtype)
    wr = rng.uniform(0.8, 1.2, n_ran).astype(dtype)
    alpha = float(np.sum(wg, dtype=np.float64) / np.sum(wr, dtype=np.float64))
    cats = [Catalog(xg, pg, wg, 1.0, 0, "galaxies"), Catalog(xr, pr, wr, -alpha, 0, "randoms")]
    return Workload(name, lmax, precision, 1, cats, {"alpha": alpha, "mask": mask})


def tomographic(nbins: int, n_min: float, n_max: float, n_ran: int, lmax: int, config_id: int = 4,
                precision: str = "fp32", dtype=np.float32, nwaves: int = 256, grid=(512, 1024)):
    """Galaxy bins of log-uniform sizes in [n_min, n_max] from one field G, and a
    shared random catalog.  Fields 0..nbins-1 are the bins (coeff +1) and field
    nbins is the random catalog (coeff +1); the FKP fields D_b - alpha_b R are
    linear combinations of these (extra['alpha'][b] = sum w_b / sum w_R)."""
    rng = rng_for(config_id)
    mask = make_cap_mask(rng, 10)
    fld = make_random_wave_field(rng, kappa_max=float(lmax), nwaves=nwaves, ntheta=grid[0],
                                 nphi=grid[1])
    sizes = np.round(10.0 ** rng.uniform(math.log10(n_min), math.log10(n_max), nbins)).astype(np.int64)
    cats = []
    for b, nb in enumerate(sizes):
        x, p = poisson_thin(rng, int(nb), mask, fld, dtype)
        w = rng.uniform(0.8, 1.2, int(nb)).astype(dtype)
        cats.append(Catalog(x, p, w, 1.0, b, f"bin{b}"))
    xr, pr = uniform_in_mask(rng, n_ran, mask, dtype)
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
    """The five configurations, optionally with point counts scaled by ``scale``.

    1 plain FP64: 1e4 galaxies + 5e4 randoms, full sky, w = 1, alpha = 0.2, lmax 128.
    2 plain FP32: 1e6 galaxies (lognormal, cap mask 40% sky) + 1e7 randoms, lmax 1024.
    3 precision: 1e7 points (1e6 galaxies + 9e6 randoms), same mask/field, lmax 2048.
    4 batching: 16 bins of 10^U[5,7] galaxies + 2e7 shared randoms, lmax 1536.
    5 differentiation: 2e6 galaxies + 1e7 randoms, lmax 1024, 32 log bins.
    6 golden spiral: 163 840 points with |cos theta| <= 1/2, w = 1, lmax 2048.
    """
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
