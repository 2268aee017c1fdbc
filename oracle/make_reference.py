"""Stored FP64 oracle values for the full-size parity tests.

TEST INFRASTRUCTURE ONLY (see the package docstring).  This script calls
nothing but this package and the seeded input generators; it writes the
expected values that the batching and differentiation tests compare the
library with at the sizes their configurations state, where the oracle needs
hours instead of seconds:

* ``tests/golden/tomographic_l1536_oracle.npz`` -- the batching workload
  (16 tomographic bins of uneven sizes plus 2e7 shared randoms, lmax 1536):
  for every catalog, a_lm for l <= 32 (the packed triangle at lmax 32) and
  the whole columns m = 0, 1200, 1535, 1536 at lmax 1536 (Eq. alm_def; the
  fields D_b - alpha_b R follow by linearity, Sec. 2.1).
* ``tests/golden/differentiation_l1024_fd.json`` -- the differentiation
  workload (2e6 galaxies + 1e7 randoms, lmax 1024, 32 log bins, cotangent
  g_b): the full a_lm of the field D - alpha R, then for each of the 64
  chosen objects the central finite difference of L = sum_b g_b C_b (C_b the
  binned, shot-noise-subtracted pseudo-C_l of Eq. pseudoCl) with step
  h = 1e-3 w_i.  a_lm is linear in w_i, so a(w_i +- h) = a +- h s_i Y*(n_i)
  exactly (s_i the catalog's coefficient), and the shot noise changes by
  +- (2 s_i^2 w_i h + s_i^2 h^2)/4pi: each difference is a rank-one update of
  the stored a_lm, exact up to FP64 rounding, with no recomputation of the
  transform.  The definition-level gradient (``grad_binned_cl``'s chain rule)
  is stored beside it.

Each file records the catalog fingerprint (point count and SHA-1 of the
arrays per catalog), so a test can tell whether the catalog it generated is
the one these values belong to, and the oracle's wall time and thread count.

Usage: python -m oracle.make_reference [tomographic] [differentiation]
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

import oracle
from paper_2312_12285_gb300 import catalogs

GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")
TOMO_FILE = os.path.join(GOLDEN, "tomographic_l1536_oracle.npz")
DIFF_FILE = os.path.join(GOLDEN, "differentiation_l1024_fd.json")
TOMO_LOW_L = 32
TOMO_COLUMNS = (0, 1200, 1535, 1536)
FD_REL_STEP = 1e-3


def tomographic():
    wl = catalogs.config(4)
    L = wl.lmax
    t0 = time.time()
    low, cols = [], []
    for c in wl.catalogs:
        w = c.w.astype(np.float64)
        low.append(oracle.alm(c.x, c.phi, w, TOMO_LOW_L))
        col = oracle.alm(c.x, c.phi, w, L, mlist=list(TOMO_COLUMNS))
        cols.append(np.concatenate([col[m] for m in TOMO_COLUMNS]))
    dt = time.time() - t0
    np.savez(TOMO_FILE, low=np.asarray(low), cols=np.asarray(cols), columns=np.asarray(TOMO_COLUMNS),
             low_lmax=TOMO_LOW_L, lmax=L, alpha=np.asarray(wl.extra["alpha"]),
             fingerprint=json.dumps(catalogs.fingerprint(wl)), oracle_seconds=dt,
             oracle_threads=os.cpu_count())
    print(f"tomographic: {len(wl.catalogs)} catalogs, {wl.npoints} points, {dt:.0f} s", flush=True)


def _loss(a, noise, gl, L):
    """L = sum_l gbar_l (C_l - N), gbar_l = sum_b g_b theta_b^l."""
    return float(np.dot(gl, oracle.cl(a, a, L) - noise))


def differentiation():
    wl = catalogs.config(5)
    L = wl.lmax
    edges, g_b = wl.extra["edges"], wl.extra["g_b"]
    gl = oracle.bin_matrix(edges, L).T @ g_b
    cats = [(c.x, c.phi, c.w.astype(np.float64), c.coeff) for c in wl.catalogs]
    t0 = time.time()
    a = oracle.field_alm(cats, L)
    dt_alm = time.time() - t0
    s2w2 = sum(float(np.sum((c.w.astype(np.float64) * c.coeff) ** 2)) for c in wl.catalogs)
    noise = s2w2 / oracle.FOUR_PI
    loss = _loss(a, noise, gl, L)
    objs, fd = [], []
    for ci, idx in enumerate(wl.extra["fd_idx"]):
        c = wl.catalogs[ci]
        for i in idx:
            i = int(i)
            wi, si = float(c.w[i]), float(c.coeff)
            h = FD_REL_STEP * wi
            y = oracle.alm(c.x[i:i + 1], c.phi[i:i + 1], np.ones(1), L)   # Y*_lm(n_i)
            dn = (2.0 * si * si * wi * h) / oracle.FOUR_PI
            dn2 = (si * si * h * h) / oracle.FOUR_PI
            lp = _loss(a + h * si * y, noise + dn + dn2, gl, L)
            lm = _loss(a - h * si * y, noise - dn + dn2, gl, L)
            objs.append([ci, i])
            fd.append((lp - lm) / (2.0 * h))
    gdef = oracle.grad_binned_cl(cats, L, edges, g_b, wl.extra["fd_idx"])
    gdef = [float(v) for arr in gdef for v in arr]
    out = {
        "what": "central finite differences of L = sum_b g_b C_b (binned shot-noise-subtracted pseudo-C_l, "
                "Eq. pseudoCl) w.r.t. 64 object weights, by exact rank-one updates of the FP64 oracle a_lm",
        "config": "differentiation: 2e6 galaxies + 1e7 randoms, lmax 1024, 32 log bins",
        "objects": objs, "fd": fd, "grad_definition": gdef, "h_rel": FD_REL_STEP, "loss": loss,
        "fingerprint": catalogs.fingerprint(wl), "oracle_alm_seconds": dt_alm, "oracle_threads": os.cpu_count(),
        "points": wl.npoints, "lmax": L,
    }
    with open(DIFF_FILE, "w") as fh:
        json.dump(out, fh, indent=1)
    print(f"differentiation: a_lm {dt_alm:.0f} s; max |fd - definition| / max |fd| = "
          f"{np.max(np.abs(np.asarray(fd) - np.asarray(gdef))) / np.max(np.abs(fd)):.2e}", flush=True)


if __name__ == "__main__":
    what = sys.argv[1:] or ["tomographic", "differentiation"]
    os.makedirs(GOLDEN, exist_ok=True)
    oracle.build()
    for w in what:
        {"tomographic": tomographic, "differentiation": differentiation}[w]()
