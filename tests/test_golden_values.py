"""The stored oracle values under tests/golden/ (written by
oracle/make_reference.py, which calls only the oracle and the seeded
generators) checked on the CPU, without the hours of oracle time that wrote
them:

* each file belongs to the catalogs the generators draw today (point counts
  and SHA-1 of the arrays per catalog), so the GPU tests that read it compare
  like with like;
* the batching workload's values (16 tomographic bins + 2e7 shared randoms,
  lmax 1536): for every catalog, a_00 = sum w / sqrt(4 pi) and
  a_10 = sqrt(3 / 4 pi) sum w x (closed forms of Y_00 and Y_10, Eq. alm_def)
  from the catalog's own arrays, and the m = 0 column taken at lmax 1536
  equal, for l <= 32, to the l <= 32 triangle of a separate oracle call (a_lm
  does not depend on lmax);
* the differentiation workload's central differences (exact rank-one
  updates of the oracle a_lm) agree with the oracle's definition-level
  gradient of the binned pseudo-C_l stored beside them, and the objects are
  the ones the generator picks.
"""
import json
import os
import shutil

import numpy as np
import pytest

import oracle
from paper_2312_12285_gb300 import catalogs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(autouse=True)
def _private_catalog_cache(tmp_path, monkeypatch):
    """The two workloads are ~0.8 GB of drawn catalogs: cache them in this
    test's temporary directory, outside the source tree, and drop them after."""
    d = tmp_path / "catalogs"
    monkeypatch.setenv("POINTSHT_CACHE_DIR", str(d))
    yield
    shutil.rmtree(d, ignore_errors=True)


def test_tomographic_values_closed_forms_and_consistency():
    ref = np.load(os.path.join(GOLDEN, "tomographic_l1536_oracle.npz"))
    wl = catalogs.config(4)
    assert catalogs.fingerprint(wl) == json.loads(str(ref["fingerprint"]))
    L, Ls = int(ref["lmax"]), int(ref["low_lmax"])
    cols = [int(m) for m in ref["columns"]]
    assert L == wl.lmax == 1536 and Ls == 32 and cols[0] == 0 and cols[-1] == L
    assert np.array_equal(ref["alpha"], np.asarray(wl.extra["alpha"]))
    low, col = ref["low"], ref["cols"]
    assert low.shape == (len(wl.catalogs), oracle.nmodes(Ls))
    assert col.shape == (len(wl.catalogs), sum(L - m + 1 for m in cols))
    for k, c in enumerate(wl.catalogs):
        w, x = c.w.astype(np.float64), c.x.astype(np.float64)
        a00 = np.sum(w) / np.sqrt(4 * np.pi)
        a10 = np.sqrt(3 / (4 * np.pi)) * np.sum(w * x)
        scale = np.sqrt(np.sum(w * w) / (4 * np.pi))  # typical |a_lm| of the catalog
        assert abs(low[k][oracle.index(0, 0, Ls)] - a00) <= 1e-11 * abs(a00)
        assert abs(low[k][oracle.index(1, 0, Ls)] - a10) <= 1e-11 * scale
        m0 = col[k][:Ls + 1]  # the m = 0 column, l = 0..32
        tri = np.asarray([low[k][oracle.index(l, 0, Ls)] for l in range(Ls + 1)])
        assert np.max(np.abs(m0 - tri)) <= 1e-12 * np.max(np.abs(tri))


def test_differentiation_values_consistent():
    with open(os.path.join(GOLDEN, "differentiation_l1024_fd.json")) as fh:
        ref = json.load(fh)
    wl = catalogs.config(5)
    assert catalogs.fingerprint(wl) == ref["fingerprint"]
    assert ref["points"] == wl.npoints and ref["lmax"] == wl.lmax
    assert [list(map(int, o)) for o in ref["objects"]] == [[ci, int(i)] for ci, idx in enumerate(wl.extra["fd_idx"])
                                                          for i in idx]
    fd, gdef = np.asarray(ref["fd"]), np.asarray(ref["grad_definition"])
    assert fd.shape == gdef.shape == (64,)
    # two routes through the oracle: rank-one central differences of the
    # loss against the chain rule of grad_binned_cl (differences exact for a
    # quadratic loss up to FP64 rounding of the full a_lm)
    assert np.max(np.abs(fd - gdef)) <= 1e-6 * np.max(np.abs(fd))
