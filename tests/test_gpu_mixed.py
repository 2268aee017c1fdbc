"""Weight columns on one point set (pointsht_alm_columns), POINTSHT_MIXED:
lambda_lm from the FP32 recurrence, the per-m contraction on the tensor cores
with fp16 hi + lo operands, through both contraction kernels (warp-level
mma.sync, the default; tcgen05 with tensor-memory accumulators).

Tolerance: pseudo-C_l within 1e-4 of the FP64 oracle, relative to C_l before
shot-noise subtraction (the mixed-path target; error metric of the C_l
comparison: max over 1 <= l <= lmax).  The a_lm rows are held to the same 1e-4.
The split itself contributes about 2^-22 per product (lo x lo dropped, lo
rounded to fp16), far below the FP32 recurrence error, so the mixed and plain
FP32 paths agree to the FP32 level.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2312_12285_gb300 import _lib, catalogs, ops  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_CL = 1e-4


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def _cl_err(a, ref, L):
    c = oracle.cl(a, a, L)
    r = oracle.cl(ref, ref, L)
    return float(np.max(np.abs(c[1:] - r[1:]) / r[1:]))


KERNELS = ["tcgen05", "mma.sync"]


def _columns(dev, x, phi, W, L, precision="mixed", kernel="mma.sync"):
    plan = ops.get_plan(L, dev)
    plan.set_mixed_kernel(kernel)
    try:
        out = ops.alm_columns(plan, torch.from_numpy(x).to(dev), torch.from_numpy(phi).to(dev),
                              torch.from_numpy(np.ascontiguousarray(W)).to(dev), precision)
        torch.cuda.synchronize()
        plan.check()
    finally:
        plan.set_mixed_kernel("mma.sync")
    return out.cpu().numpy()


NONZERO = (0, 1, 2, 3, 5, 6, 7, 8, 9)


@pytest.fixture(scope="module", params=KERNELS)
def small(dev, request):
    """25 000 points (24 full tiles and a ragged one) at lmax 256, ten columns
    (two passes: 8 columns, then 2 with the 4-column kernel): the signed FKP
    field, plain weights, weights of order 1e-6 and 1e5 (column scaling), all
    zeros, galaxies only, and four jackknife columns of the FKP field."""
    L = 256
    wl = catalogs.lognormal_cap(2_500, 22_500, L, config_id=31, nwaves=64, grid=(128, 256))
    x, phi, Wj = catalogs.weight_columns(wl, 5)
    n = x.shape[0]
    assert n == 25_000
    rng = catalogs.rng_for(31, 5)
    ng = wl.catalogs[0].n
    W = np.zeros((10, n), np.float32)
    W[0] = Wj[0]
    W[1] = rng.uniform(0.8, 1.2, n)
    W[2] = rng.uniform(0.0, 1.0, n) * 1e-6
    W[3] = rng.standard_normal(n) * 1e5
    W[5, :ng] = wl.catalogs[0].w
    W[6:10] = Wj[1:5]
    kernel = request.param
    got = _columns(dev, x, phi, W, L, kernel=kernel)
    x64, p64 = x.astype(np.float64), phi.astype(np.float64)
    ref = [oracle.alm(x64, p64, W[f].astype(np.float64), L) if f in NONZERO else None for f in range(10)]
    return L, x, phi, W, got, ref, kernel


@pytest.mark.parametrize("shape", ["tcgen05:4x64", "tcgen05:2x128"])
def test_tcgen05_other_shapes(dev, shape):
    """The tcgen05 kernel's other producer / stage shapes (4 warps x 64
    multipoles, 2 x 128) on 6 000 points (several tiles of their 256 and 128
    points and a ragged last one) at lmax 200 with five columns, against the
    oracle."""
    L = 200
    wl = catalogs.lognormal_cap(600, 5_400, L, config_id=33, nwaves=64, grid=(128, 256))
    x, phi, W = catalogs.weight_columns(wl, 5)
    got = _columns(dev, x, phi, W, L, kernel=shape)
    x64, p64 = x.astype(np.float64), phi.astype(np.float64)
    for f in range(5):
        ref = oracle.alm(x64, p64, W[f].astype(np.float64), L)
        assert oracle.rel_err_per_l(got[f], ref, L) <= TOL_CL, f
        assert _cl_err(got[f], ref, L) <= TOL_CL, f


def test_mixed_matches_oracle(small):
    L, _, _, _, got, ref, _ = small
    for f in NONZERO:
        assert oracle.rel_err_per_l(got[f], ref[f], L) <= TOL_CL, f
        assert _cl_err(got[f], ref[f], L) <= TOL_CL, f


def test_zero_column_is_exactly_zero(small):
    _, _, _, _, got, _, _ = small
    assert np.all(got[4] == 0)


def test_mixed_matches_plain_fp32_columns(small, dev):
    L, x, phi, W, got, _, _ = small
    f32 = _columns(dev, x, phi, W, L, "fp32")
    for f in NONZERO:
        assert _cl_err(got[f], f32[f], L) <= TOL_CL, f


@pytest.mark.parametrize("cols", [[5], [0, 5, 9], [1, 2, 3, 5, 6]])
def test_column_result_independent_of_pass_shape(small, dev, cols):
    """A column gives the same a_lm (to FP32 accumulation rounding) whether it
    runs alone, in a 4-column pass or in an 8-column pass."""
    L, x, phi, W, got, _, kernel = small
    g = _columns(dev, x, phi, W[cols], L, kernel=kernel)
    for j, f in enumerate(cols):
        assert oracle.rel_err_per_l(g[j], got[f], L) <= 1e-6, f


def test_power_of_two_scaling_is_exact(small, dev):
    """Columns are rescaled by powers of two only: in the same pass layout,
    w * 2^20 gives exactly 2^20 times the a_lm of w (and w * 2^-30 exactly
    2^-30 times), and the other columns are unchanged bit for bit."""
    L, x, phi, W, got, _, kernel = small
    W2 = W.copy()
    W2[1] *= np.float32(2.0 ** 20)
    W2[6] *= np.float32(2.0 ** -30)
    g2 = _columns(dev, x, phi, W2, L, kernel=kernel)
    assert np.array_equal(g2[1], got[1] * 2.0 ** 20)
    assert np.array_equal(g2[6], got[6] * 2.0 ** -30)
    for f in (0, 2, 3, 4, 5, 7, 8, 9):
        assert np.array_equal(g2[f], got[f]), f


def test_run_to_run_bitwise(small, dev):
    L, x, phi, W, got, _, kernel = small
    again = _columns(dev, x, phi, W, L, kernel=kernel)
    assert np.array_equal(again, got)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("n,L", [(5, 64), (1024, 97), (3001, 33), (2049, 1)])
def test_ragged_sizes_and_odd_lmax(dev, n, L, kernel):
    rng = catalogs.rng_for(32, n)
    x = rng.uniform(-1, 1, n).astype(np.float32)
    phi = rng.uniform(0, 2 * np.pi, n).astype(np.float32)
    W = np.stack([rng.uniform(0.5, 1.5, n), rng.standard_normal(n)]).astype(np.float32)
    got = _columns(dev, x, phi, W, L, kernel=kernel)
    for f in range(2):
        ref = oracle.alm(x.astype(np.float64), phi.astype(np.float64), W[f].astype(np.float64), L)
        assert oracle.rel_err_per_l(got[f], ref, L) <= TOL_CL
        assert np.linalg.norm(got[f] - ref) <= TOL_CL * np.linalg.norm(ref)


@pytest.mark.parametrize("kernel", KERNELS)
def test_empty_point_set(dev, kernel):
    e = np.zeros(0, np.float32)
    got = _columns(dev, e, e, np.zeros((3, 0), np.float32), 40, kernel=kernel)
    assert got.shape == (3, oracle.nmodes(40)) and np.all(got == 0)


@pytest.mark.parametrize("kernel", KERNELS)
def test_single_point_at_the_pole(dev, kernel):
    """x = 1: a_lm = 0 for m > 0 and a_l0 = w sqrt((2l+1)/4pi) (Y_lm at the pole)."""
    L = 200
    got = _columns(dev, np.ones(1, np.float32), np.full(1, 0.7, np.float32), np.full((1, 1), 1.5, np.float32), L,
                   kernel=kernel)[0]
    l = np.arange(L + 1)
    assert np.all(got[oracle.index(1, 1, L):] == 0)
    np.testing.assert_allclose(got[:L + 1].real, 1.5 * np.sqrt((2 * l + 1) / (4 * np.pi)), rtol=3e-4)
    assert np.all(got[:L + 1].imag == 0)


def test_out_of_range_point_is_flagged(dev):
    L = 16
    plan = ops.get_plan(L, dev)
    x = torch.tensor([0.5, 1.5, -0.2], dtype=torch.float32, device=dev)
    phi = torch.zeros(3, dtype=torch.float32, device=dev)
    w = torch.ones((1, 3), dtype=torch.float32, device=dev)
    ops.alm_columns(plan, x, phi, w, "mixed")
    torch.cuda.synchronize()
    with pytest.raises(_lib.PointSHTError) as ei:
        plan.check()
    assert ei.value.status == _lib.ERANGE


def test_argument_errors(dev):
    x = torch.zeros(8, dtype=torch.float32, device=dev)
    w = torch.ones((1, 8), dtype=torch.float32, device=dev)
    with pytest.raises(_lib.PointSHTError) as ei:
        ops.alm_columns(ops.get_plan(4097, dev), x, x, w, "mixed")  # beyond the FP32 recurrence's range
    assert ei.value.status == _lib.EINVAL and "lmax" in str(ei.value)
    with pytest.raises(_lib.PointSHTError):
        ops.alm_columns(ops.get_plan(32, dev), x, x, w, "fp64")


# ------------------------------------------------------------------ full size --
@pytest.fixture(scope="module")
def full(dev):
    """The lmax-2048 workload (1e6 galaxies + 9e6 randoms in the cap mask) with
    four jackknife columns, in the launch configuration bench.py times."""
    wl = catalogs.config(3)
    x, phi, W = catalogs.weight_columns(wl, 4)
    assert x.shape[0] == 10_000_000 and wl.lmax == 2048
    return wl.lmax, x, phi, W, _columns(dev, x, phi, W, wl.lmax)


def test_fullsize_sampled_columns(full):
    """Short columns m = 1900, 2047, 2048 (seeds deepest below the FP32 range)
    of every weight column, over all 1e7 points, and the long columns m = 0, 1
    of the FKP column, which carry the points next to the cap's pole, where the
    mixed path runs the standard FP32 recurrence (6e-5 measured for m = 0,
    against 1.3e-6 for the FP32 path with its near-pole form): the mixed
    path's 1e-4."""
    L, x, phi, W, got = full
    x64, p64 = x.astype(np.float64), phi.astype(np.float64)
    for f in range(W.shape[0]):
        ref = oracle.alm(x64, p64, W[f].astype(np.float64), L, mlist=[1900, 2047, 2048])
        for m, col in ref.items():
            g = got[f][oracle.index(m, m, L):oracle.index(L, m, L) + 1]
            assert np.linalg.norm(g - col) <= TOL_CL * np.linalg.norm(col), (f, m)
    ref = oracle.alm(x64, p64, W[0].astype(np.float64), L, mlist=[0, 1])
    for m, col in ref.items():
        g = got[0][oracle.index(m, m, L):oracle.index(L, m, L) + 1]
        assert np.linalg.norm(g - col) <= TOL_CL * np.linalg.norm(col), m


def test_fullsize_low_l_pseudo_cl(full):
    """C_l for 1 <= l <= 32 of the FKP column and one jackknife column: the
    oracle transforms all 1e7 points to lmax 32 (a_lm for l <= 32 does not
    depend on lmax)."""
    L, x, phi, W, got = full
    Ls = 32
    x64, p64 = x.astype(np.float64), phi.astype(np.float64)
    for f in (0, 2):
        ref = oracle.alm(x64, p64, W[f].astype(np.float64), Ls)
        sub = np.concatenate([got[f][oracle.index(m, m, L):oracle.index(Ls, m, L) + 1] for m in range(Ls + 1)])
        assert _cl_err(sub, ref, Ls) <= TOL_CL, f


def test_fullsize_linearity_across_columns(full, dev):
    """a_lm is linear in the weights: with jackknife columns built from
    disjoint wedges, sum_k (w0 - w_k) = w0, so sum_k (a_0 - a_k) = a_0 over
    the whole triangle (holds at any size)."""
    L, x, phi, W, got = full
    nw = W.shape[0] - 1
    lhs = nw * got[0] - got[1:].sum(axis=0)
    assert np.linalg.norm(lhs - got[0]) <= 1e-5 * np.linalg.norm(got[0]) * nw
