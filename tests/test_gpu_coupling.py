"""Mode coupling on the GPU (pointsht_coupling, _binned, pointsht_decouple,
pointsht_fkp_normalise) against the oracle (Eq. chat, Sec. 2.1).

The GPU evaluates the squared 3j symbols through the central-binomial product
form and sums per anti-diagonal l + l'; the oracle takes the closed form
through long-double log-factorials and sums per entry.  Both are FP64, so
entries agree to ~1e-14 of the largest; the tests allow 1e-12."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2312_12285_gb300 import _lib, catalogs, ops  # noqa: E402

pytestmark = pytest.mark.gpu

FOUR_PI = 4.0 * np.pi


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def _window(Lw, seed, slope=1.5):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.2, 1.0, Lw + 1) / (1.0 + np.arange(Lw + 1)) ** slope


def _gpu_M(dev, W, L):
    M = ops.coupling(torch.from_numpy(W).to(dev), L)
    torch.cuda.synchronize()
    return M.cpu().numpy()


@pytest.mark.parametrize("L,Lw", [(0, 0), (1, 3), (37, 37), (100, 30), (100, 250), (600, 600)])
def test_coupling_matches_oracle(dev, L, Lw):
    """Small, ragged and window-wider-than-2L cases, and L = 600 (several CTAs
    per anti-diagonal)."""
    W = _window(Lw, 11 + L)
    got = _gpu_M(dev, W, L)
    ref = oracle.coupling(W, L)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_full_sky_identity(dev):
    W = np.zeros(101)
    W[0] = FOUR_PI
    got = _gpu_M(dev, W, 300)
    assert np.max(np.abs(got - np.eye(301))) <= 1e-13


def test_negative_window_entries(dev):
    """A window spectrum with its shot noise subtracted can go negative."""
    W = _window(64, 5) - 0.02
    got = _gpu_M(dev, W, 64)
    ref = oracle.coupling(W, 64)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_run_to_run_bitwise(dev):
    W = _window(200, 6)
    assert np.array_equal(_gpu_M(dev, W, 200), _gpu_M(dev, W, 200))


def test_fullsize_sampled_rows(dev):
    """lmax 2048 with a 2048-multipole window (the a_lm's own band limit):
    sampled rows, including the first, a middle and the last, against the
    oracle row by row."""
    L = 2048
    W = _window(L, 7)
    got = _gpu_M(dev, W, L)
    for l in (0, 1, 2, 701, 1500, 2047, 2048):
        ref = oracle.coupling_row(W, L, l)
        assert np.max(np.abs(got[l] - ref)) <= 1e-12 * np.max(np.abs(ref)), l


def test_fullsize_row_sums(dev):
    """lmax 2048, window to 512: every row l <= 1536 sees the whole window, so
    its sum is sum_lambda (2 lambda+1) W_lambda / 4pi (the constant-spectrum
    identity behind the FKP normalisation); also the symmetry of
    M_ll' / (2l'+1)."""
    L, Lw = 2048, 512
    W = _window(Lw, 8)
    got = _gpu_M(dev, W, L)
    target = np.sum((2 * np.arange(Lw + 1) + 1) * W) / FOUR_PI
    rows = got[: L - Lw + 1].sum(axis=1)
    assert np.max(np.abs(rows - target)) <= 1e-11 * target
    l = np.arange(L + 1)
    K = got / (2 * l[None, :] + 1)  # symmetric up to the rounding of the two scalings
    assert np.max(np.abs(K - K.T)) <= 4e-16 * np.max(np.abs(K))


def test_binned_decouple_normalise_match_oracle(dev):
    L = 96
    W = _window(40, 9)
    edges = np.array([2, 4, 8, 13, 21, 34, 55, 97], np.int32)
    M = torch.from_numpy(oracle.coupling(W, L)).to(dev)
    e_t = torch.from_numpy(edges).to(dev)
    R, Mbb = ops.coupling_binned(M, e_t)
    Rr, Mbbr = oracle.binned_coupling(M.cpu().numpy(), edges)
    assert np.max(np.abs(R.cpu().numpy() - Rr)) <= 1e-14 * np.max(np.abs(Rr))
    assert np.max(np.abs(Mbb.cpu().numpy() - Mbbr)) <= 1e-13 * np.max(np.abs(Mbbr))
    rng = np.random.default_rng(10)
    clb = rng.uniform(0.5, 2.0, (3, edges.size - 1))
    Minv, Mcal, dec = ops.decouple(Mbb, R, torch.from_numpy(clb).to(dev))
    Mi_r, Mcal_r, dec_r = oracle.decouple(Mbbr, Rr, clb)
    assert np.max(np.abs(Minv.cpu().numpy() - Mi_r)) <= 1e-11 * np.max(np.abs(Mi_r))
    assert np.max(np.abs(Mcal.cpu().numpy() - Mcal_r)) <= 1e-11 * np.max(np.abs(Mcal_r))
    assert np.max(np.abs(dec.cpu().numpy() - dec_r)) <= 1e-11 * np.max(np.abs(dec_r))
    norm, Mp, cn = ops.fkp_normalise(torch.from_numpy(W).to(dev), R, torch.from_numpy(clb).to(dev))
    nr = oracle.fkp_norm(W)
    assert abs(float(norm.cpu()[0]) - nr) <= 1e-14 * nr
    assert np.max(np.abs(Mp.cpu().numpy() - nr * Rr)) <= 1e-13 * np.max(np.abs(nr * Rr))
    assert np.max(np.abs(cn.cpu().numpy() - nr * clb)) <= 1e-14 * np.max(np.abs(nr * clb))


def test_piecewise_constant_spectrum_recovered(dev):
    """The whole GPU chain (coupling, binning, inverse, window matrix) gives
    cal M C = C_b for a true C_l constant on each bin (Eq. expectation_value)."""
    L = 128
    W = _window(60, 12)
    edges = np.array([2, 6, 12, 24, 48, 80, 129], np.int32)
    M = ops.coupling(torch.from_numpy(W).to(dev), L)
    R, Mbb = ops.coupling_binned(M, torch.from_numpy(edges).to(dev))
    Cb = np.random.default_rng(13).uniform(0.5, 2.0, edges.size - 1)
    C = np.zeros(L + 1)
    for b in range(edges.size - 1):
        C[edges[b]:edges[b + 1]] = Cb[b]
    _, Mcal, _ = ops.decouple(Mbb, R)
    assert np.max(np.abs(Mcal.cpu().numpy() @ C - Cb)) <= 1e-11 * np.max(Cb)


def test_singular_binned_matrix_gives_nan(dev):
    Mbb = torch.tensor([[1.0, 2.0], [2.0, 4.0]], dtype=torch.float64, device=dev)
    Minv, _, _ = ops.decouple(Mbb)
    assert torch.isnan(Minv).all()
    Z = torch.zeros((3, 3), dtype=torch.float64, device=dev)
    assert torch.isnan(ops.decouple(Z)[0]).all()


def test_window_from_randoms_end_to_end(dev):
    """W_l from the scaled randoms through the FP32 transform, then M_ll',
    against the oracle's W_l (FP64 transform of the same rounded points) and
    its M_ll'."""
    L = 64
    wl = catalogs.lognormal_cap(100, 20_000, 2 * L, config_id=21, nwaves=16, grid=(64, 128))
    r = wl.catalogs[1]
    alpha = 0.05
    cat = ops.Cat(torch.from_numpy(r.x).to(dev), torch.from_numpy(r.phi).to(dev), torch.from_numpy(r.w).to(dev),
                  0, alpha)
    plan = ops.get_plan(2 * L, dev)
    W = ops.window_cl(plan, [cat], "fp32", subtract_noise=True)
    M = ops.coupling(W, L).cpu().numpy()
    plan.check()
    a = oracle.alm(r.x.astype(np.float64), r.phi.astype(np.float64), alpha * r.w.astype(np.float64), 2 * L)
    noise = np.sum((alpha * r.w.astype(np.float64)) ** 2) / FOUR_PI
    Wr = oracle.window_cl(a, 2 * L, noise)
    tot = oracle.cl(a, a, 2 * L)
    assert np.max(np.abs(W.cpu().numpy() - Wr) / tot) <= 1e-5
    Mr = oracle.coupling(Wr, L)
    assert np.max(np.abs(M - Mr)) <= 1e-5 * np.max(np.abs(Mr))


def test_argument_errors(dev):
    lib = _lib.load()
    W = torch.ones(4, dtype=torch.float64, device=dev)
    with pytest.raises(_lib.PointSHTError):
        ops.coupling(W, 8193)
    assert lib.pointsht_workspace_size_coupling(-1) == 0
    assert lib.pointsht_workspace_size_decouple(0) == 0
    assert lib.pointsht_workspace_size_decouple(513) == 0
    with pytest.raises(_lib.PointSHTError):
        ops.coupling_binned(torch.eye(4, dtype=torch.float64, device=dev), torch.tensor([0], dtype=torch.int32,
                                                                                         device=dev))
