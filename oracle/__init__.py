"""FP64 CPU oracle for the direct point-catalog spherical-harmonic transform.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library: the transform itself is the
plain C loop in ``pointsht_oracle.c`` (Appendix A recurrences, Eq. alm_def);
the spectrum, shot-noise, binning and gradient steps below are plain NumPy in
FP64, each written from the definition it cites (arXiv:2312.12285).

Layout convention shared with the library's *interface* (not its code): a full
set of a_lm for 0 <= m <= l <= lmax is a packed m-major triangle,
``index(l, m) = m*(2*lmax+1-m)//2 + l``, complex128.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pointsht_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

FOUR_PI = 4.0 * np.pi


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, OpenMP, no FMA contraction) into _liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.oracle_pbar_scaled.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, ip]
            lib.oracle_pbar_scaled.restype = None
            lib.oracle_ylm.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp]
            lib.oracle_ylm.restype = None
            lib.oracle_alm.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_int, ctypes.c_int, ip, dp,
                                       ctypes.c_int]
            lib.oracle_alm.restype = ctypes.c_int
            lib.oracle_adjoint.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_int, dp, dp, ctypes.c_int]
            lib.oracle_adjoint.restype = ctypes.c_int
            lib.oracle_spin_lambda.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
            lib.oracle_spin_lambda.restype = None
            lib.oracle_alm_spin2.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp, ctypes.c_int, dp, dp, ctypes.c_int]
            lib.oracle_alm_spin2.restype = ctypes.c_int
            lib.oracle_alm_spin2_cols.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int, ip,
                                                  dp, dp, ctypes.c_int]
            lib.oracle_alm_spin2_cols.restype = ctypes.c_int
            lib.oracle_synthesis.argtypes = [ctypes.c_int64, dp, dp, ctypes.c_int, dp, dp, dp, ctypes.c_int]
            lib.oracle_synthesis.restype = ctypes.c_int
            lib.oracle_threej000.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_threej000.restype = ctypes.c_double
            lib.oracle_coupling.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int]
            lib.oracle_coupling.restype = ctypes.c_int
            lib.oracle_coupling_row.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp]
            lib.oracle_coupling_row.restype = ctypes.c_int
            lib.oracle_hermite_basis.argtypes = [ctypes.c_double, dp]
            lib.oracle_hermite_basis.restype = None
            lib.oracle_alm_interp.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int]
            lib.oracle_alm_interp.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def nmodes(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def index(l, m, lmax):
    """Packed m-major triangle index of (l, m)."""
    return m * (2 * lmax + 1 - m) // 2 + l


# ----------------------------------------------------------- App. A values --
def pbar_scaled(x: float, lmax: int, m: int):
    """Pbar_l^m(x), l = m..lmax (App. A), as (mantissa, exponent): value = mant * 2**expo."""
    lib = _load()
    n = lmax - m + 1
    mant = np.zeros(n, np.float64)
    expo = np.zeros(n, np.int32)
    lib.oracle_pbar_scaled(float(x), int(lmax), int(m), _dptr(mant),
                           expo.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return mant, expo


def pbar(x: float, lmax: int, m: int) -> np.ndarray:
    mant, expo = pbar_scaled(x, lmax, m)
    return np.ldexp(mant, expo)


def ylm(x: float, phi: float, lmax: int, m: int) -> np.ndarray:
    """Y_lm(theta, phi) for l = m..lmax at one point, complex128 (App. A; m >= 0)."""
    lib = _load()
    out = np.zeros(2 * (lmax - m + 1), np.float64)
    lib.oracle_ylm(float(x), float(phi), int(lmax), int(m), _dptr(out))
    return out[0::2] + 1j * out[1::2]


# ------------------------------------------------------ Eq. alm_def (a_lm) --
def alm(x, phi, w, lmax: int, mlist=None, nthreads: int = 0):
    """a_lm = sum_i w_i Y*_lm(n_i) (Eq. alm_def).

    With ``mlist=None`` returns the full packed triangle (complex128, length
    (lmax+1)(lmax+2)/2).  With a list of orders returns a dict m -> column
    (l = m..lmax, complex128).
    """
    lib = _load()
    x, phi, w = _f64(x), _f64(phi), _f64(w)
    n = x.shape[0]
    assert phi.shape[0] == n and w.shape[0] == n
    full = mlist is None
    ms = np.arange(lmax + 1, dtype=np.int32) if full else np.asarray(list(mlist), np.int32)
    total = int(sum(lmax - int(m) + 1 for m in ms))
    out = np.zeros(2 * total, np.float64)
    rc = lib.oracle_alm(n, _dptr(x), _dptr(phi), _dptr(w), int(lmax), len(ms),
                        ms.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(out), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_alm failed ({rc})")
    z = out[0::2] + 1j * out[1::2]
    if full:
        return z  # columns in m order are exactly the packed m-major triangle
    res, off = {}, 0
    for m in ms:
        ln = lmax - int(m) + 1
        res[int(m)] = z[off:off + ln]
        off += ln
    return res


def field_alm(cats, lmax: int, nthreads: int = 0):
    """a_lm of the FKP field sum_c coeff_c * (catalog c): Sec. 2.1, field n_g - alpha n_r.

    ``cats`` is a list of (x, phi, w, coeff); the catalogs are joined with
    signed weights coeff*w (the transform is linear in w).
    """
    x = np.concatenate([_f64(c[0]) for c in cats])
    phi = np.concatenate([_f64(c[1]) for c in cats])
    w = np.concatenate([_f64(c[2]) * float(c[3]) for c in cats])
    return alm(x, phi, w, lmax, nthreads=nthreads)


def adjoint(x, phi, g, lmax: int, nthreads: int = 0) -> np.ndarray:
    """d/dw_i of sum_lm Re(conj(g_lm) a_lm) = sum_lm lambda_lm(x_i) Re(g_lm e^{i m phi_i}).

    ``g`` is the packed triangle of dL/dRe(a) + i dL/dIm(a).
    """
    lib = _load()
    x, phi = _f64(x), _f64(phi)
    g = np.ascontiguousarray(np.asarray(g, np.complex128))
    assert g.shape[0] == nmodes(lmax)
    gi = np.empty(2 * g.shape[0], np.float64)
    gi[0::2], gi[1::2] = g.real, g.imag
    out = np.zeros(x.shape[0], np.float64)
    rc = lib.oracle_adjoint(x.shape[0], _dptr(x), _dptr(phi), int(lmax), _dptr(gi), _dptr(out),
                            int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_adjoint failed ({rc})")
    return out


# -------------------------------------------------- Eq. pseudoCl, shot noise --
def cl(alm_f, alm_g, lmax: int) -> np.ndarray:
    """Pseudo-C_l (Eq. pseudoCl) from m >= 0 coefficients.

    The sum over m = -l..l of a_lm^f conj(a_lm^g) uses Y_{l,-m} = (-1)^m Y*_lm
    with real weights, so a_{l,-m} = (-1)^m conj(a_lm):
    C_l = [Re(a_l0 conj b_l0) + 2 sum_{m>=1} Re(a_lm conj b_lm)] / (2l+1).
    """
    a = np.asarray(alm_f, np.complex128)
    b = np.asarray(alm_g, np.complex128)
    out = np.zeros(lmax + 1, np.float64)
    for m in range(lmax + 1):
        sl = slice(index(m, m, lmax), index(lmax, m, lmax) + 1)
        prod = (a[sl] * np.conj(b[sl])).real
        out[m:] += prod if m == 0 else 2.0 * prod
    out /= 2.0 * np.arange(lmax + 1) + 1.0
    return out


def shot_noise(w_signed) -> float:
    """Poisson noise of a weighted point field: sum_i (coeff_i w_i)^2 / 4pi.

    Follows from the addition theorem with P_l(1) = 1 (Sec. 2.1): for any point
    set, sum_m |sum_i w_i Y_lm(n_i)|^2 contains the i = j terms
    sum_i w_i^2 (2l+1)/4pi, i.e. a flat spectrum sum_i w_i^2 / 4pi.
    """
    w = _f64(w_signed)
    return float(np.sum(w * w) / FOUR_PI)


def bin_matrix(edges, lmax: int) -> np.ndarray:
    """theta_b^l = 1/Delta l for l in [e_b, e_{b+1}), zero otherwise (Sec. 2.1)."""
    edges = np.asarray(edges, np.int64)
    nb = len(edges) - 1
    th = np.zeros((nb, lmax + 1), np.float64)
    for b in range(nb):
        lo, hi = int(edges[b]), int(edges[b + 1])
        th[b, lo:hi] = 1.0 / (hi - lo)
    return th


def binned(cl_vec, edges, lmax: int) -> np.ndarray:
    """C_b = sum_l theta_b^l C_l (Sec. 2.1)."""
    return bin_matrix(edges, lmax) @ np.asarray(cl_vec, np.float64)


def grad_binned_cl(cats, lmax: int, edges, g_b, idx_per_cat, nthreads: int = 0):
    """d/dw_i of L = sum_b g_b C_b, C_b binned shot-noise-subtracted pseudo-C_l of one field.

    Definition-level chain rule (Eq. pseudoCl, Eq. alm_def, shot noise):
      dC_l/dw_i = (1/(2l+1)) sum_m c_m 2 Re(a_lm conj(da_lm/dw_i)) - dN/dw_i,
      da_lm/dw_i = coeff_i Y*_lm(n_i),  N = sum (coeff w)^2/4pi,
    with c_0 = 1, c_m = 2 (m > 0).  Returns one array of gradients per catalog
    for the requested object indices.
    """
    a = field_alm(cats, lmax, nthreads=nthreads)
    gl = bin_matrix(edges, lmax).T @ np.asarray(g_b, np.float64)  # sum_b g_b theta_b^l
    ms = np.concatenate([np.full(lmax - m + 1, m) for m in range(lmax + 1)])
    lidx = np.concatenate([np.arange(m, lmax + 1) for m in range(lmax + 1)])
    cm = np.where(ms == 0, 1.0, 2.0)
    # dL/dRe a + i dL/dIm a  for L = sum_l gl_l C_l(a)
    g_alm = (2.0 * gl[lidx] / (2.0 * lidx + 1.0) * cm) * a
    dn = float(np.sum(gl))  # dL/dN
    out = []
    for (x, phi, w, coeff), idx in zip(cats, idx_per_cat):
        idx = np.asarray(idx, np.int64)
        synth = adjoint(_f64(x)[idx], _f64(phi)[idx], g_alm, lmax, nthreads=nthreads)
        wi = _f64(w)[idx]
        out.append(float(coeff) * synth - dn * 2.0 * float(coeff) ** 2 * wi / FOUR_PI)
    return out


def rel_err_per_l(a, ref, lmax: int):
    """max over 1 <= l <= lmax of ||a_l. - ref_l.||_2 / ||ref_l.||_2 (rows over m)."""
    a = np.asarray(a, np.complex128)
    ref = np.asarray(ref, np.complex128)
    num = np.zeros(lmax + 1)
    den = np.zeros(lmax + 1)
    for m in range(lmax + 1):
        sl = slice(index(m, m, lmax), index(lmax, m, lmax) + 1)
        num[m:] += np.abs(a[sl] - ref[sl]) ** 2
        den[m:] += np.abs(ref[sl]) ** 2
    r = np.sqrt(num[1:] / np.maximum(den[1:], 1e-300))
    return float(np.max(r)) if lmax >= 1 else 0.0


# ------------------------------------------- interpolated transform (App.) --
def hermite_basis(t: float) -> np.ndarray:
    """Cubic Hermite basis c_0..c_3 at t in [0, 1] (App. "Interpolation")."""
    out = np.zeros(4, np.float64)
    _load().oracle_hermite_basis(float(t), _dptr(out))
    return out


def alm_interp(x, phi, w, lmax: int, ntheta: int, nthreads: int = 0):
    """a_lm by the paper's interpolation route with ntheta samples equispaced
    in theta (s_k = (k + 1/2) pi / ntheta, ghost samples continued across the
    poles): full packed triangle, complex128."""
    lib = _load()
    x, phi, w = _f64(x), _f64(phi), _f64(w)
    out = np.zeros(2 * nmodes(lmax), np.float64)
    rc = lib.oracle_alm_interp(x.shape[0], _dptr(x), _dptr(phi), _dptr(w), int(lmax), int(ntheta), _dptr(out),
                               int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_alm_interp failed ({rc})")
    return out[0::2] + 1j * out[1::2]


# ------------------------------------------------ point-evaluation synthesis --
def synthesis(x, phi, alm_t, lmax: int, return_imag: bool = False, nthreads: int = 0):
    """f(n_i) = sum_l sum_{m=-l}^{l} a_lm Y_lm(n_i) of the real field with
    m >= 0 coefficients alm_t (packed triangle), negative orders written out
    from a_{l,-m} = (-1)^m conj(a_lm), Y_{l,-m} = (-1)^m conj(Y_lm)."""
    lib = _load()
    x, phi = _f64(x), _f64(phi)
    a = np.ascontiguousarray(np.asarray(alm_t, np.complex128))
    assert a.shape[0] == nmodes(lmax)
    ai = np.empty(2 * a.shape[0], np.float64)
    ai[0::2], ai[1::2] = a.real, a.imag
    re = np.zeros(x.shape[0], np.float64)
    im = np.zeros(x.shape[0], np.float64)
    rc = lib.oracle_synthesis(x.shape[0], _dptr(x), _dptr(phi), int(lmax), _dptr(ai), _dptr(re), _dptr(im),
                              int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_synthesis failed ({rc})")
    return (re, im) if return_imag else re


# ------------------------------------- Eq. wldef, Eq. chat, mode decoupling --
def window_cl(w_alm, lmax: int, noise: float = 0.0) -> np.ndarray:
    """W_l = (1/(2l+1)) sum_m |w_lm|^2 (Eq. wldef) of the window's a_lm (the
    scaled randoms), minus an optional shot-noise constant (the footnote to
    Eq. wldef: subtract it when few randoms estimate the window)."""
    return cl(w_alm, w_alm, lmax) - noise


def threej000(l1: int, l2: int, l3: int) -> float:
    """(l1 l2 l3; 0 0 0) from its closed form (App. "Wigner 3j symbols")."""
    return float(_load().oracle_threej000(int(l1), int(l2), int(l3)))


def coupling(W, lmax: int, nthreads: int = 0) -> np.ndarray:
    """M_ll' of Eq. chat, [lmax+1, lmax+1] row-major, from W_0..W_{lmax_w}
    (lmax_w = len(W) - 1; W beyond it is taken as zero)."""
    W = _f64(W)
    M = np.empty((lmax + 1, lmax + 1), np.float64)
    rc = _load().oracle_coupling(int(lmax), W.shape[0] - 1, _dptr(W), _dptr(M), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_coupling failed ({rc})")
    return M


def coupling_row(W, lmax: int, l: int) -> np.ndarray:
    W = _f64(W)
    row = np.empty(lmax + 1, np.float64)
    rc = _load().oracle_coupling_row(int(lmax), W.shape[0] - 1, _dptr(W), int(l), _dptr(row))
    if rc != 0:
        raise RuntimeError(f"oracle_coupling_row failed ({rc})")
    return row


def binned_coupling(M, edges):
    """R[b, l'] = sum_l theta_b^l M_ll' (theta_b^l = 1/Delta l in bin b) and
    the binned coupling M_bb' = sum_{l' in b'} R[b, l'] (Sec. 2.1: the true
    C_l piecewise constant on the same bins)."""
    edges = np.asarray(edges, np.int64)
    lmax = M.shape[0] - 1
    T = bin_matrix(edges, lmax)
    R = T @ M
    nb = edges.size - 1
    Mbb = np.empty((nb, nb))
    for b2 in range(nb):
        Mbb[:, b2] = R[:, edges[b2]:edges[b2 + 1]].sum(axis=1)
    return R, Mbb


def decouple(Mbb, R, cl_binned):
    """Mode-decoupled bandpowers C~_b = sum_b' (M^-1)_bb' C^_b' (Eq.
    mode_coupling) and the window matrix cal M_bl' = sum_b' (M^-1)_bb' R[b', l']
    (Eq. expectation_value)."""
    Minv = np.linalg.inv(Mbb)
    return Minv, Minv @ R, np.asarray(cl_binned) @ Minv.T


def fkp_norm(W) -> float:
    """cal N = 1 / [sum_l' (2l'+1) W_l' / 4pi]: the normalisation that leaves a
    shot-noise spectrum unchanged (Sec. 2.1, the FKP-like alternative)."""
    W = np.asarray(W, np.float64)
    l = np.arange(W.size)
    return 1.0 / (np.sum((2 * l + 1) * W) / FOUR_PI)


# -------------------------------------------------- spin-2 (shear) transform --
def spin_lambda(x: float, lmax: int, m: int, n: int) -> np.ndarray:
    """lambda^(n)_lm(x) = sqrt((2l+1)/4pi) d^l_{m,n}(theta), l = 0..lmax (zero
    below max(m, |n|)); _{+2}Y*_lm = lambda^(-2) e^{-i m phi},
    _{-2}Y*_lm = lambda^(+2) e^{-i m phi}."""
    out = np.zeros(lmax + 1, np.float64)
    _load().oracle_spin_lambda(float(x), int(lmax), int(m), int(n), _dptr(out))
    return out


def alm_spin2(x, phi, w, g1, g2, lmax: int, nthreads: int = 0):
    """(E_lm, B_lm), packed triangles (complex128), of the spin-2 field
    (g1, g2) carried by weighted points: _{+-2}a = sum w (g1 +- i g2) _{+-2}Y*,
    E = -(_{2}a + _{-2}a)/2, B = i(_{2}a - _{-2}a)/2; zero for l < 2."""
    lib = _load()
    x, phi, w, g1, g2 = (_f64(v) for v in (x, phi, w, g1, g2))
    M = nmodes(lmax)
    E = np.zeros(2 * M, np.float64)
    B = np.zeros(2 * M, np.float64)
    rc = lib.oracle_alm_spin2(x.shape[0], _dptr(x), _dptr(phi), _dptr(w), _dptr(g1), _dptr(g2), int(lmax),
                              _dptr(E), _dptr(B), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_alm_spin2 failed ({rc})")
    return E[0::2] + 1j * E[1::2], B[0::2] + 1j * B[1::2]


def alm_spin2_cols(x, phi, w, g1, g2, lmax: int, mlist, nthreads: int = 0):
    """{m: (E column, B column)} over l = 0..lmax (zero below max(m, 2)) for
    the orders in mlist, summed over a fixed partition of the points."""
    lib = _load()
    x, phi, w, g1, g2 = (_f64(v) for v in (x, phi, w, g1, g2))
    ms = np.ascontiguousarray(np.asarray(mlist, np.int32))
    E = np.zeros(2 * ms.size * (lmax + 1), np.float64)
    B = np.zeros_like(E)
    rc = lib.oracle_alm_spin2_cols(x.shape[0], _dptr(x), _dptr(phi), _dptr(w), _dptr(g1), _dptr(g2), int(lmax),
                                   int(ms.size), ms.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(E), _dptr(B),
                                   int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_alm_spin2_cols failed ({rc})")
    E = (E[0::2] + 1j * E[1::2]).reshape(ms.size, lmax + 1)
    B = (B[0::2] + 1j * B[1::2]).reshape(ms.size, lmax + 1)
    return {int(m): (E[t], B[t]) for t, m in enumerate(ms)}
