"""PyTorch-facing calls of libpointsht.

Torch supplies device memory and streams; every arithmetic step runs in the
library's CUDA kernels through the C ABI (``include/pointsht.h``).  The
functions here only check tensors, allocate outputs/workspace with torch and
marshal pointers.  Complex gradients follow torch's convention
(dL/dRe + i dL/dIm), which is also the ABI's.
"""
from __future__ import annotations

import ctypes
import math
import threading
from dataclasses import dataclass

import torch

from . import _lib

_plans: dict = {}
_plans_lock = threading.Lock()


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Plan:
    """Recurrence tables for one lmax on one CUDA device (pointsht_plan)."""

    def __init__(self, lmax: int, device=None):
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if dev.type != "cuda":
            raise ValueError("libpointsht runs on CUDA devices only")
        self.lib = _lib.load()
        self.lmax = int(lmax)
        self.device = dev
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            _lib.check(self.lib.pointsht_plan_create(self.lmax, ctypes.byref(h)), "plan_create")
        self.handle = h

    @property
    def nmodes(self) -> int:
        return (self.lmax + 1) * (self.lmax + 2) // 2

    def check(self):
        """Raise if a kernel recorded an error (|x| > 1, non-finite input, timeout)."""
        with torch.cuda.device(self.device):
            _lib.check(self.lib.pointsht_plan_check(self.handle), "plan_check")

    def set_timing_events(self, start=None, stop=None):
        """Record torch.cuda.Event start/stop around the analysis kernel of each
        subsequent alm call (None, None clears)."""
        s = ctypes.c_void_p(start.cuda_event) if start is not None else None
        e = ctypes.c_void_p(stop.cuda_event) if stop is not None else None
        _lib.check(self.lib.pointsht_plan_set_timing_events(self.handle, s, e), "set_timing_events")

    def set_tuning(self, variant: int = 0, chunk_log2: int = 0):
        """FP32 analysis kernel variant and accumulation chunk size (0 = defaults)."""
        _lib.check(self.lib.pointsht_plan_set_tuning(self.handle, int(variant), int(chunk_log2)), "set_tuning")
        self.tuning = (int(variant), int(chunk_log2))

    def set_pole_threshold(self, pole_x: float):
        """Tiles of points all with |x| >= pole_x (one sign) run the near-pole
        form of the FP32 recurrence; above 1 turns it off."""
        _lib.check(self.lib.pointsht_plan_set_pole_threshold(self.handle, float(pole_x)), "set_pole_threshold")

    def set_skip_counters(self, counters=None):
        """counters: a zeroed int64 CUDA tensor of 2 entries (or None to turn
        off); FP32 analysis launches add skipped / all 16-step blocks."""
        ptr = None if counters is None else ctypes.c_void_p(counters.data_ptr())
        _lib.check(self.lib.pointsht_plan_set_skip_counters(self.handle, ptr), "set_skip_counters")

    def set_mixed_kernel(self, which: str = "mma.sync"):
        """Weight-column contraction kernel: "mma.sync" (default, faster) or
        "tcgen05" (= "tcgen05:8x32"; also "tcgen05:4x64", "tcgen05:2x128":
        producer warps x multipoles per stage)."""
        code = {"mma.sync": 0, "tcgen05": 1, "tcgen05:8x32": 1, "tcgen05:4x64": 2, "tcgen05:2x128": 3}[which]
        _lib.check(self.lib.pointsht_plan_set_mixed_kernel(self.handle, code), "set_mixed_kernel")

    def set_wait_probe(self, enable: bool):
        """Test hook: the first CTA of each analysis launch gives up a bounded
        wait on a barrier nothing arrives at (see pointsht.h)."""
        _lib.check(self.lib.pointsht_plan_set_wait_probe(self.handle, int(bool(enable))), "set_wait_probe")

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.pointsht_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def get_plan(lmax: int, device=None) -> Plan:
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    key = (dev.index if dev.index is not None else torch.cuda.current_device(), int(lmax))
    with _plans_lock:
        p = _plans.get(key)
        if p is None:
            p = Plan(lmax, torch.device("cuda", key[0]))
            _plans[key] = p
        return p


@dataclass
class Cat:
    """One catalog on the device: x = cos(theta), phi, weights, field index and
    coefficient (+1 data, -alpha randoms)."""
    x: torch.Tensor
    phi: torch.Tensor
    w: torch.Tensor
    field: int = 0
    coeff: float = 1.0


def _dtype(precision: str):
    return torch.float64 if precision == "fp64" else torch.float32


def _entries(cats, precision, device, weights=None):
    dt = _dtype(precision)
    out = []
    for i, c in enumerate(cats):
        w = c.w if weights is None else weights[i]
        for name, t in (("x", c.x), ("phi", c.phi), ("w", w)):
            if t.device != device or t.dtype != dt or not t.is_contiguous() or t.dim() != 1:
                raise ValueError(f"catalog {i}: {name} must be a contiguous 1-D {dt} tensor on {device}")
        if not (c.x.shape[0] == c.phi.shape[0] == w.shape[0]):
            raise ValueError(f"catalog {i}: x, phi, w lengths differ")
        out.append((c.x.data_ptr(), c.phi.data_ptr(), w.data_ptr(), c.x.shape[0], c.field, c.coeff))
    return out


def workspace_bytes(plan: Plan, cats, nfield: int, precision: str) -> int:
    arr, n = _lib.catalog_array(_entries(cats, precision, plan.device))
    size = plan.lib.pointsht_workspace_size(plan.handle, arr, n, nfield, _lib.PRECISIONS[precision])
    if size == 0:
        _lib.check(_lib.EINVAL, "workspace_size")
    return int(size)


def _workspace(plan, cats, nfield, precision, workspace):
    need = workspace_bytes(plan, cats, nfield, precision)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=plan.device)
    return workspace


def alm_raw(plan: Plan, cats, nfield: int = 1, precision: str = "fp32", out=None, workspace=None, stream=None,
            weights=None):
    """a_lm of each field (pointsht_alm): complex128 tensor [nfield, M]."""
    entries = _entries(cats, precision, plan.device, weights)
    arr, n = _lib.catalog_array(entries)
    workspace = _workspace(plan, cats, nfield, precision, workspace)
    if out is None:
        out = torch.empty((nfield, plan.nmodes), dtype=torch.complex128, device=plan.device)
    _lib.check(plan.lib.pointsht_alm(plan.handle, arr, n, nfield, _lib.PRECISIONS[precision], _ptr(out),
                                     _ptr(workspace), workspace.numel(), _stream_ptr(stream)), "alm")
    return out


def workspace_bytes_columns(plan: Plan, n: int, ncol: int, precision: str = "mixed") -> int:
    size = plan.lib.pointsht_workspace_size_columns(plan.handle, int(n), int(ncol), _lib.PRECISIONS[precision])
    if size == 0:
        _lib.check(_lib.EINVAL, "workspace_size_columns")
    return int(size)


def alm_columns(plan: Plan, x: torch.Tensor, phi: torch.Tensor, w: torch.Tensor, precision: str = "mixed", out=None,
                workspace=None, stream=None):
    """a_lm of F weight columns on one point set (pointsht_alm_columns).

    x, phi: float32 [n]; w: float32 [F, n] (row f = column f of the ABI);
    returns complex128 [F, M].  "mixed" runs the per-m contraction on the
    tensor cores, "fp32" the plain FP32 path with one field per column."""
    dev = plan.device
    for name, t in (("x", x), ("phi", phi), ("w", w)):
        if t.device != dev or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 tensor on {dev}")
    if w.dim() != 2 or x.dim() != 1 or phi.shape != x.shape or w.shape[1] != x.shape[0]:
        raise ValueError("expected x, phi of shape [n] and w of shape [F, n]")
    ncol, n = int(w.shape[0]), int(w.shape[1])
    need = workspace_bytes_columns(plan, n, ncol, precision)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    if out is None:
        out = torch.empty((ncol, plan.nmodes), dtype=torch.complex128, device=dev)
    _lib.check(plan.lib.pointsht_alm_columns(plan.handle, _ptr(x), _ptr(phi), _ptr(w), n, ncol,
                                             _lib.PRECISIONS[precision], _ptr(out), _ptr(workspace),
                                             workspace.numel(), _stream_ptr(stream)), "alm_columns")
    return out


def workspace_bytes_interp(plan: Plan, cats, nfield: int, ntheta: int) -> int:
    arr, n = _lib.catalog_array(_entries(cats, "fp32", plan.device))
    size = plan.lib.pointsht_workspace_size_interp(plan.handle, arr, n, nfield, int(ntheta))
    if size == 0:
        _lib.check(_lib.EINVAL, "workspace_size_interp")
    return int(size)


def default_ntheta(lmax: int) -> int:
    """16 samples per multipole (relative interpolation error ~1.5e-6), at most 32768."""
    return min(32768, 16 * lmax)


def ntheta_for_tolerance(lmax: int, cl_tol: float = 1e-4, safety: float = 4.0) -> int:
    """Samples in theta for a pseudo-C_l error budget, from the cubic Hermite
    spline's h^4 error (App. "Interpolation"): the C_l error measured at 16
    samples per multipole is ~4.3e-6 (lmax 2048, lognormal workload), so
    err(N) ~ 4.3e-6 (16 lmax / N)^4; N is the smallest even count with
    err(N) <= cl_tol / safety (10 lmax for the default 1e-4 / 4), at most
    32768."""
    ratio = (cl_tol / safety / 4.3e-6) ** 0.25
    n = int(math.ceil(16.0 * lmax / ratio))
    n += n & 1
    return max(2, min(32768, n))


def alm_interp(plan: Plan, cats, nfield: int = 1, ntheta=None, out=None, workspace=None, stream=None):
    """a_lm of each field by the interpolated route (pointsht_alm_interp):
    complex128 [nfield, M].  ntheta = samples in theta (None: default_ntheta)."""
    if ntheta is None:
        ntheta = default_ntheta(plan.lmax)
    arr, n = _lib.catalog_array(_entries(cats, "fp32", plan.device))
    need = workspace_bytes_interp(plan, cats, nfield, ntheta)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=plan.device)
    if out is None:
        out = torch.empty((nfield, plan.nmodes), dtype=torch.complex128, device=plan.device)
    _lib.check(plan.lib.pointsht_alm_interp(plan.handle, arr, n, nfield, int(ntheta), _ptr(out), _ptr(workspace),
                                            workspace.numel(), _stream_ptr(stream)), "alm_interp")
    return out


def shot_noise_raw(cats, nfield: int, precision: str, device, workspace=None, stream=None, weights=None):
    """Shot-noise matrix [nfield, nfield] (pointsht_shot_noise)."""
    lib = _lib.load()
    arr, n = _lib.catalog_array(_entries(cats, precision, device, weights))
    need = 512 * max(1, n) + 256
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=device)
    out = torch.empty((nfield, nfield), dtype=torch.float64, device=device)
    _lib.check(lib.pointsht_shot_noise(arr, n, nfield, _lib.PRECISIONS[precision], _ptr(out), _ptr(workspace),
                                       workspace.numel(), _stream_ptr(stream)), "shot_noise")
    return out


def cl_raw(alm: torch.Tensor, noise=None, stream=None):
    """Pseudo-C_l of every pair f <= g (pointsht_cl): float64 [npair, lmax+1]."""
    lib = _lib.load()
    nfield, M = alm.shape
    lmax = _lmax_of(M)
    npair = nfield * (nfield + 1) // 2
    out = torch.empty((npair, lmax + 1), dtype=torch.float64, device=alm.device)
    _lib.check(lib.pointsht_cl(lmax, _ptr(alm), nfield, _ptr(noise) if noise is not None else None, _ptr(out),
                               _stream_ptr(stream)), "cl")
    return out


def cl_backward_raw(alm, grad_cl, want_noise=True, stream=None):
    lib = _lib.load()
    nfield, M = alm.shape
    lmax = _lmax_of(M)
    galm = torch.empty_like(alm)
    gnoise = torch.empty((nfield, nfield), dtype=torch.float64, device=alm.device) if want_noise else None
    _lib.check(lib.pointsht_cl_backward(lmax, _ptr(alm), nfield, _ptr(grad_cl.contiguous()), _ptr(galm),
                                        _ptr(gnoise) if gnoise is not None else None, _stream_ptr(stream)),
               "cl_backward")
    return galm, gnoise


def bin_raw(cl: torch.Tensor, edges: torch.Tensor, stream=None):
    lib = _lib.load()
    nspec, n = cl.shape
    nbin = edges.shape[0] - 1
    out = torch.empty((nspec, nbin), dtype=torch.float64, device=cl.device)
    _lib.check(lib.pointsht_bin(n - 1, _ptr(cl), nspec, _ptr(edges), nbin, _ptr(out), _stream_ptr(stream)), "bin")
    return out


def bin_backward_raw(grad_b, edges, lmax, stream=None):
    lib = _lib.load()
    nspec, nbin = grad_b.shape
    out = torch.empty((nspec, lmax + 1), dtype=torch.float64, device=grad_b.device)
    _lib.check(lib.pointsht_bin_backward(lmax, _ptr(grad_b.contiguous()), nspec, _ptr(edges), nbin, _ptr(out),
                                         _stream_ptr(stream)), "bin_backward")
    return out


def synthesis(plan: Plan, x: torch.Tensor, phi: torch.Tensor, alm_t: torch.Tensor, precision: str = "fp32",
              out=None, workspace=None, stream=None) -> torch.Tensor:
    """f(n_i) = sum_{l, |m| <= l} a_lm Y_lm(n_i) of the real field with m >= 0
    coefficients alm_t (complex128 [M] or float64 [M, 2]), at the points
    (x, phi) (pointsht_synthesis)."""
    lib = _lib.load()
    dt = _dtype(precision)
    if x.dtype != dt or phi.dtype != dt or not x.is_cuda:
        raise TypeError(f"x and phi must be {dt} CUDA tensors")
    x, phi = x.contiguous(), phi.contiguous()
    a = alm_t
    if a.is_complex():
        a = torch.view_as_real(a.contiguous())
    a = a.contiguous()
    if a.dtype != torch.float64 or a.numel() != 2 * plan.nmodes:
        raise ValueError("alm must hold the plan's packed triangle in complex128")
    n = x.shape[0]
    need = lib.pointsht_workspace_size_synthesis(plan.handle, n, _lib.PRECISIONS[precision])
    if need == 0:
        _lib.check(_lib.EINVAL, "workspace_size_synthesis")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=x.device)
    if out is None:
        out = torch.empty(n, dtype=dt, device=x.device)
    _lib.check(lib.pointsht_synthesis(plan.handle, _ptr(x), _ptr(phi), n, _lib.PRECISIONS[precision], _ptr(a),
                                      _ptr(out), _ptr(workspace), workspace.numel(), _stream_ptr(stream)),
               "synthesis")
    return out


# ------------------------------------------------------------- spin 2 --
class ShearCat:
    """A catalog of a spin-2 field: float32 CUDA tensors x = cos(theta), phi,
    w and the two components g1, g2 at each point; its field and coefficient."""

    def __init__(self, x, phi, w, g1, g2, field: int = 0, coeff: float = 1.0):
        self.x, self.phi, self.w, self.g1, self.g2 = x, phi, w, g1, g2
        self.field, self.coeff = int(field), float(coeff)


def _shear_entries(cats):
    arr = (_lib.ShearCatalog * max(1, len(cats)))()
    keep = []
    for i, c in enumerate(cats):
        ts = [t.contiguous() for t in (c.x, c.phi, c.w, c.g1, c.g2)]
        for t in ts:
            if t.dtype != torch.float32 or not t.is_cuda:
                raise TypeError("shear catalog arrays must be float32 CUDA tensors")
        n = ts[0].shape[0]
        if any(t.shape[0] != n for t in ts):
            raise ValueError("shear catalog arrays differ in length")
        keep.extend(ts)
        arr[i] = _lib.ShearCatalog(*(t.data_ptr() if n else None for t in ts), n, c.field, 0, c.coeff)
    return arr, keep


def alm_spin2(plan: Plan, cats, nfield: int = 1, workspace=None, stream=None):
    """(E, B): complex128 [nfield, M] of the spin-2 field (g1, g2) carried by
    the catalogs (pointsht_alm_spin2)."""
    lib = _lib.load()
    arr, keep = _shear_entries(cats)
    need = lib.pointsht_workspace_size_spin2(plan.handle, arr, len(cats), nfield)
    if need == 0:
        _lib.check(_lib.EINVAL, "workspace_size_spin2")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=plan.device)
    E = torch.empty((nfield, plan.nmodes), dtype=torch.complex128, device=plan.device)
    B = torch.empty_like(E)
    _lib.check(lib.pointsht_alm_spin2(plan.handle, arr, len(cats), nfield, _ptr(E), _ptr(B), _ptr(workspace),
                                      workspace.numel(), _stream_ptr(stream)), "alm_spin2")
    del keep
    return E, B


# ------------------------------------------------------- mode coupling --
def _f64_dev(t: torch.Tensor, name: str) -> torch.Tensor:
    if t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    return t.contiguous()


def window_cl(plan: Plan, randoms, precision: str = "fp32", subtract_noise: bool = False, workspace=None,
              stream=None):
    """W_l (Eq. wldef) of the window traced by the scaled randoms (their Cat
    coeff = alpha): pointsht_alm on the randoms alone, then pointsht_cl, with
    their shot noise alpha^2 sum w^2 / 4pi subtracted if asked (for a window
    estimated from few randoms)."""
    cats = [Cat(c.x, c.phi, c.w, 0, c.coeff) for c in randoms]
    a = alm_raw(plan, cats, 1, precision, workspace=workspace, stream=stream)
    noise = shot_noise_raw(cats, 1, precision, a.device, stream=stream) if subtract_noise else None
    return cl_raw(a, noise, stream=stream)[0]


def coupling(W: torch.Tensor, lmax: int, workspace=None, stream=None) -> torch.Tensor:
    """M_ll' of Eq. chat, (lmax+1, lmax+1) float64, from W_0..W_{lmax_w}
    (pointsht_coupling)."""
    lib = _lib.load()
    W = _f64_dev(W, "W")
    need = lib.pointsht_workspace_size_coupling(int(lmax))
    if need == 0:
        _lib.check(_lib.EINVAL, "workspace_size_coupling")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=W.device)
    M = torch.empty((lmax + 1, lmax + 1), dtype=torch.float64, device=W.device)
    _lib.check(lib.pointsht_coupling(int(lmax), W.shape[0] - 1, _ptr(W), _ptr(M), _ptr(workspace), workspace.numel(),
                                     _stream_ptr(stream)), "coupling")
    return M


def coupling_binned(M: torch.Tensor, edges: torch.Tensor, stream=None):
    """(R, M_bb'): R[b, l'] = sum_l theta_b^l M_ll', M_bb' = sum_{l' in b'} R[b, l']
    (pointsht_coupling_binned)."""
    lib = _lib.load()
    M = _f64_dev(M, "M")
    L = M.shape[0] - 1
    nbin = edges.shape[0] - 1
    R = torch.empty((nbin, L + 1), dtype=torch.float64, device=M.device)
    Mbb = torch.empty((nbin, nbin), dtype=torch.float64, device=M.device)
    _lib.check(lib.pointsht_coupling_binned(L, _ptr(M), _ptr(edges.contiguous()), nbin, _ptr(R), _ptr(Mbb),
                                            _stream_ptr(stream)), "coupling_binned")
    return R, Mbb


def decouple(Mbb: torch.Tensor, R=None, cl_binned=None, stream=None):
    """(Minv, Mcal, cl_dec) of Eq. mode_coupling / Eq. expectation_value
    (pointsht_decouple); Mcal / cl_dec are None when R / cl_binned are."""
    lib = _lib.load()
    Mbb = _f64_dev(Mbb, "Mbb")
    nbin = Mbb.shape[0]
    dev = Mbb.device
    L = R.shape[1] - 1 if R is not None else 0
    need = lib.pointsht_workspace_size_decouple(nbin)
    if need == 0:
        _lib.check(_lib.EINVAL, "workspace_size_decouple")
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    Minv = torch.empty((nbin, nbin), dtype=torch.float64, device=dev)
    Mcal = torch.empty((nbin, L + 1), dtype=torch.float64, device=dev) if R is not None else None
    if R is not None:
        R = _f64_dev(R, "R")
    nspec = 0
    cl_dec = None
    if cl_binned is not None:
        cl_binned = _f64_dev(cl_binned, "cl_binned")
        nspec = cl_binned.shape[0]
        cl_dec = torch.empty((nspec, nbin), dtype=torch.float64, device=dev)
    _lib.check(lib.pointsht_decouple(L, nbin, _ptr(Mbb), _ptr(R) if R is not None else None,
                                     _ptr(cl_binned) if cl_binned is not None else None, nspec, _ptr(Minv),
                                     _ptr(Mcal) if Mcal is not None else None,
                                     _ptr(cl_dec) if cl_dec is not None else None, _ptr(ws), ws.numel(),
                                     _stream_ptr(stream)), "decouple")
    return Minv, Mcal, cl_dec


def fkp_normalise(W: torch.Tensor, R=None, cl_binned=None, stream=None):
    """(norm, Mprime, cl_norm): norm = 1 / [sum_l (2l+1) W_l / 4pi], Mprime =
    norm R, cl_norm = norm cl_binned (pointsht_fkp_normalise)."""
    lib = _lib.load()
    W = _f64_dev(W, "W")
    dev = W.device
    norm = torch.empty(1, dtype=torch.float64, device=dev)
    L, nbin, nspec = 0, 0, 0
    Mp = cn = None
    if R is not None:
        R = _f64_dev(R, "R")
        nbin, L = R.shape[0], R.shape[1] - 1
        Mp = torch.empty_like(R)
    if cl_binned is not None:
        cl_binned = _f64_dev(cl_binned, "cl_binned")
        nspec, nbin = cl_binned.shape
        cn = torch.empty_like(cl_binned)
    _lib.check(lib.pointsht_fkp_normalise(W.shape[0] - 1, _ptr(W), L, nbin, _ptr(R) if R is not None else None,
                                          _ptr(cl_binned) if cl_binned is not None else None, nspec, _ptr(norm),
                                          _ptr(Mp) if Mp is not None else None, _ptr(cn) if cn is not None else None,
                                          _stream_ptr(stream)), "fkp_normalise")
    return norm, Mp, cn


def combine_raw(alm_src, coef, noise_src=None, stream=None):
    """Linear combination of fields (pointsht_combine)."""
    lib = _lib.load()
    nsrc, M = alm_src.shape
    nout = coef.shape[0]
    out = torch.empty((nout, M), dtype=torch.complex128, device=alm_src.device)
    nout_t = torch.empty((nout, nout), dtype=torch.float64, device=alm_src.device) if noise_src is not None else None
    _lib.check(lib.pointsht_combine(_lmax_of(M), _ptr(alm_src), nsrc, _ptr(coef.contiguous()), nout,
                                    _ptr(noise_src) if noise_src is not None else None, _ptr(out),
                                    _ptr(nout_t) if nout_t is not None else None, _stream_ptr(stream)), "combine")
    return out, nout_t


def alm_backward_raw(plan, cats, nfield, precision, grad_alm, grad_noise=None, workspace=None, stream=None):
    """d L / d w for every catalog (pointsht_alm_backward)."""
    entries = _entries(cats, precision, plan.device)
    arr, n = _lib.catalog_array(entries)
    workspace = _workspace(plan, cats, nfield, precision, workspace)
    grads = [torch.empty_like(c.w) for c in cats]
    gw = (ctypes.c_void_p * max(1, len(grads)))(*[g.data_ptr() for g in grads])
    _lib.check(plan.lib.pointsht_alm_backward(plan.handle, arr, n, nfield, _lib.PRECISIONS[precision],
                                              _ptr(grad_alm.contiguous()),
                                              _ptr(grad_noise.contiguous()) if grad_noise is not None else None,
                                              gw, _ptr(workspace), workspace.numel(), _stream_ptr(stream)),
               "alm_backward")
    return grads


def _lmax_of(M: int) -> int:
    # (L+1)(L+2)/2 = M
    L = int(round(((8 * M + 1) ** 0.5 - 3) / 2))
    if (L + 1) * (L + 2) // 2 != M:
        raise ValueError(f"{M} is not a triangle size (L+1)(L+2)/2")
    return L


# -------------------------------------------------------------- autograd --
class PointSHT(torch.autograd.Function):
    """weights of every catalog -> (a_lm [nfield, M] complex128, shot-noise matrix).

    Backward runs the adjoint synthesis kernel (pointsht_alm_backward)."""

    @staticmethod
    def forward(ctx, plan, cats, nfield, precision, *weights):
        cats2 = [Cat(c.x, c.phi, w, c.field, c.coeff) for c, w in zip(cats, weights)]
        a = alm_raw(plan, cats2, nfield, precision)
        noise = shot_noise_raw(cats2, nfield, precision, plan.device)
        ctx.plan, ctx.cats, ctx.nfield, ctx.precision = plan, cats2, nfield, precision
        return a, noise

    @staticmethod
    def backward(ctx, grad_alm, grad_noise):
        if grad_alm is None:
            grad_alm = torch.zeros((ctx.nfield, ctx.plan.nmodes), dtype=torch.complex128, device=ctx.plan.device)
        grads = alm_backward_raw(ctx.plan, ctx.cats, ctx.nfield, ctx.precision, grad_alm, grad_noise)
        return (None, None, None, None, *grads)


class PseudoCl(torch.autograd.Function):
    """(a_lm [nfield, M], noise [nfield, nfield] or None) -> C_l [npair, lmax+1]."""

    @staticmethod
    def forward(ctx, alm, noise):
        ctx.save_for_backward(alm)
        ctx.has_noise = noise is not None
        return cl_raw(alm, noise)

    @staticmethod
    def backward(ctx, grad_cl):
        (alm,) = ctx.saved_tensors
        galm, gnoise = cl_backward_raw(alm, grad_cl, want_noise=ctx.has_noise)
        return galm, gnoise


class BinCl(torch.autograd.Function):
    """C_l [nspec, lmax+1] -> bandpowers [nspec, nbin] (theta_b^l = 1/Delta_l)."""

    @staticmethod
    def forward(ctx, cl, edges):
        ctx.save_for_backward(edges)
        ctx.lmax = cl.shape[1] - 1
        return bin_raw(cl, edges)

    @staticmethod
    def backward(ctx, grad_b):
        (edges,) = ctx.saved_tensors
        return bin_backward_raw(grad_b, edges, ctx.lmax), None


def alm(cats, lmax: int, nfield: int = 1, precision: str = "fp32", plan: Plan | None = None):
    """Differentiable a_lm and shot-noise matrix of the fields formed by ``cats``."""
    plan = plan or get_plan(lmax, cats[0].x.device if cats else None)
    return PointSHT.apply(plan, cats, nfield, precision, *[c.w for c in cats])


def pseudo_cl(alm_t, noise=None):
    return PseudoCl.apply(alm_t, noise)


def bin_cl(cl, edges):
    return BinCl.apply(cl, edges)


def binned_pseudo_cl(cats, lmax: int, edges: torch.Tensor, nfield: int = 1, precision: str = "fp32",
                     plan: Plan | None = None):
    """Shot-noise-subtracted binned pseudo-C_l, differentiable in the weights."""
    a, noise = alm(cats, lmax, nfield, precision, plan)
    return bin_cl(pseudo_cl(a, noise), edges)


# ------------------------------------------------------------ CUDA graphs --
class GraphStep:
    """Capture one call of ``fn`` (a function that only enqueues work through
    this library on the current stream, with fixed input buffers) into a CUDA
    graph and replay it.  ``fn`` is run ``warmup`` times first so that kernel
    attributes are configured outside the capture."""

    def __init__(self, fn, warmup: int = 2):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):
                fn()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.out = fn()

    def replay(self):
        self.graph.replay()
        return self.out


def make_pipeline(plan: Plan, cats, nsrc: int, precision: str = "fp32", coef=None, edges=None):
    """One pass of the hot path as a function of fixed device buffers, ready
    for CUDA-graph capture: a_lm of the ``nsrc`` source fields in one
    persistent launch, their shot-noise matrix, the optional combination into
    fields ``coef`` [nout, nsrc] (the FKP fields D_b - alpha_b R of a shared
    random catalog, Sec. 2.1), all auto and cross pseudo-C_l, and optional
    bandpowers.  Returns fn() -> (C_l [npair, lmax+1], C_b or None)."""
    dev = plan.device
    ws = torch.empty(workspace_bytes(plan, cats, nsrc, precision), dtype=torch.uint8, device=dev)
    a_buf = torch.empty((nsrc, plan.nmodes), dtype=torch.complex128, device=dev)
    nws = torch.empty(512 * max(1, len(cats)) + 256, dtype=torch.uint8, device=dev)
    coef = None if coef is None else coef.to(device=dev, dtype=torch.float64).contiguous()

    def fn():
        a = alm_raw(plan, cats, nsrc, precision, out=a_buf, workspace=ws)
        noise = shot_noise_raw(cats, nsrc, precision, dev, workspace=nws)
        if coef is not None:
            a, noise = combine_raw(a, coef, noise)
        cl = cl_raw(a, noise)
        cb = bin_raw(cl, edges) if edges is not None else None
        return cl, cb

    return fn
