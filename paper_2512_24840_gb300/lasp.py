"""Python binding of liblasp.so (argument marshalling only).

Every call goes through the C-ABI declared in include/lasp.h; all arithmetic
of the fit runs in the library's CUDA kernels.  PyTorch provides device
memory (tensors whose data pointers are passed down) and streams.  There is
no CPU fallback: if the library cannot be loaded or no sm_103 device is
present, the calls raise.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np
import torch

from . import _build

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EGRID, ENODEV, EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
ST_CONV_TOL, ST_CONV_RISE, ST_MAXSTEPS, ST_NONPOS = 1, 2, 4, 8
ST_NONFINITE, ST_SINGULAR, ST_NODATA, ST_RUNNING = 16, 32, 64, 128
ST_TIMEOUT = 256
PREC = {"fp32": 0, "tf32": 1, "bf16": 2, "tf32x3": 3}
OPTIMIZER = {"adam": 0, "lm": 1}
LOSS_MODE = {"separable": 0, "joint": 1}

_lock = threading.Lock()
_lib = None


class LaspError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class InterpDesc(ct.Structure):
    _fields_ = [("K", ct.c_int), ("n_pix", ct.c_int), ("pad", ct.c_int), ("dln", ct.c_double),
                ("exps", ct.c_void_p), ("basis_lo", ct.c_double * 3),
                ("basis_hi", ct.c_double * 3), ("box_lo", ct.c_double * 5),
                ("box_hi", ct.c_double * 5)]


class PiecewiseDesc(ct.Structure):
    _fields_ = [("n_reg", ct.c_int), ("K", ct.c_int * 3), ("n_pix", ct.c_int), ("pad", ct.c_int),
                ("dln", ct.c_double), ("exps", ct.c_void_p),
                ("basis_lo", (ct.c_double * 3) * 3), ("basis_hi", (ct.c_double * 3) * 3),
                ("teff_blend", ct.c_double * 4), ("box_lo", ct.c_double * 5),
                ("box_hi", ct.c_double * 5)]


class Batch(ct.Structure):
    _fields_ = [("N", ct.c_int), ("n_pix", ct.c_int), ("flux", ct.c_void_p),
                ("ivar", ct.c_void_p), ("good", ct.c_void_p), ("theta0", ct.c_void_p)]


class FitOpts(ct.Structure):
    _fields_ = [("lr", ct.c_float), ("beta1", ct.c_float), ("beta2", ct.c_float),
                ("eps", ct.c_float), ("tol", ct.c_float), ("window", ct.c_int),
                ("max_steps", ct.c_int), ("legendre_deg", ct.c_int), ("edge_px", ct.c_int),
                ("quantile", ct.c_float), ("precision", ct.c_int), ("fp64_normal_eq", ct.c_int),
                ("clean", ct.c_int), ("clean_every", ct.c_int), ("clean_max", ct.c_int),
                ("optimizer", ct.c_int), ("loss_mode", ct.c_int)]


class Result(ct.Structure):
    _fields_ = [("theta", ct.c_void_p), ("loss", ct.c_void_p), ("steps", ct.c_void_p),
                ("status", ct.c_void_p), ("cont_coeff", ct.c_void_p), ("weight", ct.c_void_p)]


EXPORTS = ["lasp_init_interp", "lasp_free_interp", "lasp_default_opts", "lasp_fit_batch",
           "lasp_errors", "lasp_forward", "lasp_backward", "lasp_interp_eval",
           "lasp_last_launches", "lasp_strerror", "lasp_version", "lasp_resample_linear",
           "lasp_slots_create", "lasp_slots_free", "lasp_slots_admit", "lasp_slots_step",
           "lasp_slots_step_running",
           "lasp_slots_fetch", "lasp_interp_eval_static", "lasp_clean_mask",
           "lasp_init_interp_piecewise", "lasp_server_create", "lasp_server_destroy",
           "lasp_server_submit", "lasp_server_submit_n", "lasp_server_tick", "lasp_server_poll",
           "lasp_server_pending",
           "lasp_test_wait_limit", "lasp_profile", "lasp_profile_read"]


def library_path() -> str:
    return _build.LIB


def load(build: bool = False):
    """Load liblasp.so (building it first when build=True)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build()")
        lib = ct.CDLL(path)
        P, I = ct.c_void_p, ct.c_int
        lib.lasp_init_interp.argtypes = [P, P, P]
        lib.lasp_init_interp.restype = I
        lib.lasp_init_interp_piecewise.argtypes = [P, P, P]
        lib.lasp_init_interp_piecewise.restype = I
        lib.lasp_server_create.argtypes = [I, P, P, P, P, I, P]
        lib.lasp_server_create.restype = I
        lib.lasp_server_destroy.argtypes = [P]
        lib.lasp_server_submit.argtypes = [P, I, P, P, P, P, ct.c_int64]
        lib.lasp_server_submit.restype = I
        lib.lasp_server_submit_n.argtypes = [P, I, I, P, P, P, P, P, P]
        lib.lasp_server_submit_n.restype = I
        lib.lasp_server_tick.argtypes = [P, P]
        lib.lasp_server_tick.restype = I
        lib.lasp_server_poll.argtypes = [P, P, I, P]
        lib.lasp_server_poll.restype = I
        lib.lasp_server_pending.argtypes = [P, P]
        lib.lasp_server_pending.restype = I
        lib.lasp_free_interp.argtypes = [P]
        lib.lasp_default_opts.argtypes = [P]
        lib.lasp_fit_batch.argtypes = [P, P, P, P, P]
        lib.lasp_fit_batch.restype = I
        lib.lasp_errors.argtypes = [P, P, P, P, P, P, P, P]
        lib.lasp_errors.restype = I
        lib.lasp_forward.argtypes = [P, I, P, P, I, P, P]
        lib.lasp_forward.restype = I
        lib.lasp_backward.argtypes = [P, I, P, P, I, P, P, P, P]
        lib.lasp_backward.restype = I
        lib.lasp_interp_eval.argtypes = [P, I, P, P, I, P]
        lib.lasp_interp_eval.restype = I
        lib.lasp_last_launches.restype = I
        lib.lasp_strerror.argtypes = [I]
        lib.lasp_strerror.restype = ct.c_char_p
        lib.lasp_version.restype = I
        D = ct.c_double
        lib.lasp_resample_linear.argtypes = [I, I, D, D, P, I, D, D, P, P]
        lib.lasp_resample_linear.restype = I
        lib.lasp_clean_mask.argtypes = [I, I, P, P, P, ct.c_float, P, P, P]
        lib.lasp_clean_mask.restype = I
        lib.lasp_test_wait_limit.argtypes = [I]
        lib.lasp_test_wait_limit.restype = I
        lib.lasp_profile.argtypes = [I]
        lib.lasp_profile.restype = I
        lib.lasp_profile_read.argtypes = [P, I, P]
        lib.lasp_profile_read.restype = I
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().lasp_strerror(int(code)).decode()
    except Exception:
        return "unknown"


def _check(code, what):
    if code != OK:
        raise LaspError(code, what)


def _ptr(t):
    return None if t is None else ct.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ct.c_void_p(s.cuda_stream)


def _dev(t, dtype):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"expected a contiguous CUDA {dtype} tensor")
    return t


def _arg(t, dtype, shape, name):
    """Dtype and shape (None matches any extent) of a tensor argument, checked
    before its pointer reaches the library, which sizes every buffer from N
    and the grid."""
    if not isinstance(t, torch.Tensor) or t.dtype != dtype:
        raise TypeError(f"{name}: expected a {dtype} tensor")
    if t.dim() != len(shape) or any(n is not None and t.shape[k] != n for k, n in enumerate(shape)):
        want = "x".join("*" if n is None else str(n) for n in shape)
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {want}")
    return t


def _on_device(**ts):
    """The tensors of one call: contiguous, on CUDA and on one device (the
    kernels run on the current device)."""
    for name, t in ts.items():
        if t is not None and not (t.is_cuda and t.is_contiguous()):
            raise TypeError(f"{name}: expected a contiguous CUDA tensor")
    devs = {t.device for t in ts.values() if t is not None}
    if len(devs) > 1:
        raise ValueError(f"tensor arguments on several devices: {sorted(str(d) for d in devs)}")


def default_opts(**kw) -> FitOpts:
    o = FitOpts()
    load().lasp_default_opts(ct.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PREC[v]
        if k == "optimizer" and isinstance(v, str):
            v = OPTIMIZER[v]
        if k == "loss_mode" and isinstance(v, str):
            v = LOSS_MODE[v]
        if not hasattr(o, k):
            raise TypeError(f"unknown fit option {k}")
        setattr(o, k, v)
    return o


def last_launches() -> int:
    return int(load().lasp_last_launches())


class KernelTime(ct.Structure):
    _fields_ = [("name", ct.c_char * 48), ("launches", ct.c_int32), ("ms", ct.c_double)]


def profile(on: bool) -> None:
    """Per-kernel device timing on (calls become synchronous) or off."""
    _check(load().lasp_profile(1 if on else 0), "lasp_profile")


def profile_read() -> dict:
    """{kernel name: (launches, total ms)} since the last read; clears it."""
    buf = (KernelTime * 64)()
    n = ct.c_int()
    _check(load().lasp_profile_read(buf, 64, ct.byref(n)), "lasp_profile_read")
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].ms)) for i in range(n.value)}


def test_wait_limit(polls: int) -> None:
    """Testing hook: the first table-copy wait of every CTA of the tensor-core
    kernels launched from now on gives up after `polls` polls (< 0: normal)."""
    _check(load().lasp_test_wait_limit(int(polls)), "lasp_test_wait_limit")


def resample_linear(coeff_lin, lam1, dlam, n_out, ln_lam0, dln, stream=None):
    """Flux-conserving resampling (Eqs. 2-4) of table rows (device K x q,
    linear grid lam1 + k dlam) onto the ln grid exp(ln_lam0 + i dln)."""
    _dev(coeff_lin, torch.float32)
    K, q = coeff_lin.shape
    out = torch.empty((K, int(n_out)), device=coeff_lin.device)
    _check(load().lasp_resample_linear(K, q, float(lam1), float(dlam), _ptr(coeff_lin), int(n_out),
                                       float(ln_lam0), float(dln), _ptr(out), _stream(stream)),
           "lasp_resample_linear")
    return out


def clean_mask(r, m, used, fshift, stream=None):
    """Clean outlier mask (stage 6, Eq. 8) of N spectra: device float32 r, m
    (N x p) and uint8 used; returns (keep uint8 N x p, k int32 N)."""
    _dev(r, torch.float32), _dev(m, torch.float32), _dev(used, torch.uint8)
    N, p = r.shape
    keep = torch.empty((N, p), dtype=torch.uint8, device=r.device)
    k = torch.empty(N, dtype=torch.int32, device=r.device)
    _check(load().lasp_clean_mask(N, p, _ptr(r), _ptr(m), _ptr(used), float(fshift), _ptr(keep),
                                  _ptr(k), _stream(stream)), "lasp_clean_mask")
    return keep, k


class Interp:
    """Device-resident interpolator (Eq. 1 table) on one ln-lambda grid."""

    def __init__(self, C, exps, n_pix, pad, dln, basis_lo, basis_hi, box_lo, box_hi):
        lib = load()
        C = np.ascontiguousarray(C, dtype=np.float32)
        self._exps = np.ascontiguousarray(exps, dtype=np.int8)
        K = self._exps.shape[0]
        if C.shape != (K, n_pix + 2 * pad):
            raise ValueError("table shape must be K x (n_pix + 2 pad)")
        d = InterpDesc(K, int(n_pix), int(pad), float(dln), self._exps.ctypes.data,
                       (ct.c_double * 3)(*basis_lo), (ct.c_double * 3)(*basis_hi),
                       (ct.c_double * 5)(*box_lo), (ct.c_double * 5)(*box_hi))
        h = ct.c_void_p()
        _check(lib.lasp_init_interp(ct.byref(d), C.ctypes.data, ct.byref(h)), "lasp_init_interp")
        self._h = h
        self.K, self.n_pix, self.pad = K, int(n_pix), int(pad)
        self.n_model = self.n_pix + 2 * self.pad
        self.dln = float(dln)
        self.box_lo, self.box_hi = np.asarray(box_lo, float), np.asarray(box_hi, float)

    @classmethod
    def piecewise(cls, tables, exps, n_pix, pad, dln, basis_lo, basis_hi, teff_blend, box_lo,
                  box_hi):
        """Interpolator with Teff regimes (Eq. 1 with f1..f5): tables[r] (K_r x
        n_model) and exps[r] (K_r x 3) per regime, coolest first, each with its
        basis box basis_lo[r], basis_hi[r]; regimes r and r+1 blend linearly in
        Teff on (teff_blend[2r], teff_blend[2r+1]]."""
        lib = load()
        n_reg = len(tables)
        Ks = [int(np.asarray(e).shape[0]) for e in exps]
        C = np.ascontiguousarray(np.concatenate([np.asarray(t, np.float32) for t in tables]), np.float32)
        E = np.ascontiguousarray(np.concatenate([np.asarray(e, np.int8) for e in exps]), np.int8)
        if C.shape != (sum(Ks), int(n_pix) + 2 * int(pad)):
            raise ValueError("each table must be K_r x (n_pix + 2 pad)")
        tb = list(teff_blend) + [0.0] * (4 - len(teff_blend))
        d = PiecewiseDesc(n_reg, (ct.c_int * 3)(*(Ks + [0] * (3 - n_reg))), int(n_pix), int(pad),
                          float(dln), E.ctypes.data)
        for r in range(n_reg):
            for k in range(3):
                d.basis_lo[r][k] = float(basis_lo[r][k])
                d.basis_hi[r][k] = float(basis_hi[r][k])
        d.teff_blend = (ct.c_double * 4)(*tb)
        d.box_lo = (ct.c_double * 5)(*box_lo)
        d.box_hi = (ct.c_double * 5)(*box_hi)
        h = ct.c_void_p()
        _check(lib.lasp_init_interp_piecewise(ct.byref(d), C.ctypes.data, ct.byref(h)),
               "lasp_init_interp_piecewise")
        self = cls.__new__(cls)
        self._h = h
        self._exps = E
        self.K, self.n_pix, self.pad = int(sum(Ks)), int(n_pix), int(pad)
        self.n_model = self.n_pix + 2 * self.pad
        self.dln = float(dln)
        self.box_lo, self.box_hi = np.asarray(box_lo, float), np.asarray(box_hi, float)
        return self

    @classmethod
    def from_grid(cls, grid, C, exps, basis_lo, basis_hi, box_lo, box_hi):
        return cls(C, exps, grid.n_pix, grid.pad, grid.dln, basis_lo, basis_hi, box_lo, box_hi)

    @classmethod
    def from_linear(cls, n_pix, pad, lam0, dln, C_lin, lam1, dlam, exps, basis_lo, basis_hi,
                    box_lo, box_hi):
        """Table given on a linear wavelength grid (lam1 + k dlam): resampled on
        the GPU onto the ln grid of n_pix observed + 2 pad model pixels whose
        observed pixel 0 is at lam0 (Eqs. 2-4), then uploaded."""
        import math
        Cl = torch.as_tensor(np.ascontiguousarray(C_lin, dtype=np.float32)).cuda()
        n_model = int(n_pix) + 2 * int(pad)
        Cr = resample_linear(Cl, lam1, dlam, n_model, math.log(lam0) - pad * dln, dln)
        return cls(Cr.cpu().numpy(), exps, n_pix, pad, dln, basis_lo, basis_hi, box_lo, box_hi)

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.lasp_free_interp(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ calls

    def _batch(self, flux, ivar, good, theta0):
        N = flux.shape[0]
        _dev(flux, torch.float32), _dev(ivar, torch.float32), _dev(good, torch.uint8)
        _dev(theta0, torch.float32)
        if flux.shape != (N, self.n_pix) or ivar.shape != flux.shape or good.shape != flux.shape \
                or theta0.shape != (N, 5):
            raise ValueError("batch shapes must be N x n_pix (and N x 5 for theta0)")
        _on_device(flux=flux, ivar=ivar, good=good, theta0=theta0)
        return Batch(N, self.n_pix, flux.data_ptr(), ivar.data_ptr(), good.data_ptr(),
                     theta0.data_ptr())

    def fit(self, flux, ivar, good, theta0, out=None, stream=None, **opts):
        """lasp_fit_batch: returns dict of device tensors theta, loss, steps,
        status, cont (N x (D+1)), weight."""
        o = default_opts(**opts)
        b = self._batch(flux, ivar, good, theta0)
        N, dev = b.N, flux.device
        if out is None:
            out = dict(theta=torch.empty((N, 5), device=dev),
                       loss=torch.empty(N, device=dev),
                       steps=torch.empty(N, device=dev, dtype=torch.int32),
                       status=torch.empty(N, device=dev, dtype=torch.int32),
                       cont=torch.empty((N, o.legendre_deg + 1), device=dev),
                       weight=torch.empty(N, device=dev))
        else:      # the caller's buffers: the library writes N rows into each
            f32, i32 = torch.float32, torch.int32
            _arg(out["theta"], f32, (N, 5), "out['theta']"), _arg(out["loss"], f32, (N,), "out['loss']")
            _arg(out["steps"], i32, (N,), "out['steps']"), _arg(out["status"], i32, (N,), "out['status']")
            if out.get("cont") is not None:
                _arg(out["cont"], f32, (N, o.legendre_deg + 1), "out['cont']")
            if out.get("weight") is not None:
                _arg(out["weight"], f32, (N,), "out['weight']")
            _on_device(flux=flux, **{f"out['{k}']": out.get(k)
                                     for k in ("theta", "loss", "steps", "status", "cont", "weight")})
        r = Result(out["theta"].data_ptr(), out["loss"].data_ptr(), out["steps"].data_ptr(),
                   out["status"].data_ptr(),
                   out["cont"].data_ptr() if out.get("cont") is not None else None,
                   out["weight"].data_ptr() if out.get("weight") is not None else None)
        _check(load().lasp_fit_batch(self._h, ct.byref(b), ct.byref(o), ct.byref(r),
                                     _stream(stream)), "lasp_fit_batch")
        return out

    def errors(self, flux, ivar, good, theta, with_cov=True, stream=None, **opts):
        o = default_opts(**opts)
        _dev(theta, torch.float32)
        b = self._batch(flux, ivar, good, theta)
        N, dev = b.N, flux.device
        sigma = torch.empty((N, 5), device=dev)
        cov = torch.empty((N, 5, 5), device=dev, dtype=torch.float64) if with_cov else None
        status = torch.empty(N, device=dev, dtype=torch.int32)
        _check(load().lasp_errors(self._h, ct.byref(b), ct.byref(o), _ptr(theta), _ptr(sigma),
                                  _ptr(cov), _ptr(status), _stream(stream)), "lasp_errors")
        return dict(sigma=sigma, cov=cov, status=status)

    def forward(self, theta, b, stream=None):
        _arg(theta, torch.float32, (None, 5), "theta")
        N = theta.shape[0]
        _arg(b, torch.float32, (N, None), "b")
        _on_device(theta=theta, b=b)
        deg = b.shape[1] - 1
        model = torch.empty((N, self.n_pix), device=theta.device)
        _check(load().lasp_forward(self._h, N, _ptr(theta), _ptr(b), deg, _ptr(model),
                                   _stream(stream)), "lasp_forward")
        return model

    def backward(self, theta, b, gmodel, stream=None):
        _arg(theta, torch.float32, (None, 5), "theta")
        N = theta.shape[0]
        _arg(b, torch.float32, (N, None), "b")
        _arg(gmodel, torch.float32, (N, self.n_pix), "gmodel")
        _on_device(theta=theta, b=b, gmodel=gmodel)
        deg = b.shape[1] - 1
        gtheta = torch.empty((N, 5), device=theta.device)
        gb = torch.empty((N, deg + 1), device=theta.device)
        _check(load().lasp_backward(self._h, N, _ptr(theta), _ptr(b), deg, _ptr(gmodel),
                                    _ptr(gtheta), _ptr(gb), _stream(stream)), "lasp_backward")
        return gtheta, gb

    def interp_eval(self, theta, precision="fp32", stream=None):
        _arg(theta, torch.float32, (None, 5), "theta")
        _on_device(theta=theta)
        N = theta.shape[0]
        Fp = torch.empty((N, self.n_model), device=theta.device)
        _check(load().lasp_interp_eval(self._h, N, _ptr(theta), _ptr(Fp), PREC[precision],
                                       _stream(stream)), "lasp_interp_eval")
        return Fp
