"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline
leg import this module.  It builds `liblasp_oracle.so` from `lasp_oracle.c`
with gcc on first use and exposes numpy-level calls.  Arrays are float64
except flux/ivar (float32, as the observations are stored) and the mask
(uint8, 1 = pixel used).
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lasp_oracle.c")
_LIB = os.path.join(_HERE, "liblasp_oracle.so")
_lock = threading.Lock()
_lib = None

ST_CONV_TOL, ST_CONV_RISE, ST_MAXSTEPS = 1, 2, 4
ST_NONPOS, ST_NONFINITE, ST_SINGULAR, ST_NODATA = 8, 16, 32, 64
C_KMS = 299792.458


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP over spectra)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lasp_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Model(ct.Structure):
    _fields_ = [("K", ct.c_int), ("exps", ct.c_void_p), ("blo", ct.c_double * 3),
                ("bhi", ct.c_double * 3), ("plo", ct.c_double * 5), ("phi", ct.c_double * 5),
                ("dln", ct.c_double), ("pad", ct.c_int), ("n_pix", ct.c_int), ("deg", ct.c_int),
                ("C", ct.c_void_p), ("n_reg", ct.c_int), ("reg_K", ct.c_int * 3),
                ("rblo", (ct.c_double * 3) * 3), ("rbhi", (ct.c_double * 3) * 3),
                ("tblend", ct.c_double * 4)]


class _Opts(ct.Structure):
    _fields_ = [("lr", ct.c_double), ("beta1", ct.c_double), ("beta2", ct.c_double),
                ("eps", ct.c_double), ("tol", ct.c_double), ("window", ct.c_int),
                ("max_steps", ct.c_int), ("edge_px", ct.c_int), ("quantile", ct.c_double),
                ("clean", ct.c_int), ("clean_every", ct.c_int), ("clean_max", ct.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ct.CDLL(build())
            P = ct.c_void_p
            _lib.orc_basis.argtypes = [P, P, P, P]
            _lib.orc_kernel.argtypes = [ct.c_double, ct.c_double, ct.c_int, P, P, P]
            _lib.orc_kernel.restype = ct.c_int
            _lib.orc_legendre.argtypes = [ct.c_int, ct.c_int, P]
            _lib.orc_model_flux.argtypes = [P, P, P, P, P, P, P]
            _lib.orc_model_vjp.argtypes = [P, P, P, P, P, P]
            _lib.orc_prep.argtypes = [ct.c_int, P, P, P, ct.c_double, ct.c_int, P, P, P]
            _lib.orc_prep.restype = ct.c_int
            _lib.orc_eval.argtypes = [P, P, P, P, P, P, P, P, P]
            _lib.orc_eval.restype = ct.c_uint
            _lib.orc_adam_update.argtypes = [ct.c_int, P, P, P, P, ct.c_int, ct.c_double,
                                             ct.c_double, ct.c_double, ct.c_double, ct.c_int]
            _lib.orc_stop_rule.argtypes = [P, ct.c_int, ct.c_int, ct.c_double, ct.c_int]
            _lib.orc_stop_rule.restype = ct.c_uint
            _lib.orc_fit.argtypes = [P, P, ct.c_int, P, P, P, P, P, P, P, P, P, ct.c_int]
            _lib.orc_fit_trajectory.argtypes = [P, P, P, P, P, P, ct.c_int, P, P]
            _lib.orc_errors.argtypes = [P, P, P, P, P, P, P, P, P]
            _lib.orc_errors.restype = ct.c_uint
            _lib.orc_phys_from_x.argtypes = [P, P, P]
            _lib.orc_x_from_phys.argtypes = [P, P, P]
            _lib.orc_max_threads.restype = ct.c_int
            _lib.orc_resample.argtypes = [ct.c_int, ct.c_double, ct.c_double, P, ct.c_int,
                                          ct.c_double, ct.c_double, P]
            _lib.orc_clean_mask.argtypes = [ct.c_int, P, P, P, ct.c_double, P]
            _lib.orc_clean_mask.restype = ct.c_int
            _lib.orc_fit_lm.argtypes = [P, P, ct.c_int, P, P, P, P, ct.c_int, ct.c_double, P, P, P,
                                        P, ct.c_int]
            _lib.orc_fit_joint.argtypes = [P, P, ct.c_int, P, P, P, P, P, P, P, P, P, ct.c_int]
        return _lib


def _p(a):
    return a.ctypes.data_as(ct.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Model:
    """Interpolator table + grid + boxes, as the oracle sees them.

    Piecewise emulator (Eq. 1 with Teff regimes): pass reg_K (terms per
    regime, coolest first; the rows of C and exps stacked in that order),
    reg_blo/reg_bhi (basis box per regime) and tblend (2 (n_reg - 1) Teff
    bounds of the blend intervals); blo/bhi are then unused."""

    def __init__(self, C, exps, dln, pad, n_pix, deg, blo, bhi, plo, phi, reg_K=None, reg_blo=None,
                 reg_bhi=None, tblend=None):
        self.C = _f64(C)
        self.exps = np.ascontiguousarray(exps, dtype=np.int8)
        self.K = self.exps.shape[0]
        assert self.C.shape == (self.K, n_pix + 2 * pad)
        self.dln, self.pad, self.n_pix, self.deg = float(dln), int(pad), int(n_pix), int(deg)
        if not 0 <= self.deg <= 8:
            raise ValueError("Legendre continuum degree must be 0..8")
        self.blo, self.bhi = _f64(blo), _f64(bhi)
        self.plo, self.phi = _f64(plo), _f64(phi)
        self.reg_K = None if reg_K is None else [int(k) for k in reg_K]
        self.reg_blo, self.reg_bhi, self.tblend = reg_blo, reg_bhi, tblend
        n_reg = 1 if reg_K is None else len(reg_K)
        if n_reg > 1:
            assert sum(self.reg_K) == self.K
        self._s = _Model(self.K, self.exps.ctypes.data, (ct.c_double * 3)(*self.blo),
                         (ct.c_double * 3)(*self.bhi), (ct.c_double * 5)(*self.plo),
                         (ct.c_double * 5)(*self.phi), self.dln, self.pad, self.n_pix,
                         self.deg, self.C.ctypes.data, n_reg)
        if n_reg > 1:
            for r in range(n_reg):
                self._s.reg_K[r] = self.reg_K[r]
                for i in range(3):
                    self._s.rblo[r][i] = float(reg_blo[r][i])
                    self._s.rbhi[r][i] = float(reg_bhi[r][i])
            for q, t in enumerate(tblend):
                self._s.tblend[q] = float(t)

    @property
    def ref(self):
        return ct.byref(self._s)

    @property
    def n_model(self):
        return self.n_pix + 2 * self.pad

    def with_table(self, C):
        return Model(C, self.exps, self.dln, self.pad, self.n_pix, self.deg, self.blo, self.bhi,
                     self.plo, self.phi, self.reg_K, self.reg_blo, self.reg_bhi, self.tblend)


def make_opts(lr=0.1, beta1=0.9, beta2=0.999, eps=1e-8, tol=1e-5, window=50, max_steps=5000,
              edge_px=0, quantile=0.5, clean=0, clean_every=30, clean_max=11):
    return _Opts(lr, beta1, beta2, eps, tol, window, max_steps, edge_px, quantile, clean,
                 clean_every, clean_max)


def basis(M: Model, th):
    th = _f64(th)
    phi = np.zeros(M.K)
    dphi = np.zeros((M.K, 3))
    lib().orc_basis(M.ref, _p(th), _p(phi), _p(dphi))
    return phi, dphi


def kernel(mu, sig, H):
    g, dm, ds = np.zeros(2 * H + 1), np.zeros(2 * H + 1), np.zeros(2 * H + 1)
    h = lib().orc_kernel(float(mu), float(sig), int(H), _p(g), _p(dm), _p(ds))
    return g, dm, ds, h


def legendre(p, D):
    out = np.zeros((p, D + 1))
    lib().orc_legendre(int(p), int(D), _p(out))
    return out


def model_flux(M: Model, th, b):
    th, b = _f64(th), _f64(b)
    Fp, Fpp = np.zeros(M.n_model), np.zeros(M.n_pix)
    cont, model = np.zeros(M.n_pix), np.zeros(M.n_pix)
    lib().orc_model_flux(M.ref, _p(th), _p(b), _p(Fp), _p(Fpp), _p(cont), _p(model))
    return dict(Fp=Fp, Fpp=Fpp, cont=cont, model=model)


def model_batch(M: Model, theta, b):
    """Noise-free model spectra (N x n_pix) for rows of theta (physical) and b."""
    theta, b = np.atleast_2d(_f64(theta)), np.atleast_2d(_f64(b))
    return np.stack([model_flux(M, theta[i], b[i])["model"] for i in range(theta.shape[0])])


def model_vjp(M: Model, th, b, gm):
    th, b, gm = _f64(th), _f64(b), _f64(gm)
    gth, gb = np.zeros(5), np.zeros(M.deg + 1)
    lib().orc_model_vjp(M.ref, _p(th), _p(b), _p(gm), _p(gth), _p(gb))
    return gth, gb


def prep(flux, ivar, good, quantile=0.5, edge_px=0):
    flux = np.ascontiguousarray(flux, dtype=np.float32)
    ivar = np.ascontiguousarray(ivar, dtype=np.float32)
    good = np.ascontiguousarray(good, dtype=np.uint8)
    n = flux.shape[0]
    y, W, w = np.zeros(n), np.zeros(n), np.zeros(1)
    n_obj = lib().orc_prep(n, _p(flux), _p(ivar), _p(good), float(quantile), int(edge_px),
                           _p(y), _p(W), _p(w))
    return y, W, float(w[0]), n_obj


def evaluate(M: Model, y, W, x):
    y, W, x = _f64(y), _f64(W), _f64(x)
    loss, g = np.zeros(1), np.zeros(5)
    b, eps, cont = np.zeros(M.deg + 1), np.zeros(M.n_pix), np.zeros(M.n_pix)
    st = lib().orc_eval(M.ref, _p(y), _p(W), _p(x), _p(loss), _p(g), _p(b), _p(eps), _p(cont))
    return dict(loss=float(loss[0]), grad=g, b=b, eps=eps, cont=cont, status=int(st))


def adam_update(x, m, v, g, t, lr=0.1, b1=0.9, b2=0.999, eps=1e-8, clamp=True):
    x, m, v, g = _f64(x).copy(), _f64(m).copy(), _f64(v).copy(), _f64(g)
    lib().orc_adam_update(len(x), _p(x), _p(m), _p(v), _p(g), int(t), lr, b1, b2, eps, int(clamp))
    return x, m, v


def stop_rule(hist, t, window=50, tol=1e-5, max_steps=5000):
    hist = _f64(hist)
    return int(lib().orc_stop_rule(_p(hist), int(t), int(window), float(tol), int(max_steps)))


def phys_from_x(M: Model, x):
    x = _f64(x)
    th = np.zeros(5)
    lib().orc_phys_from_x(M.ref, _p(x), _p(th))
    return th


def x_from_phys(M: Model, th):
    th = _f64(th)
    x = np.zeros(5)
    lib().orc_x_from_phys(M.ref, _p(th), _p(x))
    return x


def fit(M: Model, flux, ivar, good, theta0, threads=None, **opts):
    flux = np.ascontiguousarray(flux, dtype=np.float32)
    ivar = np.ascontiguousarray(ivar, dtype=np.float32)
    good = np.ascontiguousarray(good, dtype=np.uint8)
    theta0 = _f64(theta0)
    n = flux.shape[0]
    theta, loss = np.zeros((n, 5)), np.zeros(n)
    steps, status = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.uint32)
    b = np.zeros((n, M.deg + 1))
    O = make_opts(**opts)
    if threads is None:
        threads = lib().orc_max_threads()
    lib().orc_fit(M.ref, ct.byref(O), n, _p(flux), _p(ivar), _p(good), _p(theta0), _p(theta),
                  _p(loss), _p(steps), _p(status), _p(b), int(threads))
    return dict(theta=theta, loss=loss, steps=steps, status=status, b=b)


def fit_joint(M: Model, flux, ivar, good, theta0, threads=None, **opts):
    """PAPER_JOINT reading of Eq. 9: one RMS over the group, group stop rules."""
    flux = np.ascontiguousarray(flux, dtype=np.float32)
    ivar = np.ascontiguousarray(ivar, dtype=np.float32)
    good = np.ascontiguousarray(good, dtype=np.uint8)
    theta0 = _f64(theta0)
    n = flux.shape[0]
    theta = np.zeros((n, 5))
    loss = np.zeros(n)
    steps = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.uint32)
    lg = np.zeros(1)
    th = lib().orc_max_threads() if threads is None else int(threads)
    O = make_opts(**opts)
    lib().orc_fit_joint(M.ref, ct.byref(O), n, _p(flux), _p(ivar), _p(good), _p(theta0), _p(theta),
                        _p(loss), _p(steps), _p(status), _p(lg), th)
    return dict(theta=theta, loss=loss, steps=steps, status=status, loss_group=float(lg[0]))


def trajectory(M: Model, flux, ivar, good, theta0, nsteps, **opts):
    flux = np.ascontiguousarray(flux, dtype=np.float32)
    ivar = np.ascontiguousarray(ivar, dtype=np.float32)
    good = np.ascontiguousarray(good, dtype=np.uint8)
    xs, ls = np.zeros((nsteps + 1, 5)), np.zeros(nsteps + 1)
    O = make_opts(**opts)
    lib().orc_fit_trajectory(M.ref, ct.byref(O), _p(flux), _p(ivar), _p(good), _p(_f64(theta0)),
                             int(nsteps), _p(xs), _p(ls))
    return xs, ls


def errors(M: Model, flux, ivar, good, theta, with_jac=False, **opts):
    flux = np.ascontiguousarray(flux, dtype=np.float32)
    ivar = np.ascontiguousarray(ivar, dtype=np.float32)
    good = np.ascontiguousarray(good, dtype=np.uint8)
    sig, cov = np.zeros(5), np.zeros(25)
    jac = np.zeros((M.n_pix, 5)) if with_jac else None
    O = make_opts(**opts)
    st = lib().orc_errors(M.ref, ct.byref(O), _p(flux), _p(ivar), _p(good), _p(_f64(theta)),
                          _p(sig), _p(cov), _p(jac))
    return dict(sigma=sig, cov=cov.reshape(5, 5), status=int(st), jac=jac)


def resample(F, lam1, dlam, n_out, ln_lam0, dln):
    """Flux-conserving resampling of F (linear grid) onto a ln grid (Eqs. 2-4)."""
    F = _f64(F)
    out = np.zeros(int(n_out))
    lib().orc_resample(len(F), float(lam1), float(dlam), _p(F), int(n_out), float(ln_lam0),
                       float(dln), _p(out))
    return out


def clean_mask(r, m, used, fshift):
    """Clean outlier mask (Eq. 8) of the weighted residual r and model m, with
    every quantity and decision in double precision."""
    r = _f64(r)
    m = _f64(m)
    used = np.ascontiguousarray(used, dtype=np.uint8)
    keep = np.zeros(len(r), dtype=np.uint8)
    k = lib().orc_clean_mask(len(r), _p(r), _p(m), _p(used), float(fshift), _p(keep))
    return keep, k


def fit_lm(M: Model, flux, ivar, good, theta0, max_iter=50, rtol=1e-9, threads=None, **opts):
    """Levenberg-Marquardt fit of the same objective (curvature-aware step)."""
    flux = np.ascontiguousarray(flux, dtype=np.float32)
    ivar = np.ascontiguousarray(ivar, dtype=np.float32)
    good = np.ascontiguousarray(good, dtype=np.uint8)
    theta0 = _f64(theta0)
    n = flux.shape[0]
    theta, loss = np.zeros((n, 5)), np.zeros(n)
    iters, status = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.uint32)
    O = make_opts(**opts)
    if threads is None:
        threads = lib().orc_max_threads()
    lib().orc_fit_lm(M.ref, ct.byref(O), n, _p(flux), _p(ivar), _p(good), _p(theta0), int(max_iter),
                     float(rtol), _p(theta), _p(loss), _p(iters), _p(status), int(threads))
    return dict(theta=theta, loss=loss, steps=iters, status=status)
