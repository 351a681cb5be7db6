"""Seeded synthetic inputs for grouped spectral fitting.

This module draws every random quantity the workloads need and nothing else:
the coefficient table of a synthetic polynomial interpolator, the true and
initial stellar parameters, the true continuum coefficients, the pixel masks,
the signal-to-noise ratios and the unit-normal noise draws.  It holds none of
the fitting method's arithmetic (no basis contraction, no broadening, no
continuum fit, no loss): turning true parameters into a model spectrum is left
to whichever implementation consumes these inputs, and `finish_obs` only adds
noise and mask spikes to a model spectrum handed to it.

Grids (ln-lambda, air wavelengths assumed):
  LAMOST-like  3909 px, 3700-9000 A   (R ~ 1800 survey, section 3.2.1)
  DESI-like    7781 px, 3600-9824 A   (DESI MWS range, section 4.4)
  small        1024 px from 4200 A with the LAMOST step (inside the
               4200-5700 A window of section 3.3)
Seeds: table 2512; spectra 24840 + workload index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import erf

C_KMS = 299792.458

# Physical parameter box (Teff K, log g dex, [Fe/H] dex, RV km/s, sigma km/s).
# The method normalises all free parameters to [-1, 1] (section 2.2, stage 8);
# the paper does not print the bounds, these are the ones this library uses.
BOX_LO = np.array([3500.0, 0.5, -2.5, -300.0, 30.0])
BOX_HI = np.array([7500.0, 5.5, 1.0, 300.0, 200.0])

# Basis normalisation box for the interpolator variables (log10 Teff, log g,
# [Fe/H]); each is mapped linearly onto [-1, 1] before forming monomials.
BASIS_LO = np.array([math.log10(3500.0), 0.5, -2.5])
BASIS_HI = np.array([math.log10(7500.0), 5.5, 1.0])


def _exponents() -> np.ndarray:
    """26 exponent triples (a, b, c) of u_T^a u_g^b u_f^c.

    All 20 monomials of total degree <= 3, then six quartic terms; 26 is the
    size of the warm-star ELODIE interpolator (section 3.1)."""
    out = []
    for deg in range(4):
        for a in range(deg, -1, -1):
            for b in range(deg - a, -1, -1):
                out.append((a, b, deg - a - b))
    out += [(4, 0, 0), (3, 1, 0), (3, 0, 1), (2, 2, 0), (2, 1, 1), (2, 0, 2)]
    return np.array(out, dtype=np.int8)


EXPS = _exponents()
K_TERMS = len(EXPS)
assert K_TERMS == 26


@dataclass(frozen=True)
class Grid:
    name: str
    n_pix: int
    lam0: float          # wavelength of observed pixel 0 (Angstrom)
    dln: float           # ln-lambda step

    @property
    def kms_per_px(self) -> float:
        return C_KMS * self.dln

    @property
    def pad(self) -> int:
        """Table margin H: enough model pixels each side for the widest kernel
        in the box, 2*ceil(|mu| + 5 sigma) + 1 taps (Eq. 5)."""
        mu = max(abs(BOX_LO[3]), abs(BOX_HI[3])) / self.kms_per_px
        sig = BOX_HI[4] / self.kms_per_px
        return int(math.ceil(mu + 5.0 * sig))

    @property
    def n_model(self) -> int:
        return self.n_pix + 2 * self.pad

    @property
    def ln_lambda0_model(self) -> float:
        return math.log(self.lam0) - self.pad * self.dln

    def wavelengths(self) -> np.ndarray:
        return np.exp(math.log(self.lam0) + self.dln * np.arange(self.n_pix))


LAMOST = Grid("lamost", 3909, 3700.0, math.log(9000.0 / 3700.0) / 3908)
DESI = Grid("desi", 7781, 3600.0, math.log(9824.0 / 3600.0) / 7780)
SMALL = Grid("small1024", 1024, 4200.0, math.log(9000.0 / 3700.0) / 3908)

TABLE_SEED = 2512
SPECTRA_SEED = 24840


def _basis_degree(k: int) -> int:
    return int(EXPS[k].sum())


def make_table(grid: Grid, seed: int = TABLE_SEED, n_lines: int | None = None) -> np.ndarray:
    """Coefficient table C (K x n_model, float32) of a smooth random
    polynomial interpolator on the padded ln-lambda grid of `grid`.

    Row 0 is a continuum near 1 with a gentle slope; rows k >= 1 add small
    smooth colour terms.  On top, absorption lines (about one per 10 A) at
    uniform random ln-lambda centres, each a pixel-integrated Gaussian of
    intrinsic width 10-30 km/s, whose depth is a polynomial in the basis with
    leading coefficient U(0.05, 0.5) and higher coefficients N(0, (0.15 a0 /
    degree)^2), so depths vary smoothly across the parameter box."""
    rng = np.random.Generator(np.random.PCG64(seed))
    K, n = K_TERMS, grid.n_model
    m = np.arange(n, dtype=np.float64)
    t = 2.0 * m / (n - 1) - 1.0               # position along the grid in [-1, 1]
    C = np.zeros((K, n))
    C[0] = 1.0
    for k in range(K):
        amp = 0.05 if k == 0 else 0.02 / _basis_degree(k)
        for d in range(1, 4):
            C[k] += rng.normal(0.0, amp) * np.cos(math.pi * d * (t + 1.0) / 2.0)
    lam_lo = math.exp(grid.ln_lambda0_model)
    lam_hi = math.exp(grid.ln_lambda0_model + (n - 1) * grid.dln)
    if n_lines is None:
        n_lines = int(round((lam_hi - lam_lo) / 10.0))
    centres = rng.uniform(2.0, n - 3.0, size=n_lines)         # pixel units
    widths = rng.uniform(10.0, 30.0, size=n_lines) / grid.kms_per_px
    a0 = rng.uniform(0.05, 0.5, size=n_lines)
    depth = np.zeros((K, n_lines))
    depth[0] = a0
    for k in range(1, K):
        depth[k] = rng.normal(0.0, 0.15 * a0 / _basis_degree(k))
    for l in range(n_lines):
        lo = max(0, int(centres[l] - 8 * widths[l] - 2))
        hi = min(n, int(centres[l] + 8 * widths[l] + 3))
        mm = m[lo:hi]
        s2 = widths[l] * math.sqrt(2.0)
        # pixel-integrated profile, peak ~1 for widths well above a pixel
        prof = widths[l] * math.sqrt(math.pi / 2.0) * (
            erf((mm + 0.5 - centres[l]) / s2) - erf((mm - 0.5 - centres[l]) / s2))
        C[:, lo:hi] -= depth[:, l:l + 1] * prof[None, :]
    return C.astype(np.float32)


# ---- piecewise emulator (Eq. 1 with Teff regimes f1..f5; section 3.1) ----
# Three regimes ordered by Teff with the term counts of the paper's cold, warm
# and hot models (25, 26, 19): all 20 monomials of total degree <= 3 plus five
# quartic terms (cold), the 26 terms above (warm), the cubic set without the
# pure [Fe/H]^3 term (hot).
EXPS_COLD = np.ascontiguousarray(EXPS[:25])
EXPS_WARM = EXPS
EXPS_HOT = np.ascontiguousarray(np.array([e for e in EXPS[:20] if tuple(e) != (0, 0, 3)],
                                         dtype=np.int8))
PW_EXPS = (EXPS_COLD, EXPS_WARM, EXPS_HOT)
assert [len(e) for e in PW_EXPS] == [25, 26, 19]
# Blend intervals of Eq. 1: cold <= 4000 K < cold/warm <= 4550 K < warm
# <= 7000 K < warm/hot <= 9000 K < hot.
TEFF_BLEND = (4000.0, 4550.0, 7000.0, 9000.0)
# Parameter box of the piecewise workloads (Teff spans all five ranges).
PW_BOX_LO = np.array([3200.0, 0.5, -2.5, -300.0, 30.0])
PW_BOX_HI = np.array([12000.0, 5.5, 1.0, 300.0, 200.0])
# Basis box of each regime: its own Teff support, the common log g, [Fe/H].
PW_BASIS_LO = tuple(np.array([math.log10(t), 0.5, -2.5]) for t in (3200.0, 4000.0, 7000.0))
PW_BASIS_HI = tuple(np.array([math.log10(t), 5.5, 1.0]) for t in (4550.0, 9000.0, 12000.0))


def make_piecewise_tables(grid: Grid, seed: int = TABLE_SEED + 1) -> list:
    """Coefficient tables (K_r x n_model, float32) of a three-regime synthetic
    emulator on the padded grid of `grid`, coolest first.  The regimes share
    one line list (as emulators fitted to one spectral library would); lines
    are deeper in the cold regime and shallower in the hot one, continua
    redder to bluer, and each regime draws its own smooth depth polynomial, so
    neighbouring regimes differ where they blend."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = grid.n_model
    m = np.arange(n, dtype=np.float64)
    t = 2.0 * m / (n - 1) - 1.0
    lam_lo = math.exp(grid.ln_lambda0_model)
    lam_hi = math.exp(grid.ln_lambda0_model + (n - 1) * grid.dln)
    n_lines = int(round((lam_hi - lam_lo) / 10.0))
    centres = rng.uniform(2.0, n - 3.0, size=n_lines)
    widths = rng.uniform(10.0, 30.0, size=n_lines) / grid.kms_per_px
    a0 = rng.uniform(0.05, 0.5, size=n_lines)
    profs = []
    for l in range(n_lines):
        lo = max(0, int(centres[l] - 8 * widths[l] - 2))
        hi = min(n, int(centres[l] + 8 * widths[l] + 3))
        mm = m[lo:hi]
        s2 = widths[l] * math.sqrt(2.0)
        profs.append((lo, hi, widths[l] * math.sqrt(math.pi / 2.0) * (
            erf((mm + 0.5 - centres[l]) / s2) - erf((mm - 0.5 - centres[l]) / s2))))
    out = []
    for exps, depth_scale, slope in zip(PW_EXPS, (1.3, 1.0, 0.5), (0.15, 0.0, -0.15)):
        K = len(exps)
        deg = np.maximum(exps.sum(axis=1), 1)
        C = np.zeros((K, n))
        C[0] = 1.0 + slope * t
        for k in range(K):
            amp = 0.05 if k == 0 else 0.02 / deg[k]
            for d in range(1, 4):
                C[k] += rng.normal(0.0, amp) * np.cos(math.pi * d * (t + 1.0) / 2.0)
        depth = np.zeros((K, n_lines))
        depth[0] = depth_scale * a0
        for k in range(1, K):
            depth[k] = rng.normal(0.0, 0.15 * depth_scale * a0 / deg[k])
        for l, (lo, hi, prof) in enumerate(profs):
            C[:, lo:hi] -= depth[:, l:l + 1] * prof[None, :]
        out.append(C.astype(np.float32))
    return out


def _mask_runs(rng, grid: Grid, frac: float) -> np.ndarray:
    """1 = pixel used, 0 = masked.  Contiguous runs of 3-12 px until about
    `frac` of the pixels are masked, plus the Na D region 5885-5900 A, the
    paper's example of a predefined masked region (stage 6)."""
    n = grid.n_pix
    good = np.ones(n, dtype=np.uint8)
    lam = grid.wavelengths()
    if frac > 0:
        good[(lam >= 5885.0) & (lam <= 5900.0)] = 0
        target = int(round(frac * n))
        while (n - int(good.sum())) < target:
            L = int(rng.integers(3, 13))
            s = int(rng.integers(0, n - L))
            good[s:s + L] = 0
    return good


def draw_batch(grid: Grid, n_spec: int, seed: int, *, snr=(5.0, 100.0), mask_frac=0.05,
               mask_frac_max=None, init: str = "cfi", noise: bool = True,
               teff=(4000.0, 7000.0), logg=(1.0, 5.0), feh=(-2.0, 0.5),
               rv=(-200.0, 200.0), sig=(50.0, 150.0), box=None) -> dict:
    """Random draws for `n_spec` spectra on `grid`.

    Returns truth (N x 5 physical), b_true (N x 7 continuum coefficients,
    s * (1, beta_1..beta_6) with beta_d ~ N(0, 0.1/d) rescaled so the sum of
    |beta_d| stays <= 0.8, hence the continuum stays >= 0.2 s), theta0 (N x 5
    initial guess), snr (N), z (N x n_pix unit normals), good (N x n_pix mask,
    1 = used).  init='cfi' perturbs the truth by N(0, diag(200 K, 0.3, 0.2,
    15 km/s, 20 km/s)) and clips to the box (a stand-in for the CFI initial
    values); init='fixed' is (7500 K, 3, -0.5, 0, 100) (section 4.2.1).
    box: (lo, hi) physical bounds that theta0 is clipped to (default the
    single-regime box BOX_LO/BOX_HI)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N, n = n_spec, grid.n_pix
    truth = np.stack([rng.uniform(*teff, N), rng.uniform(*logg, N), rng.uniform(*feh, N),
                      rng.uniform(*rv, N), rng.uniform(*sig, N)], axis=1)
    scale = np.exp(rng.uniform(math.log(0.1), math.log(100.0), N))
    beta = rng.normal(0.0, 1.0, (N, 6)) * (0.1 / np.arange(1, 7))[None, :]
    tot = np.abs(beta).sum(axis=1, keepdims=True)
    beta = np.where(tot > 0.8, beta * (0.8 / np.maximum(tot, 1e-300)), beta)
    b_true = scale[:, None] * np.concatenate([np.ones((N, 1)), beta], axis=1)
    if init == "cfi":
        theta0 = truth + rng.normal(0.0, 1.0, (N, 5)) * np.array([200.0, 0.3, 0.2, 15.0, 20.0])
        blo, bhi = (BOX_LO, BOX_HI) if box is None else box
        theta0 = np.clip(theta0, blo, bhi)
    elif init == "fixed":
        theta0 = np.tile(np.array([7500.0, 3.0, -0.5, 0.0, 100.0]), (N, 1))
    elif init == "truth":
        theta0 = truth.copy()
    else:
        raise ValueError(init)
    snr_v = np.exp(rng.uniform(math.log(snr[0]), math.log(snr[1]), N))
    z = rng.standard_normal((N, n)) if noise else np.zeros((N, n))
    good = np.ones((N, n), dtype=np.uint8)
    for i in range(N):
        f = mask_frac if mask_frac_max is None else rng.uniform(mask_frac, mask_frac_max)
        good[i] = _mask_runs(rng, grid, f)
    return dict(grid=grid, truth=truth, b_true=b_true, theta0=theta0, snr=snr_v, z=z,
                good=good, noise=noise)


def finish_obs(model: np.ndarray, draws: dict, spike: float = 50.0):
    """Observed flux and inverse variance from a noise-free model spectrum.

    sigma_ij = (median_i / SNR_i) * sqrt(max(model_ij, 0.05 median_i) / median_i)
    (photon-noise-like, so the inverse variance varies along the spectrum);
    flux = model + sigma * z.  Masked pixels get ivar 0 and flux = spike *
    median, so any leak of a masked pixel into a fit shows."""
    model = np.asarray(model, dtype=np.float64)
    med = np.median(model, axis=1, keepdims=True)
    med = np.where(med > 0, med, 1.0)
    rel = np.sqrt(np.maximum(model, 0.05 * med) / med)
    sigma = (med / draws["snr"][:, None]) * rel
    flux = model + sigma * draws["z"] if draws["noise"] else model.copy()
    ivar = 1.0 / sigma ** 2
    bad = draws["good"] == 0
    flux = np.where(bad, spike * med, flux)
    ivar = np.where(bad, 0.0, ivar)
    return flux.astype(np.float32), ivar.astype(np.float32)


def workload(name: str):
    """(grid, n_spec, seed offset, draw kwargs) of the named workloads."""
    table = {
        "small16": (SMALL, 16, 0, dict(noise=False, mask_frac=0.0)),
        "lamost4096": (LAMOST, 4096, 1, dict(snr=(5.0, 100.0), mask_frac=0.05)),
        "adjoint1024": (LAMOST, 1024, 2, dict(noise=False, mask_frac=0.0)),
        "mixed65536": (LAMOST, 65536, 3, dict(snr=(5.0, 100.0), mask_frac=0.05)),
        "stream_lamost": (LAMOST, 4096, 4, dict(snr=(5.0, 100.0), mask_frac=0.0, mask_frac_max=0.2)),
        "stream_desi": (DESI, 4096, 4, dict(snr=(5.0, 100.0), mask_frac=0.0, mask_frac_max=0.2)),
        "piecewise4096": (LAMOST, 4096, 5, dict(snr=(5.0, 100.0), mask_frac=0.05,
                                                 teff=(3300.0, 11500.0), box=(PW_BOX_LO, PW_BOX_HI))),
    }
    return table[name]
