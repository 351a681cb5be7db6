"""Shared test fixtures: synthetic inputs and the oracle model built from them.

The observed spectra of every test are made by the oracle's forward model
from the generator's random draws, so no input or expected value of a parity
test comes from the CUDA path."""
from __future__ import annotations

import functools

import numpy as np

import lasp_synth as S
from oracle import oracle as O

DEG = 6
TOL = np.array([1.0, 0.005, 0.005, 0.1])          # Teff K, logg, [Fe/H], RV km/s

# Gradient parity of the FP32 adjoint against the FP64 oracle.  A gradient
# component is a sum over the pixels (through dF' and the table contraction)
# added in FP32 in blocks: 16 pixels a thread, then a tree over the threads,
# about 30 roundings on any path, so its error is at most about 30 u sum|terms|
# (u = 2^-24).  With random-sign cotangents, as in the tests, sum|terms| / |sum|
# is about sqrt(p), 63 at 3909 pixels: 30 x 6e-8 x 63 = 1.1e-4.  Bounds: theta
# 2e-4 of |g| + 1e-3 max|g| (the floor for components that cancel to near
# zero); Legendre coefficients 1e-4 of max|g|.
GRAD_RTOL_THETA = 2e-4
GRAD_TOL_LEG = 1e-4


def oracle_model(grid, C=None, deg=DEG) -> O.Model:
    if C is None:
        C = table(grid.name)
    return O.Model(C, S.EXPS, grid.dln, grid.pad, grid.n_pix, deg, S.BASIS_LO, S.BASIS_HI,
                   S.BOX_LO, S.BOX_HI)


_GRIDS = {g.name: g for g in (S.LAMOST, S.DESI, S.SMALL)}


@functools.lru_cache(maxsize=None)
def table(grid_name: str) -> np.ndarray:
    return S.make_table(_GRIDS[grid_name])


@functools.lru_cache(maxsize=None)
def pw_tables(grid_name: str):
    return tuple(S.make_piecewise_tables(_GRIDS[grid_name]))


def piecewise_model(grid, deg=DEG, tables=None) -> O.Model:
    """Oracle model of the three-regime synthetic emulator on grid."""
    if tables is None:
        tables = pw_tables(grid.name)
    C = np.concatenate(tables)
    E = np.concatenate(S.PW_EXPS)
    return O.Model(C, E, grid.dln, grid.pad, grid.n_pix, deg, S.PW_BASIS_LO[1], S.PW_BASIS_HI[1],
                   S.PW_BOX_LO, S.PW_BOX_HI, reg_K=[len(e) for e in S.PW_EXPS],
                   reg_blo=S.PW_BASIS_LO, reg_bhi=S.PW_BASIS_HI, tblend=S.TEFF_BLEND)


def observed(grid, n, seed, M=None, **draw_kw):
    """Draws + oracle-made observed flux/ivar for n spectra on grid (model M,
    default the single-regime oracle model of grid)."""
    if M is None:
        M = oracle_model(grid)
    d = S.draw_batch(grid, n, seed, **draw_kw)
    model = O.model_batch(M, d["truth"], d["b_true"])
    flux, ivar = S.finish_obs(model, d)
    d.update(flux=flux, ivar=ivar, model=model)
    return M, d
