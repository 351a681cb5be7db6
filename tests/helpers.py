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


def oracle_model(grid, C=None, deg=DEG) -> O.Model:
    if C is None:
        C = table(grid.name)
    return O.Model(C, S.EXPS, grid.dln, grid.pad, grid.n_pix, deg, S.BASIS_LO, S.BASIS_HI,
                   S.BOX_LO, S.BOX_HI)


_GRIDS = {g.name: g for g in (S.LAMOST, S.DESI, S.SMALL)}


@functools.lru_cache(maxsize=None)
def table(grid_name: str) -> np.ndarray:
    return S.make_table(_GRIDS[grid_name])


def observed(grid, n, seed, **draw_kw):
    """Draws + oracle-made observed flux/ivar for n spectra on grid."""
    M = oracle_model(grid)
    d = S.draw_batch(grid, n, seed, **draw_kw)
    model = O.model_batch(M, d["truth"], d["b_true"])
    flux, ivar = S.finish_obs(model, d)
    d.update(flux=flux, ivar=ivar, model=model)
    return M, d
