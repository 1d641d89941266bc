"""Why the restart and Ritz products of the FP64 method slice the Lanczos basis
afresh: a numpy emulation of thick-restart LancSVD in FP64 in which the basis
enters chosen products as fixed-point values on one grid for all rows, as the
rows-layout digit planes of an orthonormal basis hold it (a fixed exponent for
every row).  The library's grid unit is 2^-54; here a coarser unit, 2^-44, makes the
effect visible at a CPU-sized matrix (the floor scales with the unit, sqrt(n) and
sqrt(r b)).

* exact: the solve converges to rounding level;
* basis on the grid in the restart products (P Vbar_s, Pbar Ubar_s, U, V): the
  kept Ritz vectors carry the grid's error, the next cycle takes them as exact, and
  the residual stops at a floor while the Lanczos estimate keeps falling;
* basis on the grid in the CGS-CQR2 products: a lower floor of the same origin.

Design check, not a pin of the oracle: the emulation is written here."""

import numpy as np

from helpers import LowRankPlusSparse, emulated_thick_lanczos

UNIT = 2.0 ** -44


def _grid(X):
    return np.round(X / UNIT) * UNIT


def test_basis_on_a_fixed_grid_in_the_restart_products_sets_a_residual_floor():
    A = LowRankPlusSparse(30_000, seed=4)
    exact = emulated_thick_lanczos(A, 8, 16, 8, 48, 5)
    restart = emulated_thick_lanczos(A, 8, 16, 8, 48, 5, restart_basis=_grid)
    orth = emulated_thick_lanczos(A, 8, 16, 8, 48, 5, orth_basis=_grid)
    res = lambda h: [r for _, r in h]  # noqa: E731
    # exact arithmetic of the products: converged to rounding level
    assert res(exact)[-1] < 3e-14
    # grid in the restart products: a flat floor far above it, while the Lanczos
    # estimate (computed from B, which takes the kept vectors as exact) keeps falling
    assert res(restart)[-1] > 100 * res(exact)[-1]
    assert max(res(restart)[-3:]) < 1.5 * min(res(restart)[-3:])
    assert restart[-1][0] < 1e-3 * res(restart)[-1]
    # grid in the CGS-CQR2 products: also above exact arithmetic
    assert res(orth)[-1] > 10 * res(exact)[-1]
