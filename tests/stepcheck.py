"""Per-cell comparison of converged step solutions.

A converged implicit step is compared cell by cell and field by field:
|u_gpu - u_oracle| <= tol |u_oracle| on every leaf cell, for E and for T
separately.  E spans about five decades across a Marshak front (1e-5 in the
cold region, ~1 behind the front), so a bound relative to the largest value
would allow large relative errors in the cold cells, where the front's
progress is decided.  Both sides are converged past the stated Newton
tolerance (1e-8) so that two correct solves agree per cell well inside it.
"""
import numpy as np


def per_cell_rel(ug, uo, leaf):
    """max over leaf cells and both fields of |ug - uo| / |uo| (leaf: one
    field's leaf mask)."""
    N = leaf.size
    worst = 0.0
    for f in range(2):
        a = np.asarray(ug[f * N:(f + 1) * N])[leaf]
        b = np.asarray(uo[f * N:(f + 1) * N])[leaf]
        if a.size:
            worst = max(worst, float((np.abs(a - b) / np.abs(b)).max()))
    return worst
