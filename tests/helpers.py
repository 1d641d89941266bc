"""Shared numerical helpers of the test suite (test code only)."""

import numpy as np


def subspace_sin(X, X0):
    """sin of the largest principal angle between span(X) and span(X0), both with
    orthonormal columns: ||(I - X0 X0^T) X||_2, accurate down to rounding level
    (unlike sqrt(1 - cos^2))."""
    X = np.asarray(X, dtype=np.float64)
    X0 = np.asarray(X0, dtype=np.float64)
    return float(np.linalg.norm(X - X0 @ (X0.T @ X), 2))



def separated_prefix(s, rel_gap=1e-4):
    """The largest j < len(s) with (s[j-1] - s[j]) / s[0] >= rel_gap (0 if none):
    span of the first j singular vectors is well conditioned (its sensitivity to a
    perturbation of size e is about e / gap), unlike a subspace whose last value
    is nearly tied with the next."""
    s = np.asarray(s, dtype=np.float64)
    gaps = (s[:-1] - s[1:]) / s[0]
    idx = np.nonzero(gaps >= rel_gap)[0]
    return int(idx[-1] + 1) if idx.size else 0


def residual_gap_bound(sin_u, sin_v, sig_rel=0.0):
    """How far two residual maxima ||A v - s u|| / s_1 of nearby triplets may differ:
    |delta| <= ||A|| ||dv|| + |ds| + s ||du|| (in units of s_1), with ||dv||, ||du||
    at most 2 sin(angle) for sign-fixed unit vectors."""
    return 2.0 * (sin_u + sin_v) + sig_rel + 1e-12
