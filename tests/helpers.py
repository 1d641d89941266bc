"""Shared numerical helpers of the test suite (test code only)."""

import numpy as np


def subspace_sin(X, X0):
    """sin of the largest principal angle between span(X) and span(X0), both with
    orthonormal columns: ||(I - X0 X0^T) X||_2, accurate down to rounding level
    (unlike sqrt(1 - cos^2))."""
    X = np.asarray(X, dtype=np.float64)
    X0 = np.asarray(X0, dtype=np.float64)
    return float(np.linalg.norm(X - X0 @ (X0.T @ X), 2))

