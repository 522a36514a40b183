"""Kernel ridge regression with the Gaussian (RBF) kernel (Section 2.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* eq. (Gausskernel): K(x, x') = exp(-||x - x'||^2 / (2 sigma^2)), written out from the
  differences of the points (no norm expansion);
* eq. (kernelridge): K (K + lambda I) alpha = K y, i.e. A alpha = b with
  A = K^T (K + lambda I), b = K^T y; predictions are K alpha.

Pinned by tests/test_oracle_kernel.py: K_ii = 1, symmetry, positive semidefiniteness
and a hand-computed entry; the solution of A alpha = b equals (K + lambda I)^{-1} y
for an invertible K (the dual of eq. (ridge_feature)); sketch-and-project on A
reaches it.
"""
from __future__ import annotations

import numpy as np


def rbf_kernel(X, sigma: float):
    """n x n Gaussian kernel matrix of the rows of X, eq. (Gausskernel)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    K = np.empty((n, n))
    for i in range(n):
        diff = X - X[i]
        K[i] = np.exp(-np.einsum("ij,ij->i", diff, diff) / (2.0 * sigma * sigma))
    return K


def kernel_system(K, y, lam: float):
    """A = K^T (K + lambda I), b = K^T y (eq. (kernelridge))."""
    K = np.asarray(K, dtype=np.float64)
    n = K.shape[0]
    A = K.T @ (K + lam * np.eye(n))
    b = K.T @ np.asarray(y, dtype=np.float64)
    return A, b
