"""Importance-sampled blocks, p_j proportional to A_jj (Section 7), and coordinate
descent with momentum.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* Eq. (mSdisccol) with unit coordinate vectors s_i = e_i is eq. (mSdisccolCD):
  P(S = e_i) = A_ii / trace(A). With this law E[H_S] = sum_i p_i e_i e_i^T / A_ii
  = I / trace(A) (the lemma of Section 7), so lambda_min(E[H_S]) = 1 / trace(A).
* tau = 1: Algorithm 2 with S = e_i is coordinate descent with momentum, eq. (CDmom):
  w^{k+1} = w^k - gamma_k (A_i: w^k - b_i) / A_ii e_i + beta_k (w^k - w^{k-1}).
* tau > 1 (a reading; the paper states the law for single columns): the tau
  coordinates of iteration k are drawn without replacement in proportion to A_jj,
  as the tau largest keys ln p_j + g_j, with g_j the Gumbel noise of iteration k
  that ``oracle.learned.gumbel`` defines (ties: smaller index), in increasing index
  order. For tau = 1 this is exactly eq. (mSdisccolCD) (the Gumbel-max law).

Pinned by tests/test_oracle_importance.py: E[H_S] = I / trace(A) by enumeration,
sample frequencies against p, the CD update of eq. (CDmom) on every recorded step,
convergence to the closed form, and the averaged-iterate bound of Section 5.2.
"""
from __future__ import annotations

import numpy as np

from .learned import gumbel
from .solver import sketch_and_project


def diag_probabilities(A):
    """p_i = A_ii / trace(A), eq. (mSdisccolCD)."""
    d = np.diag(np.asarray(A, dtype=np.float64))
    return d / d.sum()


def expected_H(A, p):
    """E[H_S] = sum_i p_i e_i (e_i^T A e_i)^+ e_i^T for S = e_i with probability p_i
    (the expectation written out over the m outcomes)."""
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    H = np.zeros((m, m))
    for i in range(m):
        e = np.zeros((m, 1))
        e[i] = 1.0
        H += p[i] * e @ np.linalg.pinv(e.T @ A @ e) @ e.T
    return H


def importance_sample(logp, tau: int, seed: int, k: int):
    """Coordinates of iteration k: the tau largest ln p_j + g_j (ties: smaller
    index), in increasing index order."""
    keys = np.asarray(logp, dtype=np.float64) + gumbel(seed, k, len(logp))
    order = np.lexsort((np.arange(len(keys)), -keys))
    return np.sort(order[:tau])


def solve_importance(A, b, tau: int, seed: int, tol: float, max_iters: int, mom=None,
                     record_first: int = 0, average: bool = False):
    """Algorithm 2 with subsample sketches S_k = I[:, C_k], C_k drawn in proportion to
    the diagonal of A (tau = 1: coordinate descent with momentum, eq. (CDmom))."""
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    logp = np.log(diag_probabilities(A))

    def sketch(k):
        C = importance_sample(logp, tau, seed, k)
        S = np.zeros((m, tau))
        S[C, np.arange(tau)] = 1.0
        return S

    out = sketch_and_project(A, b, "subsample", tau, seed, tol, max_iters, mom=mom,
                             record_first=record_first, sketch_fn=sketch, average=average)
    return out
