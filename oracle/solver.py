"""Sketch-and-project with momentum, written out in float64 (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The loop follows Algorithm 2 of the paper (Section 6.3) step by step, with the
sketch of iteration k built as an explicit matrix S_k (``oracle.sketches``):

    w^{-1} = w^0 = 0,  r^{-1} = r^0 = A w^0 - b = -b,  k = 0
    while ||r^k|| / ||r^0|| > tol  and  k < max_iters:
        gamma_k, beta_k                                  (``oracle.momentum``)
        r_S     = S_k^T r^k                              (sketched residual)
        delta_k = least_norm_solution(S_k^T A S_k, r_S)  (eq. (14))
        w^{k+1} = (1 + beta_k) w^k - beta_k w^{k-1} - gamma_k S_k delta_k
        r^{k+1} = (1 + beta_k) r^k - beta_k r^{k-1} - gamma_k A S_k delta_k   (eq. (53))

With gamma = 1 and beta = 0 this is Algorithm 1 (eqs. (12)-(13)). The printed
while-condition of Algorithms 1-3 reads "<= epsilon"; the loop runs while the
relative residual is ABOVE the tolerance (the stopping rule stated in Section 3).

Pinned by tests/test_oracle_solver.py: closed-form solution (eqs. (2)-(3)),
one-step exactness of S = I_C with tau = m, the pathwise A-norm decrease of
each projection, the expected one-step decrease computed by enumerating all
subsets, invariance under S -> S Q, residual recursion = true residual,
coordinate descent for tau = 1 (eq. (59)), primal = dual (Lemma of Appendix A).
"""
from __future__ import annotations

import numpy as np

from .momentum import momentum_schedule
from .sketches import sketch_matrix

LSTSQ_RCOND = 1e-12


def form_system(X, y, lam: float, form: str = "primal"):
    """(A, b) of eq. (4): primal A = X^T X + lam I, b = X^T y (eq. (2));
    dual A = X X^T + lam I, b = y (eq. (3)). X is widened to float64."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if form == "primal":
        A = X.T @ X
        b = X.T @ y
    elif form == "dual":
        A = X @ X.T
        b = y.copy()
    else:
        raise ValueError(form)
    A[np.diag_indices_from(A)] += lam
    return A, b


def direct_solution(X, y, lam: float):
    """w* = (X^T X + lam I)^{-1} X^T y, the closed form of eq. (2), by a LAPACK
    Cholesky solve (the paper's direct baseline in Section 8.3 is LAPACK)."""
    import scipy.linalg as sla

    A, b = form_system(X, y, lam, "primal")
    return sla.cho_solve(sla.cho_factor(A, lower=True), b)


def least_norm_solution(M, rS, rcond: float = LSTSQ_RCOND):
    """Least-norm solution of M x = rS (the ``least_norm_solution`` step of
    Algorithms 1-2; (S^T A S)^dagger S^T r in eq. (12)), by an SVD least-squares
    solve with singular values below rcond * sigma_max treated as zero."""
    x, *_ = np.linalg.lstsq(M, rS, rcond=rcond)
    return x


def sketch_and_project(A, b, kind: str, tau: int, seed: int, tol: float, max_iters: int,
                       mom=None, s=None, record_first: int = 0, apply_A=None, sketch_fn=None,
                       average: bool = False):
    """Algorithm 2 on A w = b. ``apply_A(V)`` (default ``A @ V``) gives A V for
    an m x tau block V, so that the matrix-free form can reuse the loop.
    ``sketch_fn(k)``, if given, returns S_k in place of the sketch of ``kind``
    (a sampler whose law depends on A, e.g. ``oracle.importance``).

    Returns dict(w, hist, iters, records): hist[k] = ||r^k|| / ||r^0|| for
    k = 0..iters; records holds (S, r_S, M, delta, w, r) of the first
    ``record_first`` iterations. With ``average``, also w_avg, the mean of the
    iterates w^0, ..., w^t (t = iters) of the theorem of Section 5.2.
    """
    mom = dict(mom or {"kind": "none"})
    mkind = mom.pop("kind", "none")
    b = np.asarray(b, dtype=np.float64)
    m = b.shape[0]
    if apply_A is None:
        A = np.asarray(A, dtype=np.float64)
        apply_A = lambda V: A @ V  # noqa: E731
    gam, bet = momentum_schedule(mkind, max(int(max_iters), 1), **mom)
    w = np.zeros(m)
    w_prev = np.zeros(m)
    r = -b.copy()
    r_prev = r.copy()
    r0 = np.linalg.norm(r)
    if r0 == 0.0:
        out = dict(w=w, hist=[0.0], iters=0, records=[])
        if average:
            out["w_avg"] = w.copy()
        return out
    hist = [1.0]
    records = []
    w_sum = w.copy()  # sum of w^0 .. w^k
    k = 0
    while k < max_iters and np.linalg.norm(r) / r0 > tol:
        S = sketch_fn(k) if sketch_fn is not None else sketch_matrix(kind, m, tau, seed, k, s)
        AS = apply_A(S)
        rS = S.T @ r
        M = S.T @ AS
        delta = least_norm_solution(M, rS)
        g, be = gam[k], bet[k]
        w_new = (1.0 + be) * w - be * w_prev - g * (S @ delta)
        r_new = (1.0 + be) * r - be * r_prev - g * (AS @ delta)
        w_prev, w = w, w_new
        r_prev, r = r, r_new
        if k < record_first:
            records.append(dict(k=k, S=S, rS=rS, M=M, delta=delta, w=w.copy(), r=r.copy()))
        k += 1
        w_sum = w_sum + w
        hist.append(np.linalg.norm(r) / r0)
    out = dict(w=w, hist=hist, iters=k, records=records)
    if average:
        out["w_avg"] = w_sum / (k + 1)
    return out


def solve_ridge(X, y, lam: float, form: str, kind: str, tau: int, seed: int, tol: float,
                max_iters: int, mom=None, s=None, record_first: int = 0):
    """Ridge regression through Algorithm 2: form A, b (eq. (4)), iterate, and for
    the dual form recover w = X^T alpha (eq. (3))."""
    A, b = form_system(X, y, lam, form)
    out = sketch_and_project(A, b, kind, tau, seed, tol, max_iters, mom, s, record_first)
    if form == "dual":
        out["alpha"] = out["w"]
        out["w"] = np.asarray(X, dtype=np.float64).T @ out["alpha"]
    return out


def solve_matrix_free(Xs, y, lam: float, kind: str, tau: int, seed: int, tol: float,
                      max_iters: int, mom=None, s=None, record_first: int = 0):
    """Primal ridge on a scipy.sparse X without forming A: A V = X^T (X V) + lam V
    and b = X^T y (eq. (2)); otherwise identical to ``sketch_and_project``."""
    import scipy.sparse as sp

    Xs = sp.csr_matrix(Xs, dtype=np.float64)
    XT = Xs.T.tocsr()
    b = XT @ np.asarray(y, dtype=np.float64)

    def apply_A(V):
        return XT @ (Xs @ V) + lam * V

    return sketch_and_project(None, b, kind, tau, seed, tol, max_iters, mom, s,
                              record_first, apply_A=apply_A)


def true_residual(X, y, lam: float, w, form: str = "primal"):
    """||A v - b|| / ||b|| evaluated through X in float64 (v = w for the primal,
    v = alpha for the dual form), without forming A."""
    import scipy.sparse as sp

    if sp.issparse(X):
        X = sp.csr_matrix(X, dtype=np.float64)
    else:
        X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    v = np.asarray(w, dtype=np.float64)
    if form == "primal":
        b = X.T @ y
        res = X.T @ (X @ v) + lam * v - b
    else:
        b = y
        res = X @ (X.T @ v) + lam * v - b
    return float(np.linalg.norm(res) / np.linalg.norm(b))
