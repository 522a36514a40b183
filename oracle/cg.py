"""Conjugate Gradients on the ridge system A w = b (Hestenes and Stiefel, 1952), the
competitor of Experiment 3 (Section 8.3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

With r = A w - b (the sign used by the sketch-and-project loop) and w^0 = 0:
    p^0 = -r^0;  for k = 0, 1, ...:
        v = A p^k,  alpha_k = (r^k . r^k) / (p^k . v),
        w^{k+1} = w^k + alpha_k p^k,  r^{k+1} = r^k + alpha_k v,
        beta_k = (r^{k+1} . r^{k+1}) / (r^k . r^k),  p^{k+1} = -r^{k+1} + beta_k p^k,
stopping when ||r^k|| / ||r^0|| <= tol or at max_iters. ``apply_A(v)`` replaces
A @ v (matrix-free: X^T (X v) + lambda v).

Pinned by tests/test_oracle_cg.py: w^k equals the minimiser of ||w - w*||_A over
the Krylov space span{b, A b, ..., A^{k-1} b} (computed from an explicit basis);
residuals are mutually orthogonal and directions A-conjugate; exact solution in m
steps; matrix-free = dense.
"""
from __future__ import annotations

import numpy as np


def conjugate_gradients(A, b, tol: float, max_iters: int, apply_A=None, record: bool = False):
    """Returns dict(w, hist, iters[, rs, ps]): hist[k] = ||r^k|| / ||r^0||."""
    b = np.asarray(b, dtype=np.float64)
    if apply_A is None:
        A = np.asarray(A, dtype=np.float64)
        apply_A = lambda v: A @ v  # noqa: E731
    m = b.shape[0]
    w = np.zeros(m)
    r = -b.copy()
    r0 = np.linalg.norm(r)
    out = dict(w=w, hist=[1.0 if r0 > 0 else 0.0], iters=0)
    if record:
        out.update(rs=[r.copy()], ps=[], ws=[w.copy()])
    if r0 == 0.0:
        return out
    p = -r
    rr = r @ r
    k = 0
    while k < max_iters and np.sqrt(rr) / r0 > tol:
        v = apply_A(p)
        alpha = rr / (p @ v)
        if record:
            out["ps"].append(p.copy())
        w = w + alpha * p
        r = r + alpha * v
        rr_new = r @ r
        beta = rr_new / rr
        p = -r + beta * p
        rr = rr_new
        k += 1
        out["hist"].append(np.sqrt(rr) / r0)
        if record:
            out["rs"].append(r.copy())
            out["ws"].append(w.copy())
    out.update(w=w, iters=k)
    return out
