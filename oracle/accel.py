"""Accelerated sketch-and-project (Algorithm 3, Section 9).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Parameters mu in (0, 1], nu in [1, 1 / mu]; beta = 1 - sqrt(mu / nu),
gamma = sqrt(1 / (mu nu)), alpha = 1 / (1 + sqrt(nu / mu)). From w^0 = v^0 = 0 and
r_w^0 = r_v^0 = A w^0 - b, iteration k:
    z^k = alpha v^k + (1 - alpha) w^k,   r_z^k = alpha r_v^k + (1 - alpha) r_w^k,
    delta^k = least-norm solution of (S^T A S) delta = S^T r_z^k,  g^k = S delta^k,
    w^{k+1} = z^k - g^k,                 r_w^{k+1} = r_z^k - A S delta^k,
    v^{k+1} = beta v^k + (1 - beta) z^k - gamma g^k,
    r_v^{k+1} = beta r_v^k + (1 - beta) r_z^k - gamma A S delta^k.
Readings of the printed listing: r_z^k is formed before delta^k (which uses it);
the while-condition's "<=" is read as ">"; the loop stops on ||r_w^k|| / ||r_w^0||,
the residual of the returned w^t (the listing monitors r_v, which leaves the output's
own residual unchecked).

Pinned by tests/test_oracle_accel.py: mu = nu = 1 is the plain method (z = v = w, as
Section 9 states), the residual recursions equal A w - b and A v - b, S = I solves in
one step, and with mu, nu computed from their definitions (eq. (mu+nu) with Z of
eq. (Z)) on a small problem the iteration converges to the closed form.
"""
from __future__ import annotations

import numpy as np

from .sketches import sketch_matrix
from .solver import least_norm_solution


def accel_coefficients(mu: float, nu: float):
    """(alpha, beta, gamma) of Algorithm 3."""
    if not (0.0 < mu <= 1.0 and 1.0 <= nu <= 1.0 / mu * (1.0 + 1e-12)):
        raise ValueError("need 0 < mu <= 1 <= nu <= 1 / mu")
    beta = 1.0 - np.sqrt(mu / nu)
    gamma = np.sqrt(1.0 / (mu * nu))
    alpha = 1.0 / (1.0 + np.sqrt(nu / mu))
    return alpha, beta, gamma


def accelerated_sketch_and_project(A, b, kind: str, tau: int, seed: int, tol: float,
                                   max_iters: int, mu: float, nu: float, s=None,
                                   record: bool = False):
    """Returns dict(w, hist, iters[, records of (w, v, r_w, r_v)])."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m = b.shape[0]
    alpha, beta, gamma = accel_coefficients(mu, nu)
    w = np.zeros(m)
    v = np.zeros(m)
    rw = -b.copy()
    rv = rw.copy()
    r0 = np.linalg.norm(rw)
    out = dict(w=w, hist=[1.0 if r0 > 0 else 0.0], iters=0, records=[])
    if r0 == 0.0:
        return out
    k = 0
    while k < max_iters and np.linalg.norm(rw) / r0 > tol:
        S = sketch_matrix(kind, m, tau, seed, k, s)
        AS = A @ S
        z = alpha * v + (1.0 - alpha) * w
        rz = alpha * rv + (1.0 - alpha) * rw
        delta = least_norm_solution(S.T @ AS, S.T @ rz)
        g = S @ delta
        Ag = AS @ delta
        w = z - g
        v = beta * v + (1.0 - beta) * z - gamma * g
        rw = rz - Ag
        rv = beta * rv + (1.0 - beta) * rz - gamma * Ag
        k += 1
        out["hist"].append(np.linalg.norm(rw) / r0)
        if record:
            out["records"].append(dict(w=w.copy(), v=v.copy(), rw=rw.copy(), rv=rv.copy()))
    out.update(w=w, iters=k)
    return out
