"""Momentum parameters (gamma_k, beta_k) of Algorithm 2.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Four settings (Section 8.1):

* ``none``      gamma_k = 1, beta_k = 0  (Algorithm 1).
* ``const``     gamma_k = gamma_c, beta_k = beta_c (the constant setting of
                Loizou & Richtarik; the paper uses gamma = 1, beta = 0.5).
* ``theory``    "increasing momentum", eq. (66): eta_k = eta while beta_k < 0.5,
                then eta_k = 1; zeta_k from eq. (40),
                zeta_k = (1/eta_k) sum_{t<k} eta_t (1 - eta_t), and
                gamma_k = eta_k / (1 + zeta_{k+1}), beta_k = zeta_k / (1 + zeta_{k+1})
                (eq. (38)).
* ``heuristic`` eq. (67): gamma_k = 1 and beta_k as in ``theory`` (the constant-eta
                closed form of eq. (50) until beta reaches 0.5, then frozen near
                0.5 by the eta switch); ``uncapped=True`` keeps the closed form
                beta_k = 1 - (2 - eta) / ((k + 1)(1 - eta) + 1) for every k.

Reading of the switch: the eta used at iteration k is fixed before gamma_k and
beta_k are formed (zeta_{k+1} is evaluated with eta_{k+1} = eta_k), and the
switch to eta = 1 applies from iteration k+1 on once beta_k >= beta_switch.
With constant eta this gives exactly the closed forms of eqs. (49)-(50).

Pinned by: tests/test_oracle_momentum.py (the closed forms of the corollary of
Section 6.2, the heavy-ball / iterate-averaging equivalence of the proposition
of Section 6.1, beta reaching 0.5 at k = 201 for eta = 0.995).
"""
from __future__ import annotations

import numpy as np


def momentum_schedule(kind: str, K: int, eta: float = 0.995, beta_switch: float = 0.5,
                      gamma_c: float = 1.0, beta_c: float = 0.5, uncapped: bool = False):
    """Arrays (gamma[0:K], beta[0:K]) in float64."""
    g = np.empty(K)
    b = np.empty(K)
    if kind == "none":
        g[:] = 1.0
        b[:] = 0.0
        return g, b
    if kind == "const":
        g[:] = gamma_c
        b[:] = beta_c
        return g, b
    if kind not in ("theory", "heuristic"):
        raise ValueError(f"unknown momentum kind {kind!r}")
    if kind == "heuristic" and uncapped:
        k = np.arange(K, dtype=np.float64)
        g[:] = 1.0
        b[:] = 1.0 - (2.0 - eta) / ((k + 1.0) * (1.0 - eta) + 1.0)
        return g, b
    acc = 0.0        # sum_{t<k} eta_t (1 - eta_t)
    eta_k = eta
    for k in range(K):
        zeta_k = acc / eta_k
        acc_next = acc + eta_k * (1.0 - eta_k)
        zeta_next = acc_next / eta_k
        gamma_k = eta_k / (1.0 + zeta_next)
        beta_k = zeta_k / (1.0 + zeta_next)
        g[k] = gamma_k if kind == "theory" else 1.0
        b[k] = beta_k
        acc = acc_next
        if beta_k >= beta_switch:
            eta_k = 1.0
    return g, b
