"""Pins of the momentum schedules (Sections 6.1-6.2, 8.1)."""
import numpy as np
import pytest

from oracle import form_system, momentum_schedule, sketch_and_project, sketch_matrix
from oracle.solver import least_norm_solution


def closed_gamma_beta(eta, K):
    # eq. (50): constant eta
    k = np.arange(K, dtype=float)
    den = (k + 1.0) * (1.0 - eta) + 1.0
    return eta / den, 1.0 - (2.0 - eta) / den


@pytest.mark.parametrize("eta", [0.5, 0.9, 0.995])
def test_theory_without_switch_is_closed_form(eta):
    K = 400
    g, b = momentum_schedule("theory", K, eta=eta, beta_switch=np.inf)
    gc, bc = closed_gamma_beta(eta, K)
    assert np.allclose(g, gc, rtol=1e-13, atol=0)
    assert np.allclose(b, bc, rtol=1e-12, atol=1e-15)


def test_eta_half_beta_is_k_over_k_plus_3():
    K = 50
    _, b = momentum_schedule("theory", K, eta=0.5, beta_switch=np.inf)
    k = np.arange(K)
    assert np.allclose(b, k / (k + 3.0), rtol=1e-13, atol=1e-16)


def test_switch_at_k201_and_freeze():
    K = 1000
    g, b = momentum_schedule("theory", K, eta=0.995)
    # in exact arithmetic beta_201 = 1 - 1.005/2.01 = 0.5: the switch is a tie that
    # rounding decides, so it happens at k = 201 or k = 202
    assert b[200] < 0.5 - 1e-4 and abs(b[201] - 0.5) < 1e-12
    first = int(np.argmax(b >= 0.5))
    assert first in (201, 202)
    # after the switch eta = 1 freezes zeta: beta and gamma stay constant near 0.5
    f = first + 1
    assert np.allclose(b[f:], b[f], rtol=0, atol=1e-15)
    assert abs(b[f] - 0.5) < 0.01 and abs(g[f] - 0.5) < 0.01
    assert abs(g[f] + b[f] - 1.0) < 1e-12  # gamma = 1/(1+zeta), beta = zeta/(1+zeta)


def test_heuristic_gamma_one_and_uncapped_closed_form():
    K = 500
    g, b = momentum_schedule("heuristic", K)
    assert np.all(g == 1.0)
    gt, bt = momentum_schedule("theory", K)
    assert np.array_equal(b, bt)
    gu, bu = momentum_schedule("heuristic", K, uncapped=True)
    _, bc = closed_gamma_beta(0.995, K)
    assert np.all(gu == 1.0) and np.allclose(bu, bc, rtol=1e-13)


def test_const_and_none():
    g, b = momentum_schedule("const", 10)
    assert np.all(g == 1.0) and np.all(b == 0.5)
    g, b = momentum_schedule("none", 10)
    assert np.all(g == 1.0) and np.all(b == 0.0)


@pytest.mark.parametrize("kind", ["subsample", "count"])
def test_heavy_ball_equals_iterate_averaging(kind):
    """Proposition of Section 6.1: the z/w iterate-averaging form (eqs. (36)-(37))
    with zeta_k = k(1 - eta) (eq. (49)) produces the heavy-ball iterates (eq. (35)).
    The z/w form below uses the exact residual A w - b and its own loop."""
    g = np.random.default_rng(1)
    X = g.standard_normal((40, 16))
    y = g.standard_normal(40)
    A, b = form_system(X, y, 0.3, "primal")
    eta, K, tau, seed = 0.8, 25, 5, 4
    out = sketch_and_project(A, b, kind, tau, seed, 0.0, K,
                             mom={"kind": "theory", "eta": eta, "beta_switch": np.inf},
                             record_first=K)
    hb = [rec["w"] for rec in out["records"]]
    w = np.zeros(16)
    z = w.copy()  # z^{-1} = w^0
    for k in range(K):
        S = sketch_matrix(kind, 16, tau, seed, k)
        grad = S @ least_norm_solution(S.T @ A @ S, S.T @ (A @ w - b))
        z = z - eta * grad
        zeta_next = (k + 1) * (1.0 - eta)
        w = (1.0 - 1.0 / (zeta_next + 1.0)) * w + z / (zeta_next + 1.0)
        assert np.allclose(w, hb[k], rtol=1e-9, atol=1e-11), k
