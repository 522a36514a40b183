"""Pins of the learned-proposal oracle: the network gradient against central finite
differences, Adam's first step against its closed form, the proposal's mixture
floor, the Gumbel-top-k law (tau = 1 frequencies match p; uniform inclusion), and
the per-step projection identity of Section 3 for learned samples, with the solve
reaching the closed-form ridge solution."""
import numpy as np
import pytest

import oracle
from oracle import learned as L
from synth import mlp_init


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = mlp_init(1) + 0.05 * rng.standard_normal(L.N_PARAMS)
    Z = rng.standard_normal((7, L.NF))
    y = rng.standard_normal(7)
    _, g = L.loss_grad(theta, Z, y)
    h = 1e-6
    fd = np.empty(L.N_PARAMS)
    for i in range(L.N_PARAMS):
        e = np.zeros(L.N_PARAMS)
        e[i] = h
        fd[i] = (L.loss_grad(theta + e, Z, y)[0] - L.loss_grad(theta - e, Z, y)[0]) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-5, atol=1e-9)
    # every block of the parameter vector takes part (no dropped term)
    W1, b1, W2, b2, w3, b3 = L.unpack(g)
    for blk in (W1, b1, W2, b2, w3):
        assert np.abs(blk).max() > 0
    assert b3 != 0


def test_bf16_forward_close_to_fp64():
    rng = np.random.default_rng(2)
    theta = mlp_init(3)
    Z = rng.standard_normal((200, L.NF))
    s64 = L.forward(theta, Z)
    s16 = L.forward(theta, Z, bf16_mode=True)
    assert np.abs(s16 - s64).max() <= 0.05 * (1 + np.abs(s64).max())
    assert np.array_equal(L.bf16(L.bf16(theta)), L.bf16(theta))


def test_adam_first_step_closed_form():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 4.0])
    st = {}
    t1 = L.adam_step(theta, g, st, lr=0.01)
    # m_hat = g, v_hat = g^2 after bias correction: a step of lr * g / (|g| + eps)
    assert np.allclose(t1, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    t2 = L.adam_step(t1, g, st, lr=0.01)
    assert np.allclose(t2, t1 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_proposal_is_a_distribution_with_floor():
    s = np.array([3.0, -1.0, 0.0, 10.0, -50.0])
    lp = L.log_proposal(s, 0.1)
    p = np.exp(lp)
    assert abs(p.sum() - 1.0) < 1e-12
    assert p.min() >= 0.1 / 5 - 1e-15
    assert np.argmax(p) == 3
    assert np.allclose(np.exp(L.log_proposal(s, 1.0)), 0.2)


def test_gumbel_top1_frequencies_follow_p():
    lp = np.log(np.array([0.5, 0.25, 0.15, 0.1]))
    n = 20000
    hits = np.zeros(4)
    for k in range(n):
        C, _ = L.select(lp, 7, k, 1)
        hits[C[0]] += 1
    freq = hits / n
    se = np.sqrt(np.exp(lp) * (1 - np.exp(lp)) / n)
    assert np.all(np.abs(freq - np.exp(lp)) < 5 * se)


def test_uniform_selection_inclusion_rate():
    m, tau, n = 12, 3, 6000
    hits = np.zeros(m)
    for k in range(n):
        C, _ = L.select(np.full(m, -np.log(m)), 11, k, tau)
        assert len(C) == tau and len(set(C)) == tau and np.all(np.diff(C) > 0)
        hits[C] += 1
    freq = hits / n
    assert np.all(np.abs(freq - tau / m) < 5 * np.sqrt(0.25 * 0.75 / n))


def test_learned_steps_obey_projection_identity_and_converge():
    rng = np.random.default_rng(5)
    n, d, lam = 60, 40, 0.3
    X = rng.standard_normal((n, d))
    y = rng.standard_normal(n)
    A, b = oracle.form_system(X, y, lam, "primal")
    w_star = np.linalg.solve(A, b)
    theta = mlp_init(4)
    out = L.solve_learned(A, b, theta, tau=6, seed=3, tol=1e-10, max_iters=4000, eps=0.5,
                          chunk=7, w_star=w_star, collect=True)
    assert out["iters"] < 4000
    assert np.linalg.norm(out["w"] - w_star) <= 1e-8 * np.linalg.norm(w_star)
    # replay: each step lowers ||e||_A^2 by exactly r_C . delta (Section 3)
    w = np.zeros(d)
    r = -b.copy()
    for C in out["samples"][:200]:
        e2 = (w - w_star) @ A @ (w - w_star)
        delta = np.linalg.solve(A[np.ix_(C, C)], r[C])
        w[C] -= delta
        e2n = (w - w_star) @ A @ (w - w_star)
        assert np.isclose(e2 - e2n, r[C] @ delta, rtol=1e-8, atol=1e-14)
        r = A @ w - b
    Zt, yt = out["data"]
    assert Zt.shape == (6 * out["iters"], 4) and yt.shape == (6 * out["iters"],)
    assert np.all(np.isfinite(yt))


def test_projection_identity_exact():
    rng = np.random.default_rng(8)
    d = 30
    B = rng.standard_normal((d, d))
    A = B @ B.T + 0.5 * np.eye(d)
    b = rng.standard_normal(d)
    w_star = np.linalg.solve(A, b)
    w = rng.standard_normal(d)
    r = A @ w - b
    for C in (np.array([0, 4, 9]), np.array([3]), np.arange(0, 30, 2)):
        delta = np.linalg.solve(A[np.ix_(C, C)], r[C])
        e2 = (w - w_star) @ A @ (w - w_star)
        wn = w.copy()
        wn[C] -= delta
        e2n = (wn - w_star) @ A @ (wn - w_star)
        assert np.isclose(e2 - e2n, r[C] @ delta, rtol=1e-10)
        # the label's normaliser: ||e||_A^2 = (w - w*) . r
        assert np.isclose(e2, (w - w_star) @ r, rtol=1e-10)
