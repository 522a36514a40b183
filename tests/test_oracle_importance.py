"""Pins of the importance-sampling oracle (Section 7) and of the averaged iterates
(Section 5.2), each against what the paper fixes independently of the code:

* the lemma of Section 7: with p_i = A_ii / trace(A) and S = e_i, E[H_S] equals
  I / trace(A) exactly (enumeration of the m outcomes), so lambda_min(E[H_S]) =
  1 / trace(A); the uniform law does not give a multiple of I unless A_ii is
  constant;
* the Gumbel-top-1 sampler draws coordinate i with frequency p_i (chi-square);
* eq. (CDmom) on every recorded step of coordinate descent with momentum;
* convergence to the closed-form ridge solution (eq. (2));
* the averaged-iterate bound (eq. (convressublinear)), in expectation over runs,
  with W = A and lambda_min(E[H_S]) = 1 / trace(A)."""
import numpy as np

import oracle
from oracle import importance as IM


def spd(m, seed, spread=30.0):
    g = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((m, m)))
    D = np.diag(np.exp(np.linspace(0.0, np.log(spread), m)))
    A = Q @ D @ Q.T
    s = np.exp(g.uniform(-1.0, 1.0, m))  # uneven diagonal
    return s[:, None] * A * s[None, :]


def test_expected_H_is_identity_over_trace():
    A = spd(6, 1)
    p = IM.diag_probabilities(A)
    assert abs(p.sum() - 1.0) < 1e-15 and (p > 0).all()
    H = IM.expected_H(A, p)
    assert np.allclose(H, np.eye(6) / np.trace(A), rtol=0, atol=1e-15)
    assert abs(np.linalg.eigvalsh(H)[0] - 1.0 / np.trace(A)) < 1e-15
    # the uniform law gives diag(1 / (m A_ii)): not a multiple of I here
    Hu = IM.expected_H(A, np.full(6, 1.0 / 6))
    assert np.allclose(Hu, np.diag(1.0 / (6 * np.diag(A))), atol=1e-15)
    assert np.ptp(np.diag(Hu)) > 1e-3


def test_single_coordinate_frequencies_follow_the_diagonal():
    A = spd(5, 2)
    p = IM.diag_probabilities(A)
    logp = np.log(p)
    N = 20000
    cnt = np.zeros(5)
    for k in range(N):
        (i,) = IM.importance_sample(logp, 1, seed=9, k=k)
        cnt[i] += 1
    chi2 = (((cnt - N * p) ** 2) / (N * p)).sum()
    assert chi2 < 20.5  # 4 degrees of freedom, p-value about 4e-4


def test_blocks_are_distinct_sorted_and_favour_large_diagonals():
    A = spd(40, 3, spread=5.0)
    p = IM.diag_probabilities(A)
    cnt = np.zeros(40)
    for k in range(3000):
        C = IM.importance_sample(np.log(p), 8, seed=1, k=k)
        assert len(set(C.tolist())) == 8 and (np.diff(C) > 0).all()
        cnt[C] += 1
    # inclusion rates increase with p (Spearman-style check on the extremes)
    lo, hi = np.argsort(p)[:8], np.argsort(p)[-8:]
    assert cnt[hi].mean() > 1.5 * cnt[lo].mean()


def test_cd_with_momentum_matches_eq_CDmom_step_by_step():
    A = spd(7, 4)
    b = np.random.default_rng(5).standard_normal(7)
    out = IM.solve_importance(A, b, 1, seed=3, tol=0.0, max_iters=40,
                              mom={"kind": "heuristic"}, record_first=40)
    gam, bet = oracle.momentum_schedule("heuristic", 40)
    w_prev = np.zeros(7)
    w = np.zeros(7)
    for k, rec in enumerate(out["records"]):
        (i,) = np.nonzero(rec["S"][:, 0])[0]
        step = np.zeros(7)
        step[i] = (A[i] @ w - b[i]) / A[i, i]
        expect = w - gam[k] * step + bet[k] * (w - w_prev)
        assert np.allclose(rec["w"], expect, rtol=1e-13, atol=1e-13)
        w_prev, w = w, rec["w"]


def test_importance_blocks_reach_the_closed_form():
    g = np.random.default_rng(6)
    X = g.standard_normal((60, 20)) * np.exp(g.uniform(-1.5, 1.5, 20))
    y = g.standard_normal(60)
    lam = 0.3
    A, b = oracle.form_system(X, y, lam, "primal")
    w_star = np.linalg.solve(A, b)
    for tau, mom in [(1, "none"), (4, "heuristic")]:
        out = IM.solve_importance(A, b, tau, seed=2, tol=1e-12, max_iters=200000,
                                  mom={"kind": mom})
        assert np.linalg.norm(out["w"] - w_star) <= 1e-10 * np.linalg.norm(w_star)


def test_averaged_iterates_bound_in_expectation():
    # constant step gamma in (0, 1), no momentum, W = A, CD with p_i = A_ii / trace(A):
    # E ||A wbar^t - b||^2 <= trace(A) ||w^0 - w*||_A^2 / (2 gamma (1 - gamma) t)
    A = spd(8, 7, spread=50.0)
    b = np.random.default_rng(8).standard_normal(8)
    w_star = np.linalg.solve(A, b)
    gamma, t = 0.5, 60
    runs = []
    for seed in range(200):
        out = IM.solve_importance(A, b, 1, seed=seed, tol=0.0, max_iters=t,
                                  mom={"kind": "const", "gamma_c": gamma, "beta_c": 0.0},
                                  average=True, record_first=t)
        ws = [np.zeros(8)] + [r["w"] for r in out["records"]]
        assert np.allclose(out["w_avg"], np.mean(ws, axis=0), rtol=0, atol=1e-13)
        runs.append(np.linalg.norm(A @ out["w_avg"] - b) ** 2)
    bound = np.trace(A) * (w_star @ A @ w_star) / (2 * gamma * (1 - gamma) * t)
    assert np.mean(runs) <= bound
