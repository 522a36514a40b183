"""Pins of the oracle's iteration (Algorithms 1-2) against what the paper and the
mathematics fix."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

import oracle.solver as osolver
from oracle import (direct_solution, form_system, sketch_and_project, solve_matrix_free,
                    solve_ridge, true_residual)
from oracle.rng import subsample_indices
from synth import gaussian_problem, zipf_csr

MOMS = [{"kind": "none"}, {"kind": "const"}, {"kind": "theory"}, {"kind": "heuristic"}]


def small_problem(n=60, d=14, seed=0):
    X, y, _ = gaussian_problem(n, d, seed)
    return X, y


@pytest.mark.parametrize("kind,tau", [("subsample", 4), ("count", 4), ("subcount", 3),
                                      ("gaussian", 3), ("srht", 5)])
@pytest.mark.parametrize("mom", MOMS, ids=lambda m: m["kind"])
def test_converges_to_closed_form(kind, tau, mom):
    """Eq. (2): the iteration reaches (X^T X + lam I)^{-1} X^T y."""
    X, y = small_problem()
    lam = 0.5
    w_star = direct_solution(X, y, lam)
    if mom["kind"] == "const" and kind in ("subsample", "subcount"):
        pytest.skip("constant momentum (beta = 0.5) with small blocks is not a contraction here")
    out = solve_ridge(X, y, lam, "primal", kind, tau, seed=1, tol=1e-13, max_iters=40000,
                      mom=mom, s=6 if kind == "subcount" else None)
    assert out["hist"][-1] <= 1e-13
    assert np.linalg.norm(out["w"] - w_star) <= 1e-10 * np.linalg.norm(w_star)
    assert true_residual(X, y, lam, out["w"]) <= 1e-11


def test_dual_equals_primal():
    """Lemma of Appendix A: X^T (X X^T + lam I)^{-1} y = (X^T X + lam I)^{-1} X^T y."""
    X, y, _ = gaussian_problem(12, 30, 3)
    lam = 0.7
    w_star = direct_solution(X, y, lam)
    out = solve_ridge(X, y, lam, "dual", "count", 4, seed=2, tol=1e-13, max_iters=20000,
                      mom={"kind": "heuristic"})
    assert np.linalg.norm(out["w"] - w_star) <= 1e-10 * np.linalg.norm(w_star)
    assert true_residual(X, y, lam, out["alpha"], form="dual") <= 1e-12


@pytest.mark.parametrize("kind,tau", [("subsample", 14), ("gaussian", 14), ("srht", 16)])
def test_one_step_exact(kind, tau):
    """tau = m (tau = m' for the SRHT): S has full row rank, the projection of
    eq. (10) lands on the solution in one step."""
    X, y = small_problem()
    lam = 0.2
    w_star = direct_solution(X, y, lam)
    out = solve_ridge(X, y, lam, "primal", kind, tau, seed=3, tol=0.0, max_iters=1)
    assert out["iters"] == 1
    assert np.linalg.norm(out["w"] - w_star) <= 1e-11 * np.linalg.norm(w_star)


@pytest.mark.parametrize("kind,tau", [("subsample", 3), ("count", 4), ("subcount", 2),
                                      ("gaussian", 3), ("srht", 4)])
def test_pathwise_A_norm_decrease(kind, tau):
    """Without momentum each step is an A-orthogonal projection (eqs. (10)-(12)):
    ||w^{k+1} - w*||_A^2 = ||w^k - w*||_A^2 - r_S^T delta, exactly."""
    X, y = small_problem()
    lam = 0.3
    A, b = form_system(X, y, lam)
    w_star = np.linalg.solve(A, b)
    K = 30
    out = sketch_and_project(A, b, kind, tau, 5, 0.0, K, record_first=K,
                             s=6 if kind == "subcount" else None)
    w = np.zeros_like(b)
    e2 = (w - w_star) @ A @ (w - w_star)
    for rec in out["records"]:
        e2_next = (rec["w"] - w_star) @ A @ (rec["w"] - w_star)
        dec = rec["rS"] @ rec["delta"]
        assert dec >= -1e-12
        assert abs(e2 - dec - e2_next) <= 1e-9 * max(e2, 1e-300)
        e2 = e2_next


def test_expected_one_step_decrease_by_enumeration():
    """Theorem of Section 5.1 with the subsample distribution of eq. (15): the
    exact expectation over all C(m, tau) subsets matches the oracle's Monte-Carlo
    average, and respects E||e^1||_A^2 <= (1 - rho) ||e^0||_A^2."""
    g = np.random.default_rng(7)
    m, tau = 6, 2
    Xs = g.standard_normal((10, m))
    A = Xs.T @ Xs + 0.5 * np.eye(m)
    b = g.standard_normal(m)
    w_star = np.linalg.solve(A, b)
    e0 = -w_star
    E0 = e0 @ A @ e0
    r0 = -b
    subsets = list(itertools.combinations(range(m), tau))
    EH = np.zeros((m, m))
    dec = 0.0
    for C in subsets:
        C = list(C)
        Minv = np.linalg.inv(A[np.ix_(C, C)])
        H = np.zeros((m, m))
        H[np.ix_(C, C)] = Minv
        EH += H / len(subsets)
        dec += r0[C] @ Minv @ r0[C] / len(subsets)
    exact = E0 - dec
    L = np.linalg.cholesky(A)
    rho = np.linalg.eigvalsh(L.T @ EH @ L).min()
    assert exact <= (1.0 - rho) * E0 + 1e-12
    N = 6000
    vals = np.empty(N)
    for seed in range(N):
        out = sketch_and_project(A, b, "subsample", tau, seed, 0.0, 1)
        e = out["w"] - w_star
        vals[seed] = e @ A @ e
    se = vals.std() / np.sqrt(N)
    assert abs(vals.mean() - exact) <= 4.5 * se


def test_expected_error_monotone_without_momentum():
    g = np.random.default_rng(8)
    m = 8
    Xs = g.standard_normal((12, m))
    A = Xs.T @ Xs + 0.2 * np.eye(m)
    b = g.standard_normal(m)
    w_star = np.linalg.solve(A, b)
    K, N = 6, 400
    E = np.zeros(K + 1)
    for seed in range(N):
        out = sketch_and_project(A, b, "count", 3, seed, 0.0, K, record_first=K)
        E[0] += w_star @ A @ w_star / N
        for k, rec in enumerate(out["records"]):
            e = rec["w"] - w_star
            E[k + 1] += e @ A @ e / N
    assert np.all(np.diff(E) < 0)


@pytest.mark.parametrize("kind", ["count", "gaussian", "srht"])
def test_invariance_under_right_multiplication(kind, monkeypatch):
    """S -> S Q (Q invertible) leaves S (S^T A S)^+ S^T unchanged, hence the iterates."""
    X, y = small_problem()
    A, b = form_system(X, y, 0.4)
    tau, K = 4, 12
    ref = sketch_and_project(A, b, kind, tau, 6, 0.0, K, mom={"kind": "heuristic"})
    orig = osolver.sketch_matrix
    Q = np.random.default_rng(9).standard_normal((tau, tau)) + 3 * np.eye(tau)

    def sq(*a, **kw):
        return orig(*a, **kw) @ Q

    monkeypatch.setattr(osolver, "sketch_matrix", sq)
    out = sketch_and_project(A, b, kind, tau, 6, 0.0, K, mom={"kind": "heuristic"})
    assert np.allclose(out["w"], ref["w"], rtol=1e-8, atol=1e-10)


def test_recursive_residual_is_true_residual():
    """Eqs. (13) and (53): the recursion tracks A w^k - b."""
    X, y = small_problem()
    A, b = form_system(X, y, 0.4)
    out = sketch_and_project(A, b, "count", 4, 2, 0.0, 200, mom={"kind": "heuristic"})
    true = np.linalg.norm(A @ out["w"] - b) / np.linalg.norm(b)
    assert abs(out["hist"][-1] - true) <= 1e-12


def test_tau_one_is_coordinate_descent():
    """Eq. (59) with gamma = 1, beta = 0: w_i -= (A_i: w - b_i) / A_ii."""
    X, y = small_problem()
    A, b = form_system(X, y, 0.4)
    K = 10
    out = sketch_and_project(A, b, "subsample", 1, 4, 0.0, K, record_first=K)
    w = np.zeros_like(b)
    for k in range(K):
        i = subsample_indices(4, k, b.size, 1)[0]
        w = w.copy()
        w[i] -= (A[i] @ w - b[i]) / A[i, i]
        assert np.allclose(out["records"][k]["w"], w, rtol=1e-13, atol=1e-15)


def test_empty_bucket_least_norm():
    """Count sketch with tau close to m leaves buckets empty: S^T A S is singular
    and the least-norm solve still gives the projection (delta_j = 0 there)."""
    X, y = small_problem()
    A, b = form_system(X, y, 0.4)
    out = sketch_and_project(A, b, "count", 12, 0, 0.0, 20, record_first=20)
    saw_empty = False
    for rec in out["records"]:
        empty = np.all(rec["S"] == 0, axis=0)
        if empty.any():
            saw_empty = True
            assert np.all(np.abs(rec["delta"][empty]) < 1e-12)
    assert saw_empty


def test_matrix_free_equals_dense():
    rowptr, col, val = zipf_csr(300, 40, 1500, 1)
    Xs = sp.csr_matrix((val, col, rowptr), shape=(300, 40))
    y = np.random.default_rng(2).standard_normal(300)
    lam = 0.1
    dense = solve_ridge(Xs.toarray(), y, lam, "primal", "subcount", 5, 3, 0.0, 30,
                        mom={"kind": "heuristic"}, s=20)
    mf = solve_matrix_free(Xs, y, lam, "subcount", 5, 3, 0.0, 30,
                           mom={"kind": "heuristic"}, s=20)
    assert np.allclose(mf["w"], dense["w"], rtol=1e-10, atol=1e-12)


def test_zero_rhs():
    A = np.eye(5) * 2.0
    out = sketch_and_project(A, np.zeros(5), "count", 2, 0, 1e-6, 10)
    assert out["iters"] == 0 and np.all(out["w"] == 0)
