"""Pins of the accelerated sketch-and-project oracle (Algorithm 3, Section 9)."""
import numpy as np

import oracle
from oracle.accel import accel_coefficients, accelerated_sketch_and_project


def problem(m, n, seed, lam=0.5):
    g = np.random.default_rng(seed)
    X = g.standard_normal((n, m)) * np.exp(g.uniform(-0.5, 0.5, m))
    y = g.standard_normal(n)
    return oracle.form_system(X, y, lam, "primal")


def test_mu_nu_one_is_the_plain_method():
    # alpha = 1/2, beta = 0, gamma = 1: z = v = w at every step (Section 9)
    assert np.allclose(accel_coefficients(1.0, 1.0), (0.5, 0.0, 1.0))
    A, b = problem(30, 90, 1)
    for kind in ("count", "subsample", "gaussian"):
        acc = accelerated_sketch_and_project(A, b, kind, 5, 3, 0.0, 40, 1.0, 1.0)
        ref = oracle.sketch_and_project(A, b, kind, 5, 3, 0.0, 40, mom={"kind": "none"})
        assert np.linalg.norm(acc["w"] - ref["w"]) <= 1e-12 * np.linalg.norm(ref["w"])


def test_residual_recursions_are_true_residuals():
    A, b = problem(25, 80, 2)
    out = accelerated_sketch_and_project(A, b, "count", 4, 1, 0.0, 50, 0.05, 8.0, record=True)
    for rec in out["records"]:
        assert np.linalg.norm(A @ rec["w"] - b - rec["rw"]) <= 1e-10 * np.linalg.norm(b)
        assert np.linalg.norm(A @ rec["v"] - b - rec["rv"]) <= 1e-10 * np.linalg.norm(b)


def test_no_sketching_solves_in_one_step():
    A, b = problem(12, 40, 3)
    w_star = np.linalg.solve(A, b)
    out = accelerated_sketch_and_project(A, b, "subsample", 12, 0, 0.0, 1, 0.3, 2.0)
    assert np.linalg.norm(out["w"] - w_star) <= 1e-12 * np.linalg.norm(w_star)


def test_theory_parameters_converge():
    # tau = 1 subsample (S = e_i with probability 1 / m). mu and nu of eq. (mu+nu) with Z
    # of eq. (Z) read in the A-norm, where a sketch-and-project step is an orthogonal
    # projection: Z_A = A^{1/2} S (S^T A S)^+ S^T A^{1/2}, so that 0 <= mu <= 1/nu <= 1
    # (the lemma quoted in Section 9); mu = lambda_min(E[Z_A]), nu = lambda_max of
    # E[Z_A]^{-1/2} E[Z_A E[Z_A]^{-1} Z_A] E[Z_A]^{-1/2}
    A, b = problem(8, 30, 4)
    m = 8
    ev, U = np.linalg.eigh(A)
    Ah = U @ np.diag(np.sqrt(ev)) @ U.T
    Zs = [np.outer(Ah[:, i], Ah[i, :]) / A[i, i] for i in range(m)]
    EZ = sum(Zs) / m
    EZi = np.linalg.inv(EZ)
    EZZ = sum(Z @ EZi @ Z for Z in Zs) / m
    ez, V = np.linalg.eigh(EZ)
    Ih = V @ np.diag(ez ** -0.5) @ V.T
    mu = ez[0]
    nu = np.linalg.eigvalsh(Ih @ EZZ @ Ih)[-1]
    assert 0 < mu <= 1.0 / nu <= 1.0 + 1e-12
    w_star = np.linalg.solve(A, b)
    out = accelerated_sketch_and_project(A, b, "subsample", 1, 5, 1e-11, 200000, mu, nu)
    assert np.linalg.norm(out["w"] - w_star) <= 1e-9 * np.linalg.norm(w_star)
