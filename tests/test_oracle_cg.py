"""Pins of the Conjugate Gradients oracle against properties that fix CG
independently of its recursion (Hestenes and Stiefel, 1952)."""
import numpy as np
import scipy.sparse as sp

import oracle
from oracle.cg import conjugate_gradients


def spd(m, seed, cond=50.0):
    g = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((m, m)))
    return Q @ np.diag(np.geomspace(1.0, cond, m)) @ Q.T


def test_iterates_minimise_the_A_norm_error_over_the_krylov_space():
    m = 12
    A = spd(m, 1)
    b = np.random.default_rng(2).standard_normal(m)
    w_star = np.linalg.solve(A, b)
    out = conjugate_gradients(A, b, 0.0, 6, record=True)
    K = np.zeros((m, 0))
    v = b.copy()
    for k in range(1, 7):
        K = np.column_stack([K, v])
        v = A @ v
        V, _ = np.linalg.qr(K)  # orthonormal basis of span{b, ..., A^{k-1} b}
        c = np.linalg.solve(V.T @ A @ V, V.T @ b)  # Galerkin = A-norm projection of w*
        wk = V @ c
        assert np.linalg.norm(out["ws"][k] - wk) <= 1e-10 * np.linalg.norm(w_star)


def test_orthogonal_residuals_and_conjugate_directions():
    m = 10
    A = spd(m, 3)
    b = np.random.default_rng(4).standard_normal(m)
    out = conjugate_gradients(A, b, 0.0, 8, record=True)
    R = np.array(out["rs"][:8])
    Pm = np.array(out["ps"][:8])
    G = R @ R.T
    assert np.abs(G - np.diag(np.diag(G))).max() <= 1e-10 * np.abs(np.diag(G)).max()
    C = Pm @ A @ Pm.T
    assert np.abs(C - np.diag(np.diag(C))).max() <= 1e-10 * np.abs(np.diag(C)).max()
    # the residual is the true A w - b at every step
    for w, r in zip(out["ws"], out["rs"]):
        assert np.linalg.norm(A @ w - b - r) <= 1e-10 * np.linalg.norm(b)


def test_exact_in_m_steps_and_ridge_closed_form():
    g = np.random.default_rng(5)
    X = g.standard_normal((40, 8))
    y = g.standard_normal(40)
    A, b = oracle.form_system(X, y, 0.5, "primal")
    out = conjugate_gradients(A, b, 0.0, 8)
    assert np.linalg.norm(out["w"] - np.linalg.solve(A, b)) <= 1e-12 * np.linalg.norm(b)
    out = conjugate_gradients(A, b, 1e-10, 1000)
    assert out["hist"][-1] <= 1e-10 and out["iters"] <= 12


def test_matrix_free_equals_dense():
    g = np.random.default_rng(6)
    Xs = sp.random(300, 50, density=0.05, random_state=7, format="csr")
    y = g.standard_normal(300)
    lam = 0.2
    A = (Xs.T @ Xs).toarray() + lam * np.eye(50)
    b = Xs.T @ y
    d = conjugate_gradients(A, b, 0.0, 20)
    f = conjugate_gradients(None, b, 0.0, 20, apply_A=lambda v: Xs.T @ (Xs @ v) + lam * v)
    # the two products round differently; 20 CG steps amplify that to about 1e-11
    assert np.linalg.norm(d["w"] - f["w"]) <= 1e-10 * np.linalg.norm(d["w"])
