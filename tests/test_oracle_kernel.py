"""Pins of the kernel ridge oracle (Section 2.2, eqs. (Gausskernel), (kernelridge))."""
import math

import numpy as np

import oracle
from oracle.kernel import kernel_system, rbf_kernel


def test_rbf_entries_by_hand_and_structure():
    X = np.array([[0.0, 0.0], [3.0, 4.0], [1.0, 0.0]])
    K = rbf_kernel(X, sigma=5.0)
    # ||(0,0) - (3,4)||^2 = 25: exp(-25 / 50); ||(3,4) - (1,0)||^2 = 20: exp(-20 / 50)
    assert math.isclose(K[0, 1], math.exp(-0.5), rel_tol=1e-15)
    assert math.isclose(K[1, 2], math.exp(-0.4), rel_tol=1e-15)
    assert math.isclose(K[0, 2], math.exp(-1.0 / 50.0), rel_tol=1e-15)
    assert np.all(np.diag(K) == 1.0) and np.array_equal(K, K.T)
    G = rbf_kernel(np.random.default_rng(0).standard_normal((40, 3)), 0.7)
    assert np.linalg.eigvalsh(G)[0] >= -1e-12


def test_system_solution_is_the_dual_ridge_solution():
    g = np.random.default_rng(1)
    X = g.standard_normal((30, 4))
    y = g.standard_normal(30)
    lam = 0.1
    K = rbf_kernel(X, 1.3)
    A, b = kernel_system(K, y, lam)
    alpha = np.linalg.solve(A, b)
    assert np.linalg.norm(alpha - np.linalg.solve(K + lam * np.eye(30), y)) <= 1e-9 * np.linalg.norm(alpha)
    assert np.allclose(A, A.T, atol=1e-13)


def test_sketch_and_project_solves_the_kernel_system():
    g = np.random.default_rng(2)
    X = g.standard_normal((50, 3))
    y = np.sin(X[:, 0]) + 0.1 * g.standard_normal(50)
    lam = 0.5
    A, b = kernel_system(rbf_kernel(X, 1.0), y, lam)
    ref = np.linalg.solve(A, b)
    out = oracle.sketch_and_project(A, b, "subsample", 10, 0, 1e-12, 100000,
                                    mom={"kind": "heuristic"})
    # relative error <= cond(A) x relative residual (A is ill-conditioned: cond ~ 1e6)
    assert out["hist"][-1] <= 1e-12
    assert np.linalg.norm(out["w"] - ref) <= np.linalg.cond(A) * 1e-12 * np.linalg.norm(ref)
