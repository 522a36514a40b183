"""Conjugate Gradients (rs_solve_cg, the competitor of Section 8.3) through the C ABI
against the CG oracle (oracle.cg) on the same seeded inputs: plain FP64 iterates
and residual histories within 1e-8 (dense primal and dual, matrix-free CSR, and the
dense benchmark's size m = 4096), the iteration count to a tolerance, and the mixed
path (FP32 A, FP64 refresh through X) to the FP64-checked tolerance."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle.cg import conjugate_gradients
from synth import gaussian_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import paper_2105_05565_gb300 as rs

    rs.lib()
    return rs


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("m,n,K", [(97, 300, 25), (4096, 6000, 40)])
def test_plain_dense_iterates_match_oracle(rs, m, n, K):
    X, y, _ = gaussian_problem(n, m, seed=m)
    lam = 0.5
    A, b = oracle.form_system(X, y, lam, "primal")
    with rs.Solver(X, y, lam, sketch="count", tau=8) as s:
        w, hist, iters, _ = s.solve_cg(tol=0.0, max_iters=K)
    ref = conjugate_gradients(A, b, 0.0, K)
    assert iters == K
    assert rel(w, ref["w"]) <= 1e-8
    np.testing.assert_allclose(hist, ref["hist"], rtol=1e-8, atol=1e-15)


def test_plain_dense_to_tolerance_and_dual(rs):
    X, y, _ = gaussian_problem(150, 260, seed=5)  # n < d: the dual form
    lam = 0.3
    for form in ("primal", "dual"):
        A, b = oracle.form_system(X, y, lam, form)
        with rs.Solver(X, y, lam, form=form, sketch="count", tau=8) as s:
            w, hist, iters, conv = s.solve_cg(tol=1e-10, max_iters=5000)
        ref = conjugate_gradients(A, b, 1e-10, 5000)
        assert conv and abs(iters - ref["iters"]) <= 1
        w_ref = X.T @ ref["w"] if form == "dual" else ref["w"]
        assert rel(w, w_ref) <= 1e-8
        assert rel(w, oracle.direct_solution(X, y, lam)) <= 1e-7


# On Zipf-sparse X, CG amplifies the rounding of any two FP64 implementations quickly
# (the oracle's own dense and matrix-free products agree to 1e-10 after 10 iterations
# and drift to 1e-4 by 15, at lambda = 0.1 and at 20 alike), so iterates are compared
# after 10 iterations; the solve to tolerance is checked against the direct solution.
@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("lam", [0.1, 20.0])
def test_matrix_free_csr_matches_oracle(rs, bf16, lam):
    from synth import sparse_problem

    rowptr, colidx, vals, y, _ = sparse_problem(2000, 300, 12000, 9, bf16=bf16)
    Xs = sp.csr_matrix((vals, colidx, rowptr), shape=(2000, 300))
    K = 10
    X = rs.CSR(rowptr, colidx, vals, (2000, 300), bf16=bf16)
    with rs.Solver(X, y, lam, sketch="subcount", tau=16, precision="mixed" if bf16 else "fp64",
                   sub_s=160) as s:
        w, hist, iters, _ = s.solve_cg(tol=0.0, max_iters=K)
        w2, hist2, iters2, conv = s.solve_cg(tol=1e-9, max_iters=20000)
    XT = Xs.T.tocsr()
    b = XT @ y
    ref = conjugate_gradients(None, b, 0.0, K, apply_A=lambda v: XT @ (Xs @ v) + lam * v)
    assert iters == K and rel(w, ref["w"]) <= 1e-8
    np.testing.assert_allclose(hist, ref["hist"], rtol=1e-8, atol=1e-15)
    A = (XT @ Xs).toarray() + lam * np.eye(300)
    w_star = np.linalg.solve(A, b)
    assert conv and np.linalg.norm(A @ w2 - b) <= 1.01e-9 * np.linalg.norm(b)
    assert rel(w2, w_star) <= np.linalg.cond(A) * 1e-9


def test_mixed_dense_reaches_fp64_checked_tolerance(rs):
    from synth import geometric_sigma, spectrum_problem

    X, y, _ = spectrum_problem(3000, 512, geometric_sigma(512, 1e-3), seed=4, noise=0.01,
                               dtype=np.float32)
    lam = 1e-2
    with rs.Solver(X, y, lam, sketch="count", tau=32, precision="mixed") as s:
        w, hist, iters, conv = s.solve_cg(tol=1e-8, max_iters=20000)
        _, refresh, _ = s.chunking()
    assert conv and iters > refresh  # at least one refresh inside the solve
    Xf = X.astype(np.float64)
    assert oracle.true_residual(Xf, y, lam, w) <= 1e-8
    assert abs(hist[iters] - oracle.true_residual(Xf, y, lam, w)) <= 1e-12
