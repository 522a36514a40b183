"""Matrix-free sparse path (CSR X, A never formed) through the C ABI against the FP64
oracle's matrix-free loop on the same seeded inputs: sketched systems element by
element, plain FP64 iterates within 1e-8, mixed precision with bfloat16 values to the
FP64-checked tolerance, and the full-size Zipf configuration's FP64 products."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from synth import sparse_problem

pytestmark = pytest.mark.gpu

W_TOL = 1e-8


@pytest.fixture(scope="module")
def rs():
    import paper_2105_05565_gb300 as rs

    rs.lib()
    return rs


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def problem(n, d, nnz, seed, bf16):
    rowptr, colidx, vals, y, _ = sparse_problem(n, d, nnz, seed, bf16=bf16)
    Xs = sp.csr_matrix((vals, colidx, rowptr), shape=(n, d))
    return rowptr, colidx, vals, y, Xs


KINDS = [("subsample", 12, 0), ("count", 12, 0), ("subcount", 8, 48)]


@pytest.mark.parametrize("kind,tau,s_", KINDS, ids=[k[0] for k in KINDS])
@pytest.mark.parametrize("mom", ["none", "heuristic"])
@pytest.mark.parametrize("bf16", [False, True], ids=["f64", "bf16"])
def test_matrix_free_iterates_match_oracle(rs, kind, tau, s_, mom, bf16):
    # n = 997, d = 123: ragged against the 4096-row blocks and every warp width
    rowptr, colidx, vals, y, Xs = problem(997, 123, 3000, 11, bf16)
    lam, K = 0.1, 60
    ref = oracle.solve_matrix_free(Xs, y, lam, kind, tau, seed=5, tol=0.0, max_iters=K,
                                   mom={"kind": mom}, s=s_ or None)
    X = rs.CSR(rowptr, colidx, vals, (997, 123), bf16=bf16)
    with rs.Solver(X, y, lam, sketch=kind, tau=tau, momentum=mom, seed=5, sub_s=s_) as s:
        w, hist, iters, _ = s.solve(tol=0.0, max_iters=K)
    assert iters == K
    assert rel(w, ref["w"]) <= W_TOL
    assert np.allclose(hist, ref["hist"], rtol=1e-8, atol=1e-14)


def test_matrix_free_sketched_system(rs):
    """M = S^T (X^T X + lambda I) S, r_S and delta of one iteration."""
    rowptr, colidx, vals, y, Xs = problem(800, 90, 2500, 12, False)
    lam = 0.3
    A = (Xs.T @ Xs).toarray() + lam * np.eye(90)
    b = Xs.T @ y
    X = rs.CSR(rowptr, colidx, vals, (800, 90))
    with rs.Solver(X, y, lam, sketch="subcount", tau=9, seed=3, sub_s=45) as s:
        for k in (0, 1):
            w, wp, r, rp, kk = s.get_state()
            if k == 0:
                r = -b  # state of a fresh solve
                s.set_state(np.zeros(90), np.zeros(90), r, r, 0)
            M, rS, delta = s.probe_step()
            S = oracle.sketch_matrix("subcount", 90, 9, 3, kk, s=45)
            assert np.allclose(M, S.T @ A @ S, rtol=1e-12, atol=1e-12 * np.abs(M).max())
            assert np.allclose(rS, S.T @ r, rtol=1e-12, atol=1e-12 * np.abs(rS).max())
            ref = np.linalg.lstsq(S.T @ A @ S, S.T @ r, rcond=1e-12)[0]
            assert rel(S @ delta, S @ ref) <= 1e-10
            s.step(1)


def test_matrix_free_mixed_bf16_to_tolerance(rs):
    rowptr, colidx, vals, y, Xs = problem(5000, 400, 40000, 13, True)
    lam = 0.1
    X = rs.CSR(rowptr, colidx, vals, (5000, 400), bf16=True)
    with rs.Solver(X, y, lam, sketch="subcount", tau=40, momentum="heuristic", seed=2,
                   precision="mixed", sub_s=400) as s:
        w, hist, iters, conv = s.solve(tol=1e-6, max_iters=100000)
        assert conv
        assert abs(s.true_residual(w) - oracle.true_residual(Xs, y, lam, w)) <= 1e-10
    assert oracle.true_residual(Xs, y, lam, w) <= 1e-6
    A = (Xs.T @ Xs).toarray() + lam * np.eye(400)
    w_star = np.linalg.solve(A, Xs.T @ y)
    # ||w - w*|| / ||w*|| <= cond(A) ||A w - b|| / ||b|| (Zipf columns: cond(A) is large)
    assert rel(w, w_star) <= np.linalg.cond(A) * 1e-6


def test_inconsistent_csr_rejected(rs):
    rowptr = np.array([0, 2, 3], dtype=np.int64)
    colidx = np.array([0, 7, 1], dtype=np.int32)  # 7 is out of range for d = 5
    X = rs.CSR(rowptr, colidx, np.ones(3), (2, 5))
    with pytest.raises(rs.RSError) as e:
        rs.Solver(X, np.ones(2), 1.0, sketch="subsample", tau=2)
    assert e.value.status == rs.RS_EINVAL


def test_sparse_form_and_sketch_limits(rs):
    rowptr, colidx, vals, y, _ = problem(300, 40, 900, 14, False)
    X = rs.CSR(rowptr, colidx, vals, (300, 40))
    for kw in ({"form": "dual", "sketch": "count"}, {"sketch": "gaussian"}, {"sketch": "srht"}):
        with pytest.raises(rs.RSError) as e:
            rs.Solver(X, y, 1.0, tau=4, **kw)
        assert e.value.status == rs.RS_EUNSUPPORTED


def test_zipf_full_size_products_and_progress(rs):
    """The Zipf configuration at full size: CSR X 1e6 x 5e4, ~5e6 entries, bfloat16
    values, lambda 0.1, SubCount s = 4096 -> tau = 512, heuristic momentum, mixed.
    200 iterations; the library's FP64 true residual equals scipy's, and the solve
    makes progress."""
    n, d = 1_000_000, 50_000
    rowptr, colidx, vals, y, Xs = problem(n, d, 5_000_000, 3000, True)
    lam = 0.1
    X = rs.CSR(rowptr, colidx, vals, (n, d), bf16=True)
    with rs.Solver(X, y, lam, sketch="subcount", tau=512, momentum="heuristic", seed=0,
                   precision="mixed", sub_s=4096) as s:
        w, hist, iters, conv = s.solve(tol=1e-6, max_iters=200)
        assert iters == 200 and not conv
        got = s.true_residual(w)
    ref = oracle.true_residual(Xs, y, lam, w)
    assert abs(got - ref) <= 1e-10 * ref
    assert ref < 0.9 and hist[-1] < hist[1]
