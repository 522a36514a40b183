"""Parity at the launch shape of the dense benchmark (m = d = 4096, tau = 256: the
persistent iteration kernel over the whole GPU in clusters of 16 CTAs, phase 1 in
chunks of 600 slots with the fused FP64 factor, inverse and product), on a smaller
n so that the FP64 oracle runs in seconds.

* plain FP64, count and subsample sketches, heuristic momentum: w after 50
  iterations within 1e-8 of the oracle's w (same seed, same iteration count);
* mixed precision with the FP64 small solve and a refresh every 50 iterations (the
  benchmark's settings, tensor-core X^T X): solved to 1e-9, the library's final FP64
  residual equals the oracle's FP64 residual of the returned w, and w is within
  cond(A) * 1e-9 of the oracle's closed-form solution (A-norm error bound of a
  relative residual: ||w - w*|| / ||w*|| <= cond(A) ||A w - b|| / ||b||).
"""
import numpy as np
import pytest

import oracle
from synth import gaussian_problem

pytestmark = pytest.mark.gpu

N, D, TAU, LAM = 6000, 4096, 256, 1e-2


@pytest.fixture(scope="module")
def rs():
    import paper_2105_05565_gb300 as rs

    rs.lib()
    return rs


@pytest.fixture(scope="module")
def problem():
    X, y, _ = gaussian_problem(N, D, seed=77)
    A, b = oracle.form_system(X, y, LAM, "primal")
    return X, y, A, b


@pytest.mark.parametrize("kind", ["count", "subsample"])
def test_plain_fp64_at_benchmark_launch_shape(rs, problem, kind):
    X, y, A, b = problem
    K = 50
    with rs.Solver(X, y, LAM, sketch=kind, tau=TAU, momentum="heuristic", seed=3) as s:
        assert s.iter_ctas >= 64 and s.iter_ctas % 16 == 0  # the whole-GPU kernel
        w, hist, iters, _ = s.solve(tol=0.0, max_iters=K)
        chunk, refresh, fused = s.chunking()
    assert iters == K and fused == 1 and refresh == 0
    ref = oracle.sketch_and_project(A, b, kind, TAU, 3, 0.0, K, mom={"kind": "heuristic"})
    assert np.linalg.norm(w - ref["w"]) <= 1e-8 * np.linalg.norm(ref["w"])
    np.testing.assert_allclose(hist[:K + 1], ref["hist"][:K + 1], rtol=1e-8, atol=1e-14)


def test_mixed_fp64_small_solve_reaches_the_oracle_solution(rs, problem):
    X, y, A, b = problem
    tol = 1e-9
    with rs.Solver(X.astype(np.float32), y, LAM, sketch="count", tau=TAU, momentum="heuristic",
                   seed=3, precision="mixed") as s:
        assert s.iter_ctas >= 64 and s.iter_ctas % 16 == 0
        chunk, refresh, fused = s.chunking()
        w, hist, iters, conv = s.solve(tol=tol, max_iters=20000)
    assert (chunk, refresh, fused) == (600, 50, 1)
    assert conv and iters > 2 * refresh  # several refreshes inside the solve
    Xf = X.astype(np.float32).astype(np.float64)  # the data the library was given
    rel = oracle.true_residual(Xf, y, LAM, w)
    assert rel <= tol and abs(hist[iters] - rel) <= 1e-12
    w_star = oracle.direct_solution(Xf, y, LAM)
    ev = np.linalg.eigvalsh(A)
    cond = ev[-1] / ev[0]
    assert np.linalg.norm(w - w_star) <= cond * tol * np.linalg.norm(w_star)
