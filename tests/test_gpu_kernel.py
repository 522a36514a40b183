"""Kernel ridge regression with the Gaussian kernel (Section 2.2, rs_create_kernel)
through the C ABI against the oracle (oracle.kernel):

* the kernel matrix: FP64 (differences of the points) within 1e-13; on the tensor
  cores within the TF32 bound |dK_ij| <= K_ij 2^-9 ||x_i|| ||x_j|| / (2 sigma^2) (the
  points rounded to TF32 perturb <x_i, x_j> by at most 2^-10 ||x_i|| ||x_j||), plus
  FP32 rounding of the exponential;
* plain FP64 iterates on K (K + lambda I) alpha = K y within 1e-8 of the oracle's;
* mixed sketch-and-project and mixed CG to 1e-6, FP64 CG to 1e-8, each checked in
  FP64 on the library's own K."""
import numpy as np
import pytest

import oracle
from oracle.cg import conjugate_gradients
from oracle.kernel import kernel_system, rbf_kernel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import paper_2105_05565_gb300 as rs

    rs.lib()
    return rs


def points(n, d, seed):
    g = np.random.default_rng(seed)
    P = g.standard_normal((n, d))
    y = np.sin(P[:, 0]) + 0.5 * P[:, 1] + 0.1 * g.standard_normal(n)
    return P, y


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("n,d", [(300, 5), (517, 40)])
def test_kernel_matrix_fp64_and_tensor_cores(rs, n, d):
    P, y = points(n, d, n)
    sigma = 1.5
    K_ref = rbf_kernel(P, sigma)
    with rs.Solver(P, y, 0.1, sketch="count", tau=16, kernel_sigma=sigma) as s:
        K64 = s.kernel_matrix()
    assert np.abs(K64 - K_ref).max() <= 1e-13
    P32 = P.astype(np.float32)
    K_ref32 = rbf_kernel(P32.astype(np.float64), sigma)
    with rs.Solver(P32, y, 0.1, sketch="count", tau=16, kernel_sigma=sigma,
                   precision="mixed") as s:
        K32 = s.kernel_matrix()
    nr = np.linalg.norm(P32.astype(np.float64), axis=1)
    bound = K_ref32 * (2.0 ** -9) * np.outer(nr, nr) / (2 * sigma * sigma) + 2e-7
    assert np.all(np.abs(K32 - K_ref32) <= 1.5 * bound)
    assert np.array_equal(K32, K32.T) and np.all(np.diag(K32) == 1.0)


@pytest.mark.parametrize("kind", ["count", "subsample"])
def test_plain_iterates_match_oracle(rs, kind):
    n, d, lam, sigma, K = 257, 6, 0.3, 1.2, 40
    P, y = points(n, d, 3)
    A, b = kernel_system(rbf_kernel(P, sigma), y, lam)
    with rs.Solver(P, y, lam, sketch=kind, tau=20, momentum="heuristic", seed=4,
                   kernel_sigma=sigma) as s:
        alpha, hist, iters, _ = s.solve(tol=0.0, max_iters=K)
    ref = oracle.sketch_and_project(A, b, kind, 20, 4, 0.0, K, mom={"kind": "heuristic"})
    assert iters == K and rel(alpha, ref["w"]) <= 1e-8


def test_mixed_and_cg_reach_tolerance_on_the_library_kernel(rs):
    # cond(A) ~ 1.1e8 here. The mixed iterations (sketch-and-project and CG alike) run
    # on the TF32-formed A, and their FP64 refinement contracts while cond(A) times
    # the relative TF32 error of A stays small: the FP64 residual of mixed CG stalls
    # near 1e-8, so both mixed solves target 1e-6; FP64 CG on the FP64 kernel reaches
    # 1e-8 (below)
    n, d, lam, sigma = 1024, 8, 1.0, 2.0
    P, y = points(n, d, 5)
    with rs.Solver(P.astype(np.float32), y, lam, sketch="count", tau=64, momentum="heuristic",
                   seed=1, kernel_sigma=sigma, precision="mixed") as s:
        Kl = s.kernel_matrix()
        alpha, hist, iters, conv = s.solve(tol=1e-6, max_iters=200000)
        alpha_cg, _, it_cg, conv_cg = s.solve_cg(tol=1e-6, max_iters=20000)
    A, b = kernel_system(Kl, y, lam)
    for a, tol, c in ((alpha, 1e-6, conv), (alpha_cg, 1e-6, conv_cg)):
        assert c and np.linalg.norm(A @ a - b) <= 1.01 * tol * np.linalg.norm(b)
    with rs.Solver(P, y, lam, sketch="count", tau=64, kernel_sigma=sigma) as s:
        a64, _, _, c64 = s.solve_cg(tol=1e-8, max_iters=20000)
        A64, b64 = kernel_system(s.kernel_matrix(), y, lam)
    assert c64 and np.linalg.norm(A64 @ a64 - b64) <= 1.01e-8 * np.linalg.norm(b64)
    # plain FP64 CG on the FP64 kernel: the oracle's CG iterates. At sigma = 2 this A has
    # cond ~ 2.5e8 and CG amplifies the rounding order of A (two oracle forms of A drift
    # 1e-7 apart in 8 steps); at sigma = 1 (cond ~ 7.7e3) they agree to 1e-12
    with rs.Solver(P, y, lam, sketch="count", tau=64, kernel_sigma=1.0) as s:
        a64, _, it64, _ = s.solve_cg(tol=0.0, max_iters=8)
    A64, b64 = kernel_system(rbf_kernel(P, 1.0), y, lam)
    ref = conjugate_gradients(A64, b64, 0.0, 8)
    assert it64 == 8 and rel(a64, ref["w"]) <= 1e-8
