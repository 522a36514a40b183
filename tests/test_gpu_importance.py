"""Importance-sampled subsample sketches (Section 7, p_j = A_jj / trace(A)) through
the C ABI (rs_set_sampling) against the oracle (oracle.importance) on the same
seeded inputs: the drawn rows of every iteration (rows that differ between the
FP32 keys of the GPU and the FP64 keys of the oracle must tie at the boundary
within rounding), the plain FP64 iterates with and without momentum (tau = 1 is
coordinate descent with momentum, eq. (CDmom)) within 1e-8, and the mixed path to
the FP64-checked tolerance."""
import numpy as np
import pytest

import oracle
from oracle import importance as IM
from synth import gaussian_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import paper_2105_05565_gb300 as rs

    rs.lib()
    return rs


def problem(m, n, seed, lam=0.3):
    g = np.random.default_rng(seed)
    X, y, _ = gaussian_problem(n, m, seed)
    X = X * np.exp(g.uniform(-1.0, 1.0, m))  # uneven column scales: uneven A_jj
    A, b = oracle.form_system(X, y, lam, "primal")
    return X, y, A, b, lam


@pytest.mark.parametrize("tau", [1, 5, 32])
def test_draws_follow_the_diagonal_like_the_oracle(rs, tau):
    m, seed = 97, 4
    X, y, A, b, lam = problem(m, 300, 11)
    logp = np.log(IM.diag_probabilities(A))
    with rs.Solver(X, y, lam, sketch="subsample", tau=tau, seed=seed) as s:
        s.set_sampling("diag")
        C = [s.dump_sketch(k)[0][:tau].copy() for k in range(20)]
    for k in range(20):
        keys = logp + oracle.learned.gumbel(seed, k, m)
        Cr = IM.importance_sample(logp, tau, seed, k)
        assert np.all(np.diff(C[k]) > 0) and len(C[k]) == tau
        diff = set(C[k].tolist()) ^ set(Cr.tolist())
        kth = np.sort(keys)[::-1][tau - 1]
        for j in diff:  # only rows whose keys tie with the boundary within FP32 rounding
            assert abs(keys[j] - kth) <= 1e-4 * (1 + abs(kth)), (k, j)


@pytest.mark.parametrize("tau,mom", [(1, "heuristic"), (8, "none"), (8, "heuristic")])
def test_plain_iterates_match_oracle(rs, tau, mom):
    m, seed, K = 120, 6, 60
    X, y, A, b, lam = problem(m, 400, 12)
    with rs.Solver(X, y, lam, sketch="subsample", tau=tau, momentum=mom, seed=seed) as s:
        s.set_sampling("diag")
        w, hist, iters, _ = s.solve(tol=0.0, max_iters=K)
    ref = IM.solve_importance(A, b, tau, seed, 0.0, K, mom={"kind": mom})
    assert iters == K
    assert np.linalg.norm(w - ref["w"]) <= 1e-8 * np.linalg.norm(ref["w"])


def test_back_to_uniform_draws(rs):
    m, seed, K = 64, 2, 30
    X, y, A, b, lam = problem(m, 200, 13)
    with rs.Solver(X, y, lam, sketch="subsample", tau=6, momentum="heuristic", seed=seed) as s:
        s.set_sampling("diag")
        s.solve(tol=0.0, max_iters=5)
        s.set_sampling("uniform")
        w, _, _, _ = s.solve(tol=0.0, max_iters=K)
    ref = oracle.sketch_and_project(A, b, "subsample", 6, seed, 0.0, K, mom={"kind": "heuristic"})
    assert np.linalg.norm(w - ref["w"]) <= 1e-8 * np.linalg.norm(ref["w"])


def test_mixed_importance_sampling_reaches_tolerance(rs):
    m = 512
    X, y, A, b, lam = problem(m, 2048, 14, lam=1e-2)
    with rs.Solver(X.astype(np.float32), y, lam, sketch="subsample", tau=32, momentum="heuristic",
                   seed=1, precision="mixed") as s:
        s.set_sampling("diag")
        w, hist, iters, conv = s.solve(tol=1e-6, max_iters=100000)
    Xf = X.astype(np.float32).astype(np.float64)
    assert conv and oracle.true_residual(Xf, y, lam, w) <= 1e-6


@pytest.mark.parametrize("kind,mom", [("count", "heuristic"), ("subsample", "none"),
                                      ("diag", "const")])
def test_averaged_iterates_match_oracle(rs, kind, mom):
    """rs_get_average: the mean of w^0..w^t (Section 5.2) against the oracle's, plain
    FP64; 'diag' is coordinate descent with p_i = A_ii / trace(A) and a constant step
    0.5 without momentum (the theorem's setting)."""
    m, seed, K = 150, 8, 70
    X, y, A, b, lam = problem(m, 500, 15)
    momd = {"kind": mom}
    kw = {}
    if mom == "const":
        momd.update(gamma_c=0.5, beta_c=0.0)
        kw = dict(gamma_c=0.5, beta_c=0.0)
    sk = "subsample" if kind == "diag" else kind
    tau = 1 if kind == "diag" else 12
    with rs.Solver(X, y, lam, sketch=sk, tau=tau, momentum=mom, seed=seed, **kw) as s:
        if kind == "diag":
            s.set_sampling("diag")
        s.set_averaging(True)
        w, _, iters, _ = s.solve(tol=0.0, max_iters=K)
        wbar = s.average()
    if kind == "diag":
        ref = IM.solve_importance(A, b, tau, seed, 0.0, K, mom=momd, average=True)
    else:
        ref = oracle.sketch_and_project(A, b, kind, tau, seed, 0.0, K, mom=momd, average=True)
    assert iters == K
    assert np.linalg.norm(w - ref["w"]) <= 1e-8 * np.linalg.norm(ref["w"])
    assert np.linalg.norm(wbar - ref["w_avg"]) <= 1e-8 * np.linalg.norm(ref["w_avg"])
