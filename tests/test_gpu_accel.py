"""Accelerated sketch-and-project (Algorithm 3, rs_set_acceleration) through the C ABI
against the oracle (oracle.accel) on the same seeded inputs: plain FP64 iterates
within 1e-8 for the bucket-row sketches (ragged sizes, and the dense benchmark's
launch shape m = 4096, tau = 256), mu = nu = 1 equal to Algorithm 1 on the GPU, the
mixed path to the FP64-checked tolerance, and the parameter checks."""
import numpy as np
import pytest

import oracle
from oracle.accel import accelerated_sketch_and_project
from synth import gaussian_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import paper_2105_05565_gb300 as rs

    rs.lib()
    return rs


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("kind,m,n,tau,K", [("count", 97, 300, 8, 60), ("subsample", 130, 400, 9, 60),
                                            ("subcount", 200, 500, 10, 40),
                                            ("count", 4096, 6000, 256, 30)])
def test_plain_iterates_match_oracle(rs, kind, m, n, tau, K):
    X, y, _ = gaussian_problem(n, m, seed=m + tau)
    lam = 0.5
    mu, nu = 0.02, 6.0
    A, b = oracle.form_system(X, y, lam, "primal")
    with rs.Solver(X, y, lam, sketch=kind, tau=tau, seed=7) as s:
        s.set_acceleration(mu, nu)
        w, hist, iters, _ = s.solve(tol=0.0, max_iters=K)
    ss = s.s if kind == "subcount" else None
    ref = accelerated_sketch_and_project(A, b, kind, tau, 7, 0.0, K, mu, nu, s=ss)
    assert iters == K
    assert rel(w, ref["w"]) <= 1e-8
    np.testing.assert_allclose(hist, ref["hist"], rtol=1e-8, atol=1e-15)


def test_mu_nu_one_is_algorithm_1(rs):
    X, y, _ = gaussian_problem(300, 80, seed=3)
    with rs.Solver(X, y, 0.3, sketch="count", tau=6, momentum="none", seed=2) as s:
        w0, _, _, _ = s.solve(tol=0.0, max_iters=50)
        s.set_acceleration(1.0, 1.0)
        w1, _, _, _ = s.solve(tol=0.0, max_iters=50)
        s.set_acceleration(0.0, 0.0)
        w2, _, _, _ = s.solve(tol=0.0, max_iters=50)
    assert rel(w1, w0) <= 1e-12 and rel(w2, w0) == 0.0


def test_mixed_accelerated_reaches_tolerance(rs):
    from synth import geometric_sigma, spectrum_problem

    X, y, _ = spectrum_problem(3000, 256, geometric_sigma(256), seed=7, noise=0.01,
                               dtype=np.float32)
    lam = 1e-2
    with rs.Solver(X, y, lam, sketch="count", tau=32, seed=2, precision="mixed") as s:
        s.set_acceleration(0.05, 4.0)
        w, hist, iters, conv = s.solve(tol=1e-6, max_iters=100000)
    assert conv and oracle.true_residual(X.astype(np.float64), y, lam, w) <= 1e-6


def test_bad_parameters(rs):
    X, y, _ = gaussian_problem(100, 40, seed=1)
    with rs.Solver(X, y, 0.3, sketch="count", tau=4) as s:
        for mu, nu in [(0.5, 3.0), (1.5, 1.0), (0.1, 0.5), (-0.1, 2.0)]:
            with pytest.raises(rs.RSError) as e:
                s.set_acceleration(mu, nu)
            assert e.value.status == rs.RS_EINVAL
    with rs.Solver(X, y, 0.3, sketch="gaussian", tau=4) as s:
        with pytest.raises(rs.RSError) as e:
            s.set_acceleration(0.1, 2.0)
        assert e.value.status == rs.RS_EUNSUPPORTED
