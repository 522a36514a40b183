"""Failure detection through the C ABI, without faulting the GPU.

* Bounded device waits: the persistent iteration kernel's waits on the other CTAs
  are limited by rs_opts.spin_limit_ns. A fault-injection option (stall_ns) makes
  CTA 0 publish its first partials late, so the other CTAs' waits for them run out
  (a wait on data that does not arrive in time); the solve must end with
  RS_ETIMEOUT, with no hang, and the GPU and the library stay usable: the same
  context times out again the same way, and a context without the stall then
  solves the same problem to the oracle's answer.
* Non-finite input: NaN or Inf in y (injected on the host) gives RS_ENUMERIC from
  rs_solve, in both precisions.
"""
import numpy as np
import pytest

import oracle
from synth import gaussian_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import paper_2105_05565_gb300 as rs

    rs.lib()
    return rs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_wait_limit_runs_out_and_context_stays_usable(rs, precision):
    X, y, _ = gaussian_problem(3000, 1024, seed=21)
    lam = 0.5
    Xp = X if precision == "fp64" else X.astype(np.float32)
    kw = dict(sketch="count", tau=32, momentum="heuristic", seed=4, precision=precision)
    # waits of 20 us against a first exchange held back by 3 ms
    with rs.Solver(Xp, y, lam, spin_limit_ns=20_000, stall_ns=3_000_000, **kw) as s:
        assert s.iter_ctas > 1  # the persistent kernel over many CTAs runs this problem
        for _ in range(2):
            with pytest.raises(rs.RSError) as e:
                s.solve(tol=1e-8, max_iters=200)
            assert e.value.status == rs.RS_ETIMEOUT
    # the device and the library still work: the same problem without the stall
    with rs.Solver(Xp, y, lam, **kw) as s:
        w, hist, iters, conv = s.solve(tol=0.0, max_iters=60)
    assert iters == 60
    if precision == "fp64":
        ref = oracle.solve_ridge(X, y, lam, "primal", "count", 32, seed=4, tol=0.0, max_iters=60,
                                 mom={"kind": "heuristic"})
        assert np.linalg.norm(w - ref["w"]) <= 1e-8 * np.linalg.norm(ref["w"])
    else:
        assert np.isfinite(w).all() and hist[-1] < 1.0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_non_finite_target_gives_numeric_status(rs, precision, bad):
    X, y, _ = gaussian_problem(500, 128, seed=3)
    y = y.copy()
    y[17] = bad
    Xp = X if precision == "fp64" else X.astype(np.float32)
    with rs.Solver(Xp, y, 0.1, sketch="count", tau=16, momentum="heuristic",
                   precision=precision) as s:
        with pytest.raises(rs.RSError) as e:
            s.solve(tol=1e-6, max_iters=100)
        assert e.value.status == rs.RS_ENUMERIC
