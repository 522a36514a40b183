"""Batched solve (many problems, several right-hand sides each, one persistent launch
per chunk) through the C ABI against the FP64 oracle run problem by problem and
right-hand side by right-hand side on the same seeded inputs: plain FP64 iterates
within 1e-8, per-pair stopping, mixed precision to the FP64-checked tolerance, and
the degenerate cases (b = 0, one problem, one right-hand side)."""
import numpy as np
import pytest

import oracle
from synth import batched_problem, batched_specs

pytestmark = pytest.mark.gpu

W_TOL = 1e-8


@pytest.fixture(scope="module")
def rs():
    import paper_2105_05565_gb300 as rs

    rs.lib()
    return rs


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def make_batch(dims, nrhs, seed, dtype=np.float64):
    Xs, Ys = [], []
    for p, d in enumerate(dims):
        X, Y = batched_problem(4 * d, d, nrhs, seed + 31 * p, dtype=dtype)
        Xs.append(X)
        Ys.append(Y)
    return Xs, Ys


KINDS = [("subsample", None), ("count", None), ("subcount", 5)]


@pytest.mark.parametrize("kind,sfac", KINDS, ids=[k[0] for k in KINDS])
@pytest.mark.parametrize("mom", ["none", "heuristic"])
def test_plain_batch_iterates_match_oracle(rs, kind, sfac, mom):
    # three uneven problems, d ragged against every warp and CTA width
    dims, nrhs = [64, 100, 37], 3
    lams = [0.1, 0.5, 1e-3]
    taus = [8, 12, 4]
    Xs, Ys = make_batch(dims, nrhs, 40)
    K = 45
    sub_s = 0
    if sfac:
        taus = [4, 6, 3]
        sub_s = 0  # subcount: s = the default rule of each problem
    with rs.Batch(Xs, Ys, lams, sketch=kind, taus=taus, momentum=mom, seed=7,
                  sub_s=sub_s) as b:
        W, iters, resid, conv = b.solve(tol=0.0, max_iters=K)
    assert not conv
    assert (iters == K).all()
    for p, d in enumerate(dims):
        for r in range(nrhs):
            ref = oracle.solve_ridge(Xs[p], Ys[p][r], lams[p], "primal", kind, taus[p],
                                     seed=7 + p, tol=0.0, max_iters=K, mom={"kind": mom},
                                     s=None)
            assert rel(W[p][r], ref["w"]) <= W_TOL, (p, r)
            assert resid[p, r] == pytest.approx(ref["hist"][-1], rel=1e-8, abs=1e-14)


def test_plain_batch_stops_each_pair_at_tolerance(rs):
    dims, nrhs = [48, 80], 4
    lams = [1.0, 0.3]
    Xs, Ys = make_batch(dims, nrhs, 50)
    Ys[1][2] *= 1e-3  # a right-hand side of another scale stops on its own ||b||
    tol = 1e-5
    with rs.Batch(Xs, Ys, lams, sketch="count", taus=[6, 10], momentum="heuristic",
                  seed=3) as b:
        W, iters, resid, conv = b.solve(tol=tol, max_iters=20000)
    assert conv
    for p in range(2):
        for r in range(nrhs):
            ref = oracle.solve_ridge(Xs[p], Ys[p][r], lams[p], "primal", "count", [6, 10][p],
                                     seed=3 + p, tol=tol, max_iters=20000,
                                     mom={"kind": "heuristic"})
            k_ref = len(ref["hist"]) - 1
            assert abs(int(iters[p, r]) - k_ref) <= 1, (p, r, iters[p, r], k_ref)
            if iters[p, r] == k_ref:
                assert rel(W[p][r], ref["w"]) <= 1e-7
            assert oracle.true_residual(Xs[p], Ys[p][r], lams[p], W[p][r]) <= 1.01 * tol
            assert resid[p, r] <= tol


def test_mixed_batch_to_tolerance(rs):
    dims, nrhs = [96, 160, 57, 128], 4
    lams = [1e-2, 1.0, 0.1, 3e-3]
    Xs, Ys = make_batch(dims, nrhs, 60, dtype=np.float32)
    tol = 1e-6
    with rs.Batch(Xs, Ys, lams, sketch="count", momentum="heuristic", seed=11,
                  precision="mixed") as b:
        W, iters, resid, conv = b.solve(tol=tol, max_iters=200000)
        info = b.info()
    assert conv
    assert info["iter_threads"] in (128, 256, 512) and info["phase1_streams"] in (1, 2, 4)
    for p in range(len(dims)):
        X64 = Xs[p].astype(np.float64)
        A = X64.T @ X64 + lams[p] * np.eye(dims[p])
        for r in range(nrhs):
            t = oracle.true_residual(X64, Ys[p][r], lams[p], W[p][r])
            assert t <= tol * (1 + 1e-9), (p, r, t)
            assert abs(resid[p, r] - t) <= 1e-9 * tol + 1e-12, (p, r)
            w_star = np.linalg.solve(A, X64.T @ Ys[p][r])
            assert rel(W[p][r], w_star) <= np.linalg.cond(A) * tol


def test_batch_degenerate_cases(rs):
    # b = 0 for one right-hand side: converged at once with w = 0; one problem
    X, Y = batched_problem(120, 30, 2, 70, dtype=np.float64)
    Y[1] = 0.0
    with rs.Batch([X], [Y], [0.2], sketch="subsample", taus=[5], momentum="none", seed=1) as b:
        W, iters, resid, conv = b.solve(tol=1e-8, max_iters=50000)
    assert conv
    assert iters[0, 1] == 0 and resid[0, 1] == 0.0 and not W[0][1].any()
    ref = oracle.solve_ridge(X, Y[0], 0.2, "primal", "subsample", 5, seed=1, tol=1e-8,
                             max_iters=50000, mom={"kind": "none"})
    assert abs(int(iters[0, 0]) - (len(ref["hist"]) - 1)) <= 1
    # one right-hand side, tau = d (the subsample sketch solves in one step)
    X, Y = batched_problem(80, 20, 1, 71, dtype=np.float64)
    with rs.Batch([X], [Y], [0.5], sketch="subsample", taus=[20], seed=2) as b:
        W, iters, resid, conv = b.solve(tol=1e-10, max_iters=10)
    assert conv and iters[0, 0] == 1
    A = X.T @ X + 0.5 * np.eye(20)
    assert rel(W[0][0], np.linalg.solve(A, X.T @ Y[0])) <= 1e-10
    # max_iters = 0: nothing runs, w = 0
    with rs.Batch([X], [Y], [0.5], sketch="count", taus=[4], seed=2) as b:
        W, iters, resid, conv = b.solve(tol=1e-6, max_iters=0)
    assert not conv and iters[0, 0] == 0 and not W[0][0].any()


def test_batch_rejects_bad_arguments(rs):
    X, Y = batched_problem(40, 10, 2, 72, dtype=np.float64)
    with pytest.raises(rs.RSError) as e:
        rs.Batch([X], [Y], [1.0], sketch="gaussian", taus=[2])
    assert e.value.status == rs.RS_EUNSUPPORTED
    with pytest.raises(rs.RSError) as e:
        rs.Batch([X], [np.zeros((9, 40))], [1.0], sketch="count", taus=[2])
    assert e.value.status == rs.RS_EINVAL
    with pytest.raises(rs.RSError) as e:
        rs.Batch([X], [Y], [-1.0], sketch="count", taus=[2])
    assert e.value.status == rs.RS_EINVAL


def test_uneven_batch_mixed_sampled_pairs(rs):
    """24 problems with the uneven-size recipe (d log-uniform in [256, 1024], n = 4 d,
    lambda log-uniform in [1e-4, 1], tau = min(128, d / 8)), 4 right-hand sides,
    mixed precision: every pair reaches 1e-6 in the FP64 check, which the oracle's
    true residual confirms on sampled pairs."""
    d, n, lam = batched_specs(24, 5, dmin=256, dmax=1024)
    Xs, Ys = [], []
    for p in range(24):
        X, Y = batched_problem(int(n[p]), int(d[p]), 4, 900 + p)
        Xs.append(X)
        Ys.append(Y)
    taus = [min(128, int(v) // 8) for v in d]
    with rs.Batch(Xs, Ys, list(lam), sketch="count", taus=taus, momentum="heuristic", seed=0,
                  precision="mixed") as b:
        W, iters, resid, conv = b.solve(tol=1e-6, max_iters=100000)
    assert conv, (iters.max(), resid.max())
    for p, r in [(0, 0), (7, 3), (13, 1), (23, 2)]:
        t = oracle.true_residual(Xs[p].astype(np.float64), Ys[p][r], float(lam[p]), W[p][r])
        assert t <= 1e-6 * (1 + 1e-9) and abs(t - resid[p, r]) <= 1e-12


def test_tune_cache_keeps_the_autotuners_choice(rs, tmp_path):
    """rs_opts.tune_cache: the first batch tunes and writes its choice under a key of
    its shape; a second batch of the same shape takes the choice from the file. The
    file is then edited to another valid launch shape, which a third batch must use
    (so the file is really read), with the same iterates."""
    dims, nrhs = [64, 100, 37], 2
    lams, taus = [0.1, 0.5, 1e-3], [8, 12, 4]
    Xs, Ys = make_batch(dims, nrhs, 90)
    path = tmp_path / "tune.txt"

    def run():
        with rs.Batch(Xs, Ys, lams, sketch="count", taus=taus, momentum="heuristic", seed=2,
                      tune_cache=str(path)) as b:
            W, iters, resid, conv = b.solve(tol=0.0, max_iters=30)
            return W, b.info()

    W1, info1 = run()
    lines = path.read_text().split("\n")
    lines = [l for l in lines if l.strip()]
    assert len(lines) == 1
    key, t, ns = lines[0].split()
    assert (int(t), int(ns)) == (info1["iter_threads"], info1["phase1_streams"])
    W2, info2 = run()
    assert (info2["iter_threads"], info2["phase1_streams"]) == (int(t), int(ns))
    # another valid shape in the file: the next batch must take it
    other = 256 if int(t) != 256 else 128
    path.write_text(f"{key} {other} 1\n")
    W3, info3 = run()
    assert (info3["iter_threads"], info3["phase1_streams"]) == (other, 1)
    for p in range(len(dims)):
        for r in range(nrhs):
            assert rel(W3[p][r], W1[p][r]) <= 1e-12
            assert rel(W2[p][r], W1[p][r]) <= 1e-12
