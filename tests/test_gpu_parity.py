"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same
seeded inputs. Sketch indices/signs/buckets bit-exact; plain FP64 iterates within
1e-8 relative; sketched systems and steps element by element."""
import numpy as np
import pytest

import oracle
from oracle import rng as orng
from oracle.sketches import srht_pad, subcount_params
from synth import gaussian_problem

pytestmark = pytest.mark.gpu

W_TOL = 1e-8  # plain FP64 path: relative error of w vs the oracle (same seed, same k)


@pytest.fixture(scope="module")
def rs():
    import paper_2105_05565_gb300 as rs

    rs.lib()
    return rs


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- sketches ---
@pytest.mark.parametrize("m,tau", [(50, 7), (500, 50), (4096, 256), (1000, 1000)])
def test_subsample_indices_bitexact(rs, m, tau):
    X, y, _ = gaussian_problem(m + 3, m, 0)
    with rs.Solver(X, y, 1.0, sketch="subsample", tau=tau, seed=12) as s:
        for k in [0, 1, 7, 123]:
            idx, _, _ = s.dump_sketch(k)
            assert np.array_equal(idx[:tau], orng.subsample_indices(12, k, m, tau))


@pytest.mark.parametrize("m,tau", [(97, 5), (500, 50), (4096, 256), (300, 290)])
def test_count_buckets_signs_bitexact(rs, m, tau):
    X, y, _ = gaussian_problem(m + 1, m, 1)
    with rs.Solver(X, y, 1.0, sketch="count", tau=tau, seed=3) as s:
        for k in [0, 2, 55]:
            idx, sign, bucket = s.dump_sketch(k)
            osign, obucket = orng.signs_buckets(3, k, m, tau)
            assert np.array_equal(bucket[:m], obucket)
            assert np.array_equal(sign[:m], osign)
            # rows grouped by bucket, ascending row inside a bucket
            assert np.array_equal(idx[:m], np.lexsort((np.arange(m), obucket)))


@pytest.mark.parametrize("m,tau,s_", [(500, 10, 0), (4096, 256, 0), (1000, 50, 400), (64, 8, 64)])
def test_subcount_bitexact(rs, m, tau, s_):
    X, y, _ = gaussian_problem(m + 1, m, 2)
    with rs.Solver(X, y, 1.0, sketch="subcount", tau=tau, seed=4, sub_s=s_) as sv:
        ss, kk = subcount_params(m, tau, s_ or None)
        assert (sv.s, sv.k_sum) == (ss, kk)
        for k in [0, 9]:
            idx, sign, bucket = sv.dump_sketch(k)
            assert np.array_equal(idx[:ss], orng.subsample_indices(4, k, m, ss))
            assert np.array_equal(sign[:ss], orng.signs_buckets(4, k, ss, tau)[0])
            assert np.array_equal(bucket[:ss], np.arange(ss) // kk)


@pytest.mark.parametrize("m,tau", [(100, 20), (512, 64), (4096, 256)])
def test_srht_bitexact(rs, m, tau):
    X, y, _ = gaussian_problem(m + 1, m, 5)
    with rs.Solver(X, y, 1.0, sketch="srht", tau=tau, seed=6) as s:
        mp = srht_pad(m)
        assert s.m_pad == mp
        for k in [0, 3]:
            idx, sign, _ = s.dump_sketch(k)
            assert np.array_equal(idx[:tau], orng.subsample_indices(6, k, mp, tau))
            assert np.array_equal(sign[:m], orng.signs_buckets(6, k, m, 1)[0])


def test_gaussian_entries_close(rs):
    m, tau = 200, 16
    X, y, _ = gaussian_problem(m + 1, m, 7)
    with rs.Solver(X, y, 1.0, sketch="gaussian", tau=tau, seed=8) as s:
        for k in [0, 4]:
            S = s.dump_gaussian(k)
            ref = oracle.sketch_matrix("gaussian", m, tau, 8, k)
            assert np.max(np.abs(S - ref)) <= 1e-13 * np.max(np.abs(ref))


# ------------------------------------------------------- plain FP64 iterates ---
KINDS = [("subsample", 12, None), ("count", 12, None), ("subcount", 8, 48),
         ("gaussian", 6, None), ("srht", 10, None)]
MOMS = ["none", "const", "theory", "heuristic"]


@pytest.mark.parametrize("kind,tau,s_", KINDS, ids=[k[0] for k in KINDS])
@pytest.mark.parametrize("mom", MOMS)
def test_plain_iterates_match_oracle(rs, kind, tau, s_, mom):
    X, y, _ = gaussian_problem(160, 97, 21)  # m = 97: ragged against every tile size
    lam, K = 0.05, 60
    ref = oracle.solve_ridge(X, y, lam, "primal", kind, tau, seed=9, tol=0.0, max_iters=K,
                             mom={"kind": mom}, s=s_)
    with rs.Solver(X, y, lam, sketch=kind, tau=tau, momentum=mom, seed=9, sub_s=s_ or 0) as s:
        w, hist, iters, _ = s.solve(tol=0.0, max_iters=K)
    assert iters == K
    assert rel(w, ref["w"]) <= W_TOL
    assert np.allclose(hist, ref["hist"], rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("kind,tau,s_", KINDS[:3], ids=[k[0] for k in KINDS[:3]])
def test_plain_iterates_one_cluster_of_ctas(rs, kind, tau, s_):
    """The persistent iteration kernel as one cluster of 16 CTAs of 8 rows (the last
    three CTAs idle) against the oracle."""
    X, y, _ = gaussian_problem(160, 97, 21)
    lam, K = 0.05, 40
    ref = oracle.solve_ridge(X, y, lam, "primal", kind, tau, seed=9, tol=0.0, max_iters=K,
                             mom={"kind": "heuristic"}, s=s_)
    with rs.Solver(X, y, lam, sketch=kind, tau=tau, momentum="heuristic", seed=9,
                   sub_s=s_ or 0, iter_ctas=16) as s:
        assert (s.iter_ctas, s.iter_rows) == (16, 8)
        w, hist, iters, _ = s.solve(tol=0.0, max_iters=K)
    assert iters == K
    assert rel(w, ref["w"]) <= W_TOL
    assert np.allclose(hist, ref["hist"], rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("kind,tau,s_", [("subsample", 64, 0), ("count", 64, 0),
                                         ("subcount", 64, 640)], ids=["subsample", "count", "subcount"])
def test_persistent_kernel_matches_cluster_kernel(rs, kind, tau, s_):
    """Plain FP64 iterates of the two iteration kernels (CTAs spread over the GPU vs
    one cluster) agree to rounding; m = 1999 is ragged against the 4-row slices;
    chunk 128 with 300 iterations spans several launches."""
    X, y, _ = gaussian_problem(2600, 1999, 31)
    lam, K = 0.1, 300
    out = []
    for ctas in (0, -1):
        with rs.Solver(X, y, lam, sketch=kind, tau=tau, momentum="heuristic", seed=5,
                       sub_s=s_, iter_ctas=ctas) as s:
            assert (s.iter_ctas > 0) == (ctas == 0)
            w, hist, iters, _ = s.solve(tol=0.0, max_iters=K)
            out.append((w, hist))
    assert rel(out[0][0], out[1][0]) <= 1e-10
    assert np.allclose(out[0][1], out[1][1], rtol=1e-9, atol=0)


def test_cfg_small_to_tolerance(rs):
    """Dense primal FP64: X 2000 x 500 iid N(0,1), lambda = 1e-3, subsample tau = 50,
    no momentum, seed 0, relative residual 1e-6."""
    X, y, _ = gaussian_problem(2000, 500, 0)
    lam = 1e-3
    ref = oracle.solve_ridge(X, y, lam, "primal", "subsample", 50, seed=0, tol=1e-6,
                             max_iters=20000)
    with rs.Solver(X, y, lam, sketch="subsample", tau=50, seed=0) as s:
        w, hist, iters, conv = s.solve(tol=1e-6, max_iters=20000)
    assert conv and iters == ref["iters"]
    assert rel(w, ref["w"]) <= W_TOL
    assert oracle.true_residual(X, y, lam, w) <= 1.01e-6
    assert rel(w, oracle.direct_solution(X, y, lam)) <= 1e-4


def test_plain_chunking_and_forecast_leave_iterates_unchanged(rs):
    """Plain FP64 persistent path (count sketch, heuristic momentum) to tolerance in
    chunks of 50, 128 and the default: each chunk's start sets a convergence forecast
    that can end the chunk early, but the sketches are drawn by iteration index and
    the state carries over in FP64, so every chunking stops at the oracle's iteration
    with the same w."""
    X, y, _ = gaussian_problem(3000, 700, 1)
    lam = 1e-2
    ref = oracle.solve_ridge(X, y, lam, "primal", "count", 64, seed=3, tol=1e-6, max_iters=5000,
                             mom={"kind": "heuristic"})
    ws = []
    for ch in (50, 128, 0):
        with rs.Solver(X, y, lam, sketch="count", tau=64, momentum="heuristic", seed=3,
                       chunk=ch) as s:
            w, hist, iters, conv = s.solve(tol=1e-6, max_iters=5000)
        assert conv and iters == ref["iters"], (ch, iters, ref["iters"])
        assert rel(w, ref["w"]) <= W_TOL
        ws.append(w)
    for w in ws[1:]:
        assert rel(w, ws[0]) <= 1e-13


@pytest.mark.parametrize("kind", ["subsample", "count", "subcount", "gaussian", "srht"])
def test_probe_sketched_system(rs, kind):
    """M = S^T A S, r_S = S^T r and delta of one iteration, from the oracle's state."""
    X, y, _ = gaussian_problem(150, 70, 31)
    lam, tau = 0.3, 9
    s_ = 27 if kind == "subcount" else None
    ref = oracle.solve_ridge(X, y, lam, "primal", kind, tau, seed=2, tol=0.0, max_iters=6,
                             mom={"kind": "heuristic"}, s=s_, record_first=6)
    with rs.Solver(X, y, lam, sketch=kind, tau=tau, momentum="heuristic", seed=2,
                   sub_s=s_ or 0) as s:
        A, b = oracle.form_system(X, y, lam)
        w_prev = np.zeros(70)
        w = np.zeros(70)
        for k in range(5):
            r = A @ w - b
            r_prev = A @ w_prev - b
            s.set_state(w, w_prev, r, r_prev, k)
            M, rS, delta = s.probe_step()
            rec = ref["records"][k]
            assert np.allclose(M, rec["M"], rtol=1e-12, atol=1e-12 * np.abs(rec["M"]).max())
            assert np.allclose(rS, rec["rS"], rtol=1e-12, atol=1e-12 * np.abs(rec["rS"]).max())
            assert rel(rec["S"] @ delta, rec["S"] @ rec["delta"]) <= 1e-10
            w_prev, w = w, rec["w"]


def test_step_matches_oracle_history(rs):
    X, y, _ = gaussian_problem(300, 130, 41)
    lam = 0.1
    ref = oracle.solve_ridge(X, y, lam, "primal", "count", 13, seed=1, tol=0.0, max_iters=30,
                             mom={"kind": "heuristic"})
    with rs.Solver(X, y, lam, sketch="count", tau=13, momentum="heuristic", seed=1) as s:
        m = 130
        A, b = oracle.form_system(X, y, lam)
        s.set_state(np.zeros(m), np.zeros(m), -b, -b, 0)
        h = s.step(30)
        w, _, _, _, k = s.get_state()
    assert k == 30
    assert np.allclose(h, ref["hist"][1:], rtol=1e-9)
    assert rel(w, ref["w"]) <= W_TOL


def test_dual_form(rs):
    X, y, _ = gaussian_problem(60, 150, 51)  # n < d: the dual is the smaller system
    lam = 0.5
    ref = oracle.solve_ridge(X, y, lam, "dual", "count", 8, seed=3, tol=0.0, max_iters=50,
                             mom={"kind": "heuristic"})
    with rs.Solver(X, y, lam, form="dual", sketch="count", tau=8, momentum="heuristic", seed=3) as s:
        assert s.m == 60
        w, hist, iters, _ = s.solve(tol=0.0, max_iters=50)
    assert rel(w, ref["w"]) <= W_TOL
    with rs.Solver(X, y, lam, form="dual", sketch="subsample", tau=20, momentum="heuristic",
                   seed=3) as s:
        w, hist, iters, conv = s.solve(tol=1e-10, max_iters=20000)
    assert conv and rel(w, oracle.direct_solution(X, y, lam)) <= 1e-8


# ------------------------------------------------------------- edge cases ---
def test_subsample_tau_equals_m_one_step(rs):
    X, y, _ = gaussian_problem(90, 40, 61)
    lam = 0.2
    with rs.Solver(X, y, lam, sketch="subsample", tau=40, seed=0) as s:
        w, hist, iters, conv = s.solve(tol=1e-12, max_iters=5)
    assert iters == 1 and conv
    assert rel(w, oracle.direct_solution(X, y, lam)) <= 1e-11


def test_tau_one_and_empty_buckets(rs):
    X, y, _ = gaussian_problem(80, 33, 62)
    lam = 0.4
    for kind, tau in [("subsample", 1), ("count", 1), ("count", 30)]:
        ref = oracle.solve_ridge(X, y, lam, "primal", kind, tau, seed=4, tol=0.0, max_iters=40)
        with rs.Solver(X, y, lam, sketch=kind, tau=tau, seed=4) as s:
            w, _, _, _ = s.solve(tol=0.0, max_iters=40)
        assert rel(w, ref["w"]) <= W_TOL, (kind, tau)


def test_zero_rhs_returns_zero(rs):
    X, _, _ = gaussian_problem(50, 20, 63)
    with rs.Solver(X, np.zeros(50), 1.0, sketch="count", tau=4) as s:
        w, hist, iters, conv = s.solve(tol=1e-6, max_iters=10)
    assert iters == 0 and conv and np.all(w == 0)


def test_invalid_sizes_rejected(rs):
    X, y, _ = gaussian_problem(30, 10, 64)
    with pytest.raises(rs.RSError):
        rs.Solver(X, y, 1.0, sketch="subsample", tau=11)
    with pytest.raises(rs.RSError):
        rs.Solver(X, y, 1.0, sketch="subcount", tau=3, sub_s=7)
    with pytest.raises(rs.RSError):
        rs.Solver(X, y, 0.0, sketch="count", tau=3)


def test_max_iters_reports_not_converged(rs):
    X, y, _ = gaussian_problem(200, 60, 65)
    with rs.Solver(X, y, 1e-3, sketch="count", tau=4, seed=1) as s:
        w, hist, iters, conv = s.solve(tol=1e-12, max_iters=7)
    assert iters == 7 and not conv and hist.shape == (8,)


# ------------------------------------------------------------ mixed path ---
@pytest.mark.parametrize("kind", ["count", "subsample", "subcount"])
def test_mixed_reaches_tolerance(rs, kind):
    from synth import geometric_sigma, spectrum_problem

    X, y, _ = spectrum_problem(3000, 256, geometric_sigma(256), seed=7, noise=0.01, dtype=np.float32)
    lam = 1e-2
    with rs.Solver(X, y, lam, sketch=kind, tau=32, momentum="heuristic", seed=2,
                   precision="mixed") as s:
        w, hist, iters, conv = s.solve(tol=1e-6, max_iters=50000)
    Xd = X.astype(np.float64)
    assert conv
    assert oracle.true_residual(Xd, y, lam, w) <= 1e-6
    w_star = oracle.direct_solution(Xd, y, lam)
    assert rel(w, w_star) <= 1e-4


@pytest.mark.parametrize("kind,tau,s_", [("count", 32, 0), ("subsample", 32, 0),
                                         ("subcount", 32, 160)], ids=["count", "subsample", "subcount"])
def test_mixed_iterates_close_to_oracle(rs, kind, tau, s_):
    """Mixed path (FP32 A formed on the CUDA cores, S^T A and M^+ by FP32 sweeps;
    FP64 vectors) against the FP64 oracle on the same FP32 data for 12 iterations:
    the difference is FP32 rounding of the products."""
    from synth import geometric_sigma, spectrum_problem

    X, y, _ = spectrum_problem(1500, 256, geometric_sigma(256, 1e-1), seed=8, noise=0.01,
                               dtype=np.float32)
    lam, K = 1e-1, 12
    Xd = X.astype(np.float64)
    ref = oracle.solve_ridge(Xd, y, lam, "primal", kind, tau, seed=6, tol=0.0, max_iters=K,
                             mom={"kind": "heuristic"}, s=s_)
    with rs.Solver(X, y, lam, sketch=kind, tau=tau, momentum="heuristic", seed=6, sub_s=s_,
                   precision="mixed", setup_tc=False) as s:
        assert s.iter_ctas > 0
        w, hist, iters, _ = s.solve(tol=0.0, max_iters=K)
    assert iters == K
    assert rel(w, ref["w"]) <= 2e-5
    assert np.allclose(hist[:K], ref["hist"][:K], rtol=2e-5, atol=0)


def test_mixed_sweep_empty_buckets(rs):
    """Count sketch with tau close to m: empty buckets make S^T A S singular; the
    sweep drops those indices and the solve still reaches the FP64-checked tolerance."""
    from synth import geometric_sigma, spectrum_problem

    X, y, _ = spectrum_problem(1200, 256, geometric_sigma(256, 1e-2), seed=3, noise=0.01,
                               dtype=np.float32)
    lam = 1e-2
    with rs.Solver(X, y, lam, sketch="count", tau=230, momentum="none", seed=1,
                   precision="mixed") as s:
        w, hist, iters, conv = s.solve(tol=1e-6, max_iters=5000)
    Xd = X.astype(np.float64)
    assert conv and oracle.true_residual(Xd, y, lam, w) <= 1e-6
    assert rel(w, oracle.direct_solution(Xd, y, lam)) <= 1e-4


# ------------------------------------------------------- small SPD solve ---
@pytest.mark.parametrize("tau", [1, 5, 16, 17, 33, 100, 256, 300, 512])
def test_cholesky_solve_sizes(rs, tau):
    """delta of the sketched system against a LAPACK solve of the same M, r_S
    (covers the single-CTA and cluster factorisations, padding and several row
    blocks per CTA)."""
    m = 700
    X, y, _ = gaussian_problem(900, m, 71)
    with rs.Solver(X, y, 0.5, sketch="subsample", tau=tau, seed=3) as s:
        M, rS, delta = s.probe_step()
    ref = np.linalg.solve(M, rS)
    assert rel(delta, ref) <= 1e-10


@pytest.mark.parametrize("tau", [7, 64, 256, 512])
def test_cholesky_fp32_factor(rs, tau):
    """Mixed path with the FP32 factorisation of S^T A S."""
    m = 700
    X, y, _ = gaussian_problem(900, m, 72)
    with rs.Solver(X.astype(np.float32), y, 0.5, sketch="subsample", tau=tau, seed=3,
                   precision="mixed", chol_fp64=False) as s:
        M, rS, delta = s.probe_step()
    ref = np.linalg.solve(M, rS)
    assert rel(delta, ref) <= 1e-4


@pytest.mark.parametrize("tau", [7, 64, 256])
def test_cholesky_fp64_factor_mixed(rs, tau):
    """Mixed path with the FP64 factorisation of S^T A S (the default): delta solves
    the sketched system of the FP32 A to FP64 accuracy."""
    m = 700
    X, y, _ = gaussian_problem(900, m, 73)
    with rs.Solver(X.astype(np.float32), y, 0.5, sketch="subsample", tau=tau, seed=3,
                   precision="mixed") as s:
        M, rS, delta = s.probe_step()
    ref = np.linalg.solve(M, rS)
    assert rel(delta, ref) <= 1e-10


def test_mixed_fp32_factor_reaches_tolerance(rs):
    from synth import geometric_sigma, spectrum_problem

    X, y, _ = spectrum_problem(3000, 256, geometric_sigma(256), seed=7, noise=0.01, dtype=np.float32)
    lam = 1e-2
    with rs.Solver(X, y, lam, sketch="count", tau=32, momentum="heuristic", seed=2,
                   precision="mixed", chol_fp64=False) as s:
        w, hist, iters, conv = s.solve(tol=1e-6, max_iters=50000)
    assert conv and oracle.true_residual(X.astype(np.float64), y, lam, w) <= 1e-6


@pytest.mark.parametrize("f64", [True, False])
@pytest.mark.parametrize("kind", ["count", "subsample", "gaussian", "subcount"])
def test_mixed_fp64_factor_and_kinds(rs, kind, f64):
    """Mixed path with the FP64 factor of S^T A S (the default) and with the FP32
    factor, every dense sketch kind, to the FP64-checked tolerance."""
    from synth import geometric_sigma, spectrum_problem

    X, y, _ = spectrum_problem(2000, 192, geometric_sigma(192), seed=9, noise=0.01, dtype=np.float32)
    lam = 1e-2
    with rs.Solver(X, y, lam, sketch=kind, tau=24, momentum="heuristic", seed=4,
                   precision="mixed", chol_fp64=f64) as s:
        w, hist, iters, conv = s.solve(tol=1e-6, max_iters=50000)
    assert conv and oracle.true_residual(X.astype(np.float64), y, lam, w) <= 1e-6


@pytest.mark.parametrize("d", [700, 2048, 4096])
def test_true_residual_fp32_x(rs, d):
    """A v - b through FP32 X in one pass with float pairs vs the FP64 oracle."""
    n = 3000
    g = np.random.default_rng(d)
    X = g.standard_normal((n, d)).astype(np.float32)
    y = g.standard_normal(n)
    lam = 0.3
    v = g.standard_normal(d)
    with rs.Solver(X, y, lam, sketch="count", tau=16, seed=1, precision="mixed") as s:
        got = s.true_residual(v)
    ref = oracle.true_residual(X.astype(np.float64), y, lam, v)
    assert abs(got - ref) <= 1e-12 * ref
    # near a solution the residual is a small difference of large terms
    w_star = oracle.direct_solution(X.astype(np.float64), y, lam)
    w_near = w_star * (1.0 + 1e-7 * g.standard_normal(d))
    with rs.Solver(X, y, lam, sketch="count", tau=16, seed=1, precision="mixed") as s:
        got = s.true_residual(w_near)
    ref = oracle.true_residual(X.astype(np.float64), y, lam, w_near)
    assert abs(got - ref) <= 1e-6 * ref


@pytest.mark.parametrize("n,d", [(2000, 300), (1000, 256), (5000, 130), (1001, 500)])
def test_gram_tensor_cores(rs, n, d):
    """X^T X + lambda I formed by the tensor-core kernel (TF32 inputs, FP32
    accumulation): M = S^T A S with S = I_C, tau = m, equals the FP64 A[C, C] within
    the TF32 rounding of both inputs, and the CUDA-core path within FP32 rounding."""
    g = np.random.default_rng(n + d)
    X = g.standard_normal((n, d)).astype(np.float32)
    y = g.standard_normal(n)
    lam = 0.7
    C = orng.subsample_indices(5, 0, d, d)
    A64, _ = oracle.form_system(X.astype(np.float64), y, lam)
    ref = A64[np.ix_(C, C)]
    bound = 2.0 ** -9 * (np.abs(X.astype(np.float64)).T @ np.abs(X.astype(np.float64)))[np.ix_(C, C)]
    for tc in (True, False):
        with rs.Solver(X, y, lam, sketch="subsample", tau=d, seed=5, precision="mixed",
                       setup_tc=tc) as s:
            M, _, _ = s.probe_step()
        assert np.all(np.abs(M - ref) <= bound + 1e-6), tc
        assert np.allclose(M, M.T, rtol=0, atol=0)


def test_mixed_refresh_beyond_4096_columns(rs):
    """d = 4500 (past the one-pass refresh kernel): the FP64 true residual through X in
    two passes equals the oracle's, and the mixed solve reaches 1e-6 by it."""
    from synth import geometric_sigma, spectrum_problem

    X, y, _ = spectrum_problem(5000, 4500, geometric_sigma(4500, 1e-1), 44, noise=0.01)
    X = X.astype(np.float32)
    X64 = X.astype(np.float64)
    lam = 1e-1
    with rs.Solver(X, y, lam, sketch="count", tau=256, momentum="heuristic", seed=2,
                   precision="mixed") as s:
        w, hist, iters, conv = s.solve(tol=1e-6, max_iters=20000)
        assert conv
        got = s.true_residual(w)
    ref = oracle.true_residual(X64, y, lam, w)
    # float-pair products carry about 48 bits: the residual relative to ||b|| to ~1e-14
    assert abs(got - ref) <= 1e-12
    assert ref <= 1e-6 * (1 + 1e-6)


def test_pool_reuse_across_contexts(rs):
    """Contexts created and destroyed back to back on one stream reuse the blocks of
    the library's memory pool: every repetition gives bit-identical iterates (the
    solves are deterministic), and the pool's unused memory can be trimmed."""
    from synth import geometric_sigma, spectrum_problem

    X, y, _ = spectrum_problem(2000, 300, geometric_sigma(300, 1e-1), seed=21, noise=0.01,
                               dtype=np.float32)
    first = {}
    for rep in range(3):
        for sketch, tau, prec in (("count", 32, "mixed"), ("subsample", 48, "fp64"),
                                  ("count", 64, "mixed")):
            with rs.Solver(X, y, 0.1, sketch=sketch, tau=tau, momentum="heuristic", seed=3,
                           precision=prec) as s:
                w, hist, iters, conv = s.solve(tol=1e-8, max_iters=400)
            key = (sketch, tau, prec)
            if rep == 0:
                first[key] = (w.copy(), np.array(hist).copy(), iters)
            else:
                w0, h0, i0 = first[key]
                assert iters == i0 and np.array_equal(w, w0) and np.array_equal(hist, h0), key
        if rep == 1:
            rs.trim_memory(0)


@pytest.mark.parametrize("m,tau,kind", [(301, 16, "count"), (1000, 64, "count"),
                                        (1000, 64, "subcount")])
def test_mixed_sketched_system_matches_fp64(rs, m, tau, kind):
    """Mixed path (FP32 A on the CUDA cores, S^T A and M = S^T A S in FP32 sums, m not
    a multiple of 4): M equals the plain FP64 path's M of the same draw within FP32
    rounding."""
    g = np.random.default_rng(m + tau)
    X = g.standard_normal((3 * m, m)).astype(np.float32)
    y = g.standard_normal(3 * m)
    with rs.Solver(X, y, 0.3, sketch=kind, tau=tau, seed=11, precision="mixed",
                   setup_tc=False) as s:
        M32, _, _ = s.probe_step()
    with rs.Solver(X, y, 0.3, sketch=kind, tau=tau, seed=11, precision="fp64") as s:
        M64, _, _ = s.probe_step()
    assert np.linalg.norm(M32 - M64) <= 1e-5 * np.linalg.norm(M64)


def test_host_upload_in_pieces_matches_device_input(rs):
    """FP32 X in host memory with n >= 16384: X is uploaded in four row ranges, each
    range's part of X^T X (tensor cores, added into A) and of X^T y formed after its
    copy. The system equals the one formed from the same X already on the device:
    b to the bit (the same 512-row blocks summed in the same order), M = A[C, C] (S
    the sample of all d columns) within the TF32 bound of the tensor-core Gram for both
    (the range sums change only the FP32 rounding of the accumulation), and the mixed
    solve reaches the FP64-checked tolerance."""
    import torch

    n, d = 40000 + 77, 256
    g = np.random.default_rng(5)
    X = g.standard_normal((n, d)).astype(np.float32)
    y = g.standard_normal(n)
    v = g.standard_normal(d)
    Xd = torch.from_numpy(X).cuda()
    out = {}
    for name, Xin in (("host", X), ("device", Xd)):
        with rs.Solver(Xin, y, 0.5, sketch="subsample", tau=d, seed=2, precision="mixed") as s:
            M, _, _ = s.probe_step()
            rel = s.true_residual(v)
            w, hist, iters, conv = s.solve(tol=1e-8, max_iters=20000)
        out[name] = (M, rel, w, conv)
    Mh, rh, wh, ch = out["host"]
    Md, rd, wd, cd = out["device"]
    assert rh == rd
    C = orng.subsample_indices(2, 0, d, d)
    X64 = X.astype(np.float64)
    ref = (X64.T @ X64 + 0.5 * np.eye(d))[np.ix_(C, C)]
    bound = 2.0 ** -9 * (np.abs(X64).T @ np.abs(X64))[np.ix_(C, C)]
    for M in (Mh, Md):
        assert np.all(np.abs(M - ref) <= bound + 1e-6)
    assert ch and cd
    assert oracle.true_residual(X.astype(np.float64), y, 0.5, wh) <= 1e-8


@pytest.mark.parametrize("refresh", [16, 48])
def test_mixed_chunk_forecast_reaches_tolerance(rs, refresh):
    """Mixed persistent path with short refresh periods, so that the convergence
    forecast sets the end of many chunks (some forecasts fall short and cost one more
    refresh): the solve still stops only on an FP64-checked residual below tol, with
    the weights of the FP64 direct solution."""
    from synth import geometric_sigma, spectrum_problem

    X, y, _ = spectrum_problem(4000, 384, geometric_sigma(384, 1e-2), seed=17, noise=0.01,
                               dtype=np.float32)
    lam = 1e-3
    with rs.Solver(X, y, lam, sketch="count", tau=32, momentum="heuristic", seed=5,
                   precision="mixed", refresh_every=refresh) as s:
        assert s.iter_ctas > 0
        w, hist, iters, conv = s.solve(tol=1e-7, max_iters=100000)
    Xd = X.astype(np.float64)
    assert conv and hist[iters] <= 1e-7
    assert oracle.true_residual(Xd, y, lam, w) <= 1e-7
    assert rel(w, oracle.direct_solution(Xd, y, lam)) <= 1e-4


def test_gaussian_sketched_system_on_tensor_cores(rs):
    """Mixed Gaussian sketch: S^T A of the chunk's slots is one TF32 tensor-core product
    (and A the TF32 Gram), then M = S^T A S. Against S^T (X^T X + lambda I) S in FP64
    from the library's own S: each TF32 product perturbs a term by at most 2^-10 of
    its magnitude, so |dM| <= 4 * 2^-10 |S|^T (|X|^T |X| + lambda I) |S| (two
    products, FP32 sums), checked with that bound."""
    n, m, tau, lam = 700, 300, 24, 0.5
    X, y, _ = gaussian_problem(n, m, 74)
    X32 = X.astype(np.float32)
    with rs.Solver(X32, y, lam, sketch="gaussian", tau=tau, seed=3, precision="mixed",
                   chol_fp64=False) as s:
        S = s.dump_gaussian(0)
        M, rS, delta = s.probe_step()
    Xf = X32.astype(np.float64)
    A = Xf.T @ Xf + lam * np.eye(m)
    M_ref = S.T @ A @ S
    Aabs = np.abs(Xf).T @ np.abs(Xf) + lam * np.eye(m)
    bound = 4 * 2.0 ** -10 * (np.abs(S).T @ Aabs @ np.abs(S))
    assert np.all(np.abs(M - M_ref) <= bound)
    assert np.abs(M - M_ref).max() > 0  # the tensor-core path ran (not an FP64 product)


@pytest.mark.parametrize("m,prec,kind", [(8192, "fp64", "count"), (8192, "mixed", "count"),
                                         (4100, "fp64", "subcount"), (6000, "mixed", "subsample")])
def test_sketched_system_large_and_ragged_m(rs, m, prec, kind):
    """S^T A and M = S^T A S of the bucket-row sketches where A exceeds L2 (m = 8192 in
    FP64 and FP32, m = 6000 in FP32) or m is ragged (4100 in FP64): M of slot 0 against
    S^T (X^T X + lambda I) S in FP64 from X S."""
    n, tau, lam = 48, 256, 0.3
    g = np.random.default_rng(m)
    X = g.standard_normal((n, m))
    y = g.standard_normal(n)
    s_ = 1024 if kind == "subcount" else None
    Xin = X.astype(np.float32) if prec == "mixed" else X
    kw = {"sub_s": s_} if s_ else {}
    with rs.Solver(Xin, y, lam, sketch=kind, tau=tau, seed=5, precision=prec, setup_tc=False,
                   **kw) as s:
        M, _, _ = s.probe_step()
    Xr = Xin.astype(np.float64)
    S = oracle.sketch_matrix(kind, m, tau, 5, 0, s=s_)
    XS = Xr @ S
    ref = XS.T @ XS + lam * (S.T @ S)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.linalg.norm(M - ref) <= tol * np.linalg.norm(ref)


def test_inputs_produced_on_the_default_stream_just_before(rs):
    """Device inputs that torch is still writing on its default stream when the context
    is made (no synchronize between): the library's own stream orders after that work,
    so the setup reads complete inputs and the solve equals the one from inputs that
    were complete."""
    torch = pytest.importorskip("torch")
    n, m = 32768, 2048
    gen = torch.Generator(device="cuda").manual_seed(3)
    Xf = torch.randn(n, m, device="cuda", generator=gen)
    y = torch.randn(n, device="cuda", dtype=torch.float64, generator=gen)
    torch.cuda.synchronize()

    def make():  # several kernels on torch's stream, the last one writing X
        return ((Xf.double() * 2.0 + 1.0) - 1.0) * 0.5

    Xd = make()
    torch.cuda.synchronize()
    with rs.Solver(Xd, y, 0.1, sketch="subsample", tau=64, seed=2) as s:
        w_ref, h_ref, _, _ = s.solve(tol=0.0, max_iters=10)
    w_ref = np.asarray(w_ref)
    for _ in range(3):
        Xd = make()
        with rs.Solver(Xd, y, 0.1, sketch="subsample", tau=64, seed=2) as s:
            w, h, _, _ = s.solve(tol=0.0, max_iters=10)
        assert np.array_equal(np.asarray(h), np.asarray(h_ref))
        assert np.array_equal(np.asarray(w), w_ref)
