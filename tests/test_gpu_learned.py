"""Learned sketch proposal through the C ABI against the oracle: the network's
scores, gradient and Adam steps (bfloat16 tolerance), the standardised features,
the Gumbel-top-tau draws (the same rows, or rows whose keys tie to within
rounding), the plain FP64 iterates of the first chunks (1e-8), and the gain of a
network trained with the library's kernels over uniform draws on held-out
problems."""
import numpy as np
import pytest

import oracle
from oracle import learned as OL
from synth import mlp_init, power_sigma, spectrum_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import paper_2105_05565_gb300 as rs

    rs.lib()
    return rs


def bf16_bits(theta):
    f = np.ascontiguousarray(theta, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)


def problem(m, n, seed, lam=1e-3):
    X, y, _ = spectrum_problem(n, m, power_sigma(m, 0.8), seed, noise=0.01)
    X = X.astype(np.float64)
    A, b = oracle.form_system(X, y, lam, "primal")
    return X, y, A, b, lam


def test_network_scores_match_oracle(rs):
    theta = mlp_init(1).astype(np.float32)
    Z = np.random.default_rng(0).standard_normal((1000, 4)).astype(np.float32)
    with rs.MLP(theta) as net:
        s = net.scores(Z)
    ref = OL.forward(theta.astype(np.float64), Z, bf16_mode=True)
    assert np.all(np.abs(s - ref) <= 1e-2 * (1 + np.abs(ref)))
    assert np.median(np.abs(s - ref)) <= 1e-4 * (1 + np.abs(ref).max())


def test_network_gradient_and_adam_match_oracle(rs):
    theta = mlp_init(2).astype(np.float32)
    rng = np.random.default_rng(1)
    Z = rng.standard_normal((700, 4)).astype(np.float32)  # ragged against 128-row blocks
    y = rng.standard_normal(700).astype(np.float32)
    with rs.MLP(theta) as net:
        loss, g = net.grad(Z, y)
        l0, g0 = OL.loss_grad(theta.astype(np.float64), Z, y, bf16_mode=True)
        assert abs(loss - l0) <= 1e-3 * l0
        assert np.linalg.norm(g - g0) <= 2e-2 * np.linalg.norm(g0)
        for blk, ref in zip(OL.unpack(g), OL.unpack(g0)):
            assert np.linalg.norm(np.ravel(blk) - np.ravel(ref)) <= 5e-2 * np.linalg.norm(np.ravel(ref)) + 1e-7
        net.step(Z, y, lr=1e-2)
        net.step(Z, y, lr=1e-2)
        th = net.params()
    st = {}
    t = theta.astype(np.float64)
    for _ in range(2):
        _, gg = OL.loss_grad(t, Z, y, bf16_mode=True)
        t = OL.adam_step(t, gg, st, lr=1e-2)
    # Adam moves every weight by about lr per step; both sides agree to well below that
    assert np.abs(th - t).max() <= 2e-3


def test_features_and_first_draws_match_oracle(rs):
    m, n, tau, seed, eps = 256, 1024, 16, 5, 0.1
    X, y, A, b, lam = problem(m, n, 31)
    theta = mlp_init(3)
    wb = bf16_bits(theta)
    with rs.Solver(X, y, lam, sketch="subsample", tau=tau, momentum="none", seed=seed,
                   chunk=8) as s:
        s.set_proposal(wb, eps)
        s.set_state(np.zeros(m), np.zeros(m), -b, -b, 0)
        Z = s.proposal_features()
        C = [s.dump_sketch(k)[0][:tau].copy() for k in range(3)]
    static = OL.static_features(A)
    Zr = OL.features(static, -b, np.ones(m))
    assert np.abs(Z - Zr).max() <= 1e-4
    th16 = OL.bf16(theta)
    logp = OL.log_proposal(OL.forward(th16, Zr, bf16_mode=True), eps)
    for k in range(3):
        Cr, keys = OL.select(logp, seed, k, tau)
        assert np.all(np.diff(C[k]) > 0)
        diff = set(C[k].tolist()) ^ set(Cr.tolist())
        kth = np.sort(keys)[::-1][tau - 1]
        for j in diff:  # only rows whose keys tie with the boundary within rounding
            assert abs(keys[j] - kth) <= 1e-3 * (1 + abs(kth)), (k, j)


@pytest.mark.parametrize("chunk", [1, 8])
def test_learned_plain_iterates_match_oracle(rs, chunk):
    m, n, tau, seed, eps = 200, 800, 12, 9, 0.2
    X, y, A, b, lam = problem(m, n, 32)
    theta = mlp_init(4)
    K = 3 * chunk + 2
    ref = OL.solve_learned(A, b, OL.bf16(theta), tau, seed, tol=0.0, max_iters=K, eps=eps,
                           chunk=chunk, bf16_mode=True)
    with rs.Solver(X, y, lam, sketch="subsample", tau=tau, momentum="none", seed=seed,
                   chunk=chunk) as s:
        s.set_proposal(bf16_bits(theta), eps)
        w, hist, iters, _ = s.solve(tol=0.0, max_iters=K)
    assert iters == K
    assert np.linalg.norm(w - ref["w"]) <= 1e-8 * np.linalg.norm(ref["w"])
    assert np.allclose(hist, ref["hist"], rtol=1e-8, atol=1e-14)


def test_learned_solve_converges_to_the_closed_form(rs):
    m, n, tau = 128, 512, 8
    X, y, A, b, lam = problem(m, n, 33, lam=1e-2)
    w_star = np.linalg.solve(A, b)
    with rs.Solver(X, y, lam, sketch="subsample", tau=tau, momentum="none", seed=1,
                   chunk=4) as s:
        s.set_proposal(bf16_bits(mlp_init(5)), 0.5)
        w, hist, iters, conv = s.solve(tol=1e-10, max_iters=200000)
    assert conv
    assert np.linalg.norm(w - w_star) <= 1e-7 * np.linalg.norm(w_star) * np.linalg.cond(A) ** 0.5


def test_trained_proposal_beats_uniform_on_held_out_problems(rs):
    """Trajectories of the uniform proposal on 4 training problems (m = 256,
    X = U diag(i^-0.8) V^T), a network trained on them with the library's Adam
    kernels, then iterations to 1e-6 on 3 held-out problems: learned against
    uniform, both through the library."""
    from paper_2105_05565_gb300 import learned

    m, n, tau, ch = 256, 1024, 16, 1
    Zs, Ys = [], []
    for sd in range(4):
        X, y, A, b, lam = problem(m, n, 100 + sd)
        w_star = np.linalg.solve(A, b)
        with rs.Solver(X, y, lam, sketch="subsample", tau=tau, momentum="none", seed=sd,
                       chunk=ch) as s:
            s.set_proposal(None, 0.1)
            s.set_state(np.zeros(m), np.zeros(m), -b, -b, 0)
            Z, t = learned.collect(s, w_star, 3000, tol=1e-6)
        Zs.append(Z)
        Ys.append(t)
    wb, _, losses = learned.train(np.concatenate(Zs), np.concatenate(Ys), steps=2500, batch=512,
                                  lr=3e-3, seed=0)
    assert losses[-200:].mean() < losses[:50].mean()
    its_u, its_l = [], []
    for sd in range(3):
        X, y, A, b, lam = problem(m, n, 900 + sd)
        for w8, out in ((None, its_u), (wb, its_l)):
            with rs.Solver(X, y, lam, sketch="subsample", tau=tau, momentum="none",
                           seed=50 + sd, chunk=ch) as s:
                s.set_proposal(w8, 0.1)
                w, hist, iters, conv = s.solve(tol=1e-6, max_iters=20000)
                assert conv
                out.append(iters)
            assert oracle.true_residual(X, y, lam, w) <= 1.01e-6
    assert np.mean(its_l) <= 0.85 * np.mean(its_u), (its_l, its_u)


def test_collected_training_pairs_match_oracle(rs):
    """rs_collect (features and targets formed on the device along the trajectory)
    against the oracle's collected pairs on the same seeded problem, network and
    draws: features within 1e-4, targets (1/2) ln(m a / e + 1e-3) within FP32
    rounding of the FP64 values."""
    m, n, tau, seed, eps, K = 96, 400, 6, 3, 0.2, 25
    X, y, A, b, lam = problem(m, n, 41)
    theta = mlp_init(5)
    w_star = np.linalg.solve(A, b)
    with rs.Solver(X, y, lam, sketch="subsample", tau=tau, momentum="none", seed=seed,
                   chunk=1) as s:
        s.set_proposal(bf16_bits(theta), eps)
        s.set_state(np.zeros(m), np.zeros(m), -b, -b, 0)
        Z, t = s.collect(w_star, K, tol=1e-12)
    ref = OL.solve_learned(A, b, OL.bf16(theta), tau, seed, tol=0.0, max_iters=K, eps=eps,
                           chunk=1, bf16_mode=True, w_star=w_star, collect=True)
    Zr, tr = ref["data"]
    assert Z.shape == (K * tau, 4) and t.shape == (K * tau,)
    assert np.abs(Z - Zr).max() <= 1e-4
    assert np.all(np.abs(t - tr) <= 1e-5 * (1 + np.abs(tr)))


def test_collect_needs_its_setting(rs):
    X, y, A, b, lam = problem(64, 256, 42)
    with rs.Solver(X, y, lam, sketch="subsample", tau=4, momentum="heuristic", chunk=1) as s:
        s.set_proposal(None, 0.1)
        with pytest.raises(rs.RSError) as e:
            s.collect(np.zeros(64), 10)
        assert e.value.status == rs.RS_EINVAL
