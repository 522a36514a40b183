"""Hand-worked pins of the learned-proposal oracle: features, the scoring network,
the proposal mixture, the visit ages and the training label, each on a case small
enough to be worked out on paper. The expected numbers below are written out (with
their derivation in the comments), not recomputed by the oracle, so that a dropped
logarithm, a transposed weight matrix, a row/column mix-up, an age off by one or a
wrong factor in the label fails one of them.

Feature readings (the paper names none; these are this library's): x0 = ln A_jj,
x1 = ln(1 + |r_j| / rms(r)), x2 = ln ||A[:, j]||_2, x3 = ln(1 + age_j), each
standardised over the coordinates as z = (x - mean) / (std + 1e-6) with the
population deviation. The label uses the projection identity of Section 3: one
step of sketch-and-project lowers ||w - w*||_A^2 by exactly r_C . delta."""
import math

import numpy as np

from oracle import learned as L

E = math.e


def _matrix_3x3():
    """Lower-triangular A with diagonal (1, e, e^2), so ln A_jj = (0, 1, 2), and
    column norms (e^3, e^2.5, e^2): column 0 = (1, sqrt(e^6 - 1), 0), column 1 =
    (0, e, sqrt(e^5 - e^2)), column 2 = (0, 0, e^2). Its row norms (1, ~20.2, ~13.9)
    differ from its column norms, so reading rows instead of columns is caught."""
    a = math.sqrt(E ** 6 - 1.0)   # 20.060627943629655
    c = math.sqrt(E ** 5 - E ** 2)  # 11.875356963209398
    return np.array([[1.0, 0.0, 0.0],
                     [a, E, 0.0],
                     [0.0, c, E ** 2]])


def test_static_features_by_hand():
    A = _matrix_3x3()
    z0, z2 = L.static_features(A)
    # (0, 1, 2): mean 1, population std sqrt(2/3) = 0.8164965809; z = +-1 / (0.8164965809 + 1e-6)
    assert np.allclose(z0, [-1.2247433713934262, 0.0, 1.2247433713934262], atol=1e-12, rtol=0)
    # (3, 2.5, 2): mean 2.5, std 0.5 sqrt(2/3) = 0.4082482905; z = +-0.5 / (0.4082482905 + 1e-6)
    assert np.allclose(z2, [1.2247418713989375, 0.0, -1.2247418713989375], atol=1e-12, rtol=0)


def test_residual_and_age_features_by_hand():
    A = _matrix_3x3()
    static = L.static_features(A)
    r = np.array([0.0, -0.7, 1.4])  # |r| = (0, 1, 2) t with t = 0.7
    age = np.array([2, 1, 3])
    Z = L.features(static, r, age)
    assert Z.shape == (3, 4)
    # rms = t sqrt(5/3); |r_j| / rms = (0, 0.7745966692, 1.5491933385);
    # x1 = ln(1 + .) = (0, 0.5735731685, 0.9357769713); mean 0.5031167133,
    # std 0.3852698553; z = (-1.3058972227, 0.1828778230, 1.1230193997)
    assert np.allclose(Z[:, 1], [-1.3058972226579102, 0.18287782298292166, 1.1230193996749884],
                       atol=1e-9, rtol=0)
    # x3 = (ln 3, ln 2, ln 4) = (1.0986122887, 0.6931471806, 1.3862943611); mean 1.0593512768,
    # std 0.2843390563; z = (0.1380797884, -1.2879287030, 1.1498489146)
    assert np.allclose(Z[:, 3], [0.13807978839184945, -1.287928702963058, 1.149848914571209],
                       atol=1e-9, rtol=0)
    # columns 0 and 2 are the static pair, in that order
    assert np.allclose(Z[:, 0], static[0]) and np.allclose(Z[:, 2], static[1])
    # a zero residual gives a zero residual feature
    assert np.all(L.features(static, np.zeros(3), age)[:, 1] == 0.0)


def _small_network():
    """The real 4 -> 64 -> 64 -> 1 layout with all but a few weights zero:
      h1_0 = relu(z0 + 0.5), h1_1 = relu(-z1 + z3 - 3), h1_2 = relu(z2 - 1);
      h2_0 = relu(3 h1_2 - 1), h2_1 = relu(-2 h1_0), h2_2 = relu(7 h1_1 + 0.25);
      s = 2 h2_0 + 10 h2_1 + 4 h2_2 - 0.5.
    W2 is not symmetric: W2[0, 2] = 3 reads unit 2 of the first layer into unit 0."""
    theta = np.zeros(L.N_PARAMS)
    W1, b1, W2, b2, w3, _ = L.unpack(theta)  # views into theta
    W1[0] = [1, 0, 0, 0]
    W1[1] = [0, -1, 0, 1]
    W1[2] = [0, 0, 1, 0]
    b1[:3] = [0.5, -3.0, -1.0]
    W2[0, 2] = 3.0
    W2[1, 0] = -2.0
    W2[2, 1] = 7.0
    b2[:3] = [-1.0, 0.0, 0.25]
    w3[:3] = [2.0, 10.0, 4.0]
    theta[-1] = -0.5
    return theta


def test_network_forward_by_hand():
    theta = _small_network()
    Z = np.array([[1.0, 2.0, 3.0, 4.0],
                  [0.0, 0.0, 0.0, 9.0]])
    # row 0: h1 = (1.5, relu(-2 + 4 - 3) = 0, 2); h2 = (relu(6 - 1) = 5, relu(-3) = 0, 0.25);
    #        s = 10 + 0 + 1 - 0.5 = 10.5. (With W2 transposed: h2 = (0, 14, 4.75), s = 158.5.)
    # row 1: h1 = (0.5, relu(9 - 3) = 6, relu(-1) = 0); h2 = (relu(-1) = 0, relu(-1) = 0, 42.25);
    #        s = 169 - 0.5 = 168.5
    s = L.forward(theta, Z)
    assert np.array_equal(s, [10.5, 168.5])
    # every value above is a bfloat16 number, so the bfloat16 pipeline gives the same
    assert np.array_equal(L.forward(theta, Z, bf16_mode=True), [10.5, 168.5])


def test_proposal_mixture_by_hand():
    # s = (0, ln 3): softmax = (1/4, 3/4); eps = 0.2, m = 2: p = 0.8 (1/4, 3/4) + 0.1 = (0.3, 0.7)
    lp = L.log_proposal(np.array([0.0, math.log(3.0)]), 0.2)
    assert np.allclose(np.exp(lp), [0.3, 0.7], rtol=0, atol=1e-15)


def test_label_from_a_2x2_projection_by_hand():
    # A = [[2, 1], [1, 2]], b = (3, 3): w* = (1, 1). From w = 0, r = A w - b = (-3, -3) and
    # ||w - w*||_A^2 = (1, 1) A (1, 1)^T = 6 = (w - w*) . r. Sampling C = {0} (tau = 1):
    # delta = r_0 / A_00 = -1.5, a_0 = r_0 delta = 4.5 = r_0^2 / A_00, the whole decrease.
    # Label = (1/2) ln(m a / ||e||_A^2 + 1e-3) = (1/2) ln(2 * 4.5 / 6 + 0.001) = (1/2) ln 1.501.
    assert math.isclose(float(L.label(np.array([4.5]), 6.0, 2)[0]), 0.20306577632566242,
                        rel_tol=1e-14)
    A = np.array([[2.0, 1.0], [1.0, 2.0]])
    b = np.array([3.0, 3.0])
    out = L.solve_learned(A, b, None, 1, seed=0, tol=0.0, max_iters=1, chunk=1,
                          w_star=np.array([1.0, 1.0]), collect=True)
    (j,) = out["samples"][0]
    feats, target = out["data"]
    assert feats.shape == (1, 4) and target.shape == (1,)
    # either coordinate gives the same numbers (A and b are symmetric under the swap)
    assert math.isclose(float(target[0]), 0.20306577632566242, rel_tol=1e-12)
    # after the step: w_j = 1.5, the other 0; the A-norm error fell by exactly 4.5 (6 -> 1.5)
    e = out["w"] - 1.0
    assert math.isclose(float(e @ A @ e), 1.5, rel_tol=1e-14)
    assert out["w"][j] == 1.5 and out["w"][1 - j] == 0.0


def test_visit_ages_by_hand():
    """Chunks of one iteration and tau = 1, uniform draws: at iteration 2 the
    coordinate drawn at iteration 1 has age 1, the one drawn at iteration 0 age 2,
    and a never-drawn one age k0 + 1 = 3. The training row of iteration 2 carries
    the standardised ln(1 + age) of the coordinate it draws, which takes one of three
    hand-computed values (ages {1, 2, 3}: ln 2, ln 3, ln 4)."""
    A = np.diag([2.0, 3.0, 5.0]) + 0.1
    b = np.array([1.0, -2.0, 0.5])
    w_star = np.linalg.solve(A, b)
    expect = {1: -1.287928702963058, 2: 0.13807978839184945, 3: 1.149848914571209}
    checked = 0
    for seed in range(40):
        out = L.solve_learned(A, b, None, 1, seed=seed, tol=0.0, max_iters=3, chunk=1,
                              w_star=w_star, collect=True)
        c0, c1, c2 = (int(s[0]) for s in out["samples"])
        if c0 == c1:
            continue  # needs three distinct ages
        age = 1 if c2 == c1 else (2 if c2 == c0 else 3)
        z3 = out["data"][0][2, 3]
        assert math.isclose(z3, expect[age], abs_tol=1e-9), (seed, age, z3)
        # iteration 0: every coordinate is unvisited (age 1), so the feature is constant -> 0
        assert out["data"][0][0, 3] == 0.0
        checked += 1
    assert checked >= 10
