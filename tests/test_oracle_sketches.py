"""Pins of the explicit sketch matrices against their definitions (Section 4)."""
import json
import os

import numpy as np
import pytest

from oracle import sketches as sk
from oracle.rng import subsample_indices

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_hadamard_recursion_matches_printed_H2_and_entry_formula():
    assert np.array_equal(sk.hadamard_matrix(1), np.array(GOLD["hadamard_H2"]["value"]))
    for q in range(0, 7):
        H = sk.hadamard_matrix(q)
        n = 1 << q
        E = sk.hadamard_entry(np.arange(n)[:, None], np.arange(n)[None, :])
        assert np.array_equal(H, E)
        assert np.array_equal(H @ H, n * np.eye(n))


def test_tau_rule_values_printed():
    g = GOLD["tau_rule_rcv1"]
    assert sk.default_tau(g["m"]) == g["tau"]
    # the ceiling rule is the exact integer ceiling of m^(2/3)
    for m in [1, 8, 27, 64, 500, 4096, 50000]:
        t = sk.default_tau(m)
        assert t ** 3 >= m * m and (t - 1) ** 3 < m * m
    ga = GOLD["tau_rule_accel"]
    assert sk.default_tau(ga["m"]) - 1 == ga["tau_floor"]  # ceil = floor + 1 here


def test_subcount_params_rule():
    ex = GOLD["subcount_example"]
    assert sk.subcount_params(100, ex["tau"], ex["s"]) == (ex["s"], ex["k"])
    assert sk.subcount_params(4096, 256) == (2560, 10)
    assert sk.subcount_params(506, 126) == (504, 4)
    assert sk.subcount_params(500, 50) == (500, 10)
    with pytest.raises(ValueError):
        sk.subcount_params(100, 30, 50)


@pytest.mark.parametrize("k", [0, 1, 5])
def test_subsample_structure(k):
    m, tau = 37, 9
    S = sk.sketch_matrix("subsample", m, tau, 3, k)
    assert np.array_equal(S.T @ S, np.eye(tau))
    C = subsample_indices(3, k, m, tau)
    assert np.array_equal(S[C, np.arange(tau)], np.ones(tau))


@pytest.mark.parametrize("k", [0, 4])
def test_count_structure(k):
    m, tau = 200, 16
    S = sk.sketch_matrix("count", m, tau, 8, k)
    nz = (S != 0).sum(axis=1)
    assert np.all(nz == 1)
    assert set(np.unique(S[S != 0])) <= {-1.0, 1.0}
    StS = S.T @ S
    assert np.array_equal(StS, np.diag((S != 0).sum(axis=0).astype(float)))


def test_subcount_structure():
    m, tau, s = 300, 12, 96
    S = sk.sketch_matrix("subcount", m, tau, 2, 1, s=s)
    kk = s // tau
    assert (np.abs(S).sum(axis=1) > 0).sum() == s
    assert np.all((S != 0).sum(axis=0) == kk)
    assert np.array_equal(S.T @ S, kk * np.eye(tau))


def test_srht_orthogonal_without_padding():
    m, tau = 64, 10
    S = sk.sketch_matrix("srht", m, tau, 4, 2)
    assert np.allclose(S.T @ S, np.eye(tau) / tau, atol=1e-15)


def test_srht_padding_shape():
    m, tau = 100, 20
    assert sk.srht_pad(m) == 128
    S = sk.sketch_matrix("srht", m, tau, 4, 2)
    assert S.shape == (m, tau)
    assert np.allclose(np.abs(S), 1.0 / np.sqrt(tau * 128))


def test_gaussian_sketch_moments():
    S = sk.sketch_matrix("gaussian", 400, 50, 1, 0)
    assert abs(S.mean()) < 0.02 and abs(S.var() - 1.0) < 0.03


@pytest.mark.parametrize("kind", sk.KINDS)
def test_sketched_matrix_symmetric_psd(kind):
    g = np.random.default_rng(0)
    X = g.standard_normal((30, 20))
    A = X.T @ X + 0.1 * np.eye(20)
    S = sk.sketch_matrix(kind, 20, 6, 5, 3, s=12 if kind == "subcount" else None)
    M = S.T @ A @ S
    assert np.allclose(M, M.T, atol=1e-12)
    assert np.linalg.eigvalsh((M + M.T) / 2).min() > -1e-10
