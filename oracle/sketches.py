"""Explicit sketching matrices S (m x tau, dense float64), one per definition of
Section 4 of the paper.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Each function builds S literally from its definition so that a reader can check
it against the paper by eye; the iteration then uses S only through the
products S^T A S, S^T r, S delta and A S (Algorithm 2).

Pinned by: tests/test_oracle_sketches.py (structure: S^T S, bucket sizes,
Hadamard orthogonality, sample uniformity) and by the iteration pins of
tests/test_oracle_solver.py (one-step exactness, closed form).
"""
from __future__ import annotations

import math

import numpy as np

from .rng import gaussian_entries, signs_buckets, subsample_indices

KINDS = ("gaussian", "subsample", "count", "subcount", "srht")


def default_tau(m: int) -> int:
    """Rule of thumb tau = ceil(m^(2/3)) (Section 8.1 conclusions; the RCV1 run of
    Section 8.3 quotes tau = ceil(47236^(2/3)) = 1307). Exact integer ceiling:
    the smallest t with t^3 >= m^2."""
    t = max(1, int(round(m ** (2.0 / 3.0))))
    while t ** 3 < m * m:
        t += 1
    while t > 1 and (t - 1) ** 3 >= m * m:
        t -= 1
    return t


def subcount_params(m: int, tau: int, s: int | None = None):
    """(s, k) of the SubCount sketch. Paper rule (Section 4.2): k = 10 if
    10 tau <= m, else k = floor(m / tau); s = k tau. A caller-given s must be a
    multiple of tau no larger than m (then k = s / tau)."""
    if s is None or s == 0:
        k = 10 if 10 * tau <= m else m // tau
        if k < 1:
            raise ValueError("SubCount needs tau <= m")
        return k * tau, k
    if s % tau != 0 or s > m or s < tau:
        raise ValueError("SubCount s must be a multiple of tau in [tau, m]")
    return s, s // tau


def srht_pad(m: int) -> int:
    """m' = 2^ceil(log2 m): rows after zero padding (Section 4.3)."""
    return 1 << max(0, int(m - 1).bit_length()) if m > 1 else 1


def hadamard_entry(i, c):
    """Entry (i, c) of the Sylvester Hadamard matrix H_{2^q} of eq. (18):
    (-1)^{popcount(i & c)} (the recursive block definition unrolled bit by bit)."""
    x = np.bitwise_and(np.asarray(i, dtype=np.int64), np.asarray(c, dtype=np.int64))
    par = np.zeros_like(x)
    while np.any(x):
        par ^= x & 1
        x = x >> 1
    return 1 - 2 * par


def hadamard_matrix(q: int) -> np.ndarray:
    """H_{2^q} built by the recursion of eq. (18): H_1 = [1],
    H_{2n} = [[H_n, H_n], [H_n, -H_n]]."""
    H = np.ones((1, 1))
    for _ in range(q):
        H = np.block([[H, H], [H, -H]])
    return H


def sketch_matrix(kind: str, m: int, tau: int, seed: int, k: int, s: int | None = None):
    """S_k for iteration k as a dense m x tau float64 matrix.

    * gaussian  (Gaussian sketch, Section 4.1): S_ij iid N(0, 1); the lane of
      (i, j) is i*tau + j.
    * subsample (Subsampling sketch, Section 4.1, eq. (15)): S = I_C, C a uniform
      tau-subset of [m] in the order of the sample: S[C_j, j] = 1.
    * count     (Section 4.2): every row i of A gets a random sign and is added to
      a uniformly random output row: S[i, bucket(i)] = sign(i).
    * subcount  (SubCount sketch, Section 4.2, eq. (16)): S^T = Sigma D I_C with C
      an ordered s-sample, D random signs, Sigma summing k contiguous rows:
      S[C_p, p // k] = sign(p), p < s.
    * srht      (SRHT, Section 4.3, eq. (17)): S^T = (tau m')^{-1/2} I_C H_{m'} D on A padded
      with m' - m zero rows, so S = (tau m')^{-1/2} D_m H_{m'}[0:m, C] with C a
      tau-subset of [m'].
    """
    S = np.zeros((m, tau))
    if kind == "gaussian":
        S[:, :] = gaussian_entries(seed, k, m * tau).reshape(m, tau)
    elif kind == "subsample":
        C = subsample_indices(seed, k, m, tau)
        S[C, np.arange(tau)] = 1.0
    elif kind == "count":
        sign, bucket = signs_buckets(seed, k, m, tau)
        S[np.arange(m), bucket] = sign
    elif kind == "subcount":
        s_, kk = subcount_params(m, tau, s)
        C = subsample_indices(seed, k, m, s_)
        sign, _ = signs_buckets(seed, k, s_, tau)
        S[C, np.arange(s_) // kk] = sign
    elif kind == "srht":
        mp = srht_pad(m)
        if tau > mp:
            raise ValueError("SRHT needs tau <= m'")
        C = subsample_indices(seed, k, mp, tau)
        sign, _ = signs_buckets(seed, k, m, 1)
        H = hadamard_entry(np.arange(m)[:, None], C[None, :])
        S[:, :] = sign[:, None] * H / math.sqrt(tau * mp)
    else:
        raise ValueError(f"unknown sketch kind {kind!r}")
    return S
