"""Counter-based random draws for the sketches (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper draws its sketches with NumPy's global generator (Appendix B); any
source of independent uniform draws serves the method. Here every draw is a pure
function of (seed, iteration k, stream s, lane i) so that a second, independent
implementation (the CUDA library) can reproduce it exactly.

Definition (all arithmetic modulo 2^64):

    mix64(z):  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
               z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31
    GAMMA   =  0x9E3779B97F4A7C15
    key(seed, k)         = mix64(seed + (k + 1) * GAMMA)
    draw(seed, k, s, i)  = mix64(key(seed, k) + (1 + i + s * 2^40) * GAMMA)

``mix64`` and ``GAMMA`` are the output function and increment of SplitMix64
(Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014). Streams:  s = 0 sample keys, s = 1 sign + bucket,
s = 2 and s = 3 Gaussian uniforms, s = 4 proposal (Gumbel) noise.

Derived quantities:

* sign(i)   = -1 if bit 63 of draw(seed, k, 1, i) is set, else +1
* bucket(i) = ((draw(seed, k, 1, i) & 0xFFFFFFFF) * tau) >> 32   (multiply-shift
  range reduction, Lemire 2019), uniform on [0, tau) up to 2^-32 bias
* a uniformly random ordered sample without replacement C_0..C_{t-1} of [0, n):
  the t lanes with the smallest keys draw(seed, k, 0, i), i < n, in increasing
  order of (key, i). Every ordering of [0, n) by iid uniform keys is equally
  likely, so every ordered t-sample is too (ties, probability ~ n^2 2^-65, are
  broken by the lane index).
* Gaussian entry (Box-Muller): u1 = ((draw(.,2,i) >> 11) + 1) 2^-53,
  u2 = (draw(.,3,i) >> 11) 2^-53, z = sqrt(-2 ln u1) cos(2 pi u2).
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_G = np.uint64(GAMMA)


def mix64(z):
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def iter_key(seed: int, k: int) -> np.uint64:
    """key(seed, k) = mix64(seed + (k+1) GAMMA)."""
    v = (int(seed) + (int(k) + 1) * GAMMA) & MASK64
    return mix64(np.array([v], dtype=np.uint64))[0]


def draw(seed: int, k: int, s: int, i) -> np.ndarray:
    """draw(seed, k, s, i) for an integer array of lanes i (uint64 result)."""
    key = iter_key(seed, k)
    i = np.asarray(i, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = np.uint64(1) + i + np.uint64(int(s) << 40)
        return mix64(key + ctr * _G)


def sample_keys(seed: int, k: int, n: int) -> np.ndarray:
    """The keys draw(seed, k, 0, i) for i < n."""
    return draw(seed, k, 0, np.arange(n, dtype=np.uint64))


def subsample_indices(seed: int, k: int, n: int, count: int) -> np.ndarray:
    """Ordered sample C_0..C_{count-1} of distinct indices in [0, n): the lanes
    of the ``count`` smallest keys, by increasing (key, lane)."""
    if count > n:
        raise ValueError("sample larger than population")
    keys = sample_keys(seed, k, n)
    order = np.lexsort((np.arange(n), keys))
    return order[:count].astype(np.int64)


def signs_buckets(seed: int, k: int, count: int, tau: int):
    """(sign[i] in {-1,+1} as int8, bucket[i] in [0, tau) as int64) for i < count."""
    d = draw(seed, k, 1, np.arange(count, dtype=np.uint64))
    sign = np.where((d >> np.uint64(63)) != 0, -1, 1).astype(np.int8)
    with np.errstate(over="ignore"):
        bucket = ((d & np.uint64(0xFFFFFFFF)) * np.uint64(tau)) >> np.uint64(32)
    return sign, bucket.astype(np.int64)


def gaussian_entries(seed: int, k: int, count: int) -> np.ndarray:
    """``count`` standard normal draws (Box-Muller on two 53-bit uniforms)."""
    lanes = np.arange(count, dtype=np.uint64)
    u1 = ((draw(seed, k, 2, lanes) >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (draw(seed, k, 3, lanes) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
