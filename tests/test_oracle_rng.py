"""Pins of the oracle's counter-based draws: the published SplitMix64 outputs,
samples that are permutations, and uniformity of samples, buckets, signs and
Gaussian entries (what the sketch definitions of Section 4 require)."""
import itertools
import json
import os

import numpy as np
import pytest
from scipy import stats

from oracle import rng

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_splitmix64_published_outputs():
    outs = GOLD["splitmix64_seed0"]["outputs_hex"]
    for n, hx in enumerate(outs, start=1):
        z = np.array([(n * rng.GAMMA) % 2 ** 64], dtype=np.uint64)
        assert int(rng.mix64(z)[0]) == int(hx, 16)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 16, 63, 64, 65, 100, 500, 4097])
def test_full_sample_is_a_permutation(n):
    for k in range(3):
        p = rng.subsample_indices(7, k, n, n)
        assert sorted(p.tolist()) == list(range(n))
        # a prefix sample is the prefix of the full ordering
        assert np.array_equal(rng.subsample_indices(7, k, n, (n + 1) // 2), p[: (n + 1) // 2])


def test_subsample_pairs_uniform():
    # every unordered 2-subset of [6] has probability 1/15 (eq. (15))
    n, t, N = 6, 2, 15000
    counts = {}
    for k in range(N):
        c = tuple(sorted(rng.subsample_indices(3, k, n, t).tolist()))
        counts[c] = counts.get(c, 0) + 1
    allp = list(itertools.combinations(range(n), 2))
    obs = np.array([counts.get(c, 0) for c in allp])
    assert obs.sum() == N
    chi2 = stats.chisquare(obs)
    assert chi2.pvalue > 1e-4


def test_ordered_triples_uniform():
    # the ordered sample is uniform over the 5*4*3 ordered triples of [5]
    n, t, N = 5, 3, 12000
    counts = {}
    for k in range(N):
        c = tuple(rng.subsample_indices(13, k, n, t).tolist())
        counts[c] = counts.get(c, 0) + 1
    allp = list(itertools.permutations(range(n), t))
    obs = np.array([counts.get(c, 0) for c in allp])
    assert obs.sum() == N
    assert stats.chisquare(obs).pvalue > 1e-4


def test_first_sample_position_uniform():
    n, N = 37, 20000
    first = np.array([rng.subsample_indices(11, k, n, 1)[0] for k in range(N)])
    obs = np.bincount(first, minlength=n)
    assert stats.chisquare(obs).pvalue > 1e-4


def test_buckets_and_signs_uniform():
    tau = 50
    sign, bucket = rng.signs_buckets(5, 0, 200000, tau)
    assert bucket.min() >= 0 and bucket.max() < tau
    assert stats.chisquare(np.bincount(bucket, minlength=tau)).pvalue > 1e-4
    assert set(np.unique(sign).tolist()) == {-1, 1}
    assert abs(sign.mean()) < 4.0 / np.sqrt(sign.size)


def test_gaussian_entries_standard_normal():
    z = rng.gaussian_entries(9, 3, 200000)
    assert np.all(np.isfinite(z))
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert abs(z.mean()) < 0.02 and abs(z.var() - 1.0) < 0.02


def test_draws_depend_on_every_counter_field():
    base = rng.draw(1, 2, 1, np.arange(4, dtype=np.uint64))
    assert not np.array_equal(base, rng.draw(2, 2, 1, np.arange(4, dtype=np.uint64)))
    assert not np.array_equal(base, rng.draw(1, 3, 1, np.arange(4, dtype=np.uint64)))
    assert not np.array_equal(base, rng.draw(1, 2, 2, np.arange(4, dtype=np.uint64)))
    assert len(set(base.tolist())) == 4
