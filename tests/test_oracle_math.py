"""Pins of the oracle's elementary functions and of its random-draw stream.

ln / exp are pinned against numpy's libm (an independent implementation):
the oracle's own series must stay within 2 ulp.  The Philox4x32-10 block
function (Salmon et al. 2011) is pinned bit for bit to its published
known-answer values (tests/golden/philox4x32_10_kat.txt), and the draw
stream built on it statistically (uniformity, independence, avalanche); the
CUDA side implements the same definition independently and the parity tests
compare the two streams.
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle


def _ulp_err(a, ref):
    return np.abs(a - ref) / np.spacing(np.abs(ref))


def test_log_within_2ulp_of_libm():
    rng = np.random.default_rng(11)
    # the draws the transport takes: multiples of 2^-53 in (0, 1]
    u = (rng.integers(0, 2**53, size=400_000, dtype=np.uint64).astype(np.float64) + 1.0) * 2.0**-53
    wide = np.exp(rng.uniform(-700, 700, size=400_000))
    near1 = 1.0 + rng.uniform(-0.3, 0.3, size=200_000)
    for x in (u, wide, near1):
        x = x[x != 1.0]
        err = _ulp_err(oracle.log(x), np.log(x))
        assert err.max() <= 2.0, err.max()
    assert oracle.log(np.array([1.0]))[0] == 0.0
    # products of four draws (Planck sampler) reach 2^-212
    assert abs(oracle.log(np.array([2.0**-212]))[0] / (-212 * np.log(2.0)) - 1) < 1e-15


def test_exp_within_2ulp_of_libm():
    rng = np.random.default_rng(12)
    x = np.concatenate([rng.uniform(-700, 700, 400_000), rng.uniform(-60, 0, 400_000),
                        rng.uniform(-1e-3, 1e-3, 100_000)])
    err = _ulp_err(oracle.exp(x), np.exp(x))
    assert err.max() <= 2.0, err.max()
    assert oracle.exp(np.array([0.0]))[0] == 1.0
    assert oracle.exp(np.array([-800.0]))[0] == 0.0


def test_draws_are_53bit_grid_uniform():
    z = oracle.uniforms(5469, 0, 17, 200_000)
    assert np.all(z >= 0.0) and np.all(z < 1.0)
    assert np.all(np.floor(z * 2.0**53) == z * 2.0**53)
    counts, _ = np.histogram(z, bins=200, range=(0, 1))
    chi2 = ((counts - z.size / 200) ** 2 / (z.size / 200)).sum()
    assert stats.chi2.sf(chi2, 199) > 1e-4
    assert stats.kstest(z, "uniform").pvalue > 1e-4


def test_streams_of_neighbouring_counters_are_independent():
    a = oracle.uniforms(5469, 0, 1000, 50_000)
    b = oracle.uniforms(5469, 0, 1001, 50_000)
    c = oracle.uniforms(5469, 1, 1000, 50_000)
    d = oracle.uniforms(5470, 0, 1000, 50_000)
    for o in (b, c, d):
        r = np.corrcoef(a, o)[0, 1]
        assert abs(r) < 5 * (1 / np.sqrt(a.size)), r
    # consecutive draws of one stream uncorrelated
    assert abs(np.corrcoef(a[:-1], a[1:])[0, 1]) < 5 / np.sqrt(a.size)


def test_philox_avalanche_and_key_dependence():
    rng = np.random.default_rng(3)
    flips = []
    for _ in range(300):
        ctr = rng.integers(0, 2**32, size=4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, size=2, dtype=np.uint64).astype(np.uint32)
        o = oracle.philox(ctr, key)
        bit = int(rng.integers(0, 128))
        c2 = ctr.copy()
        c2[bit // 32] ^= np.uint32(1 << (bit % 32))
        o2 = oracle.philox(c2, key)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(o, o2)))
        k2 = key.copy()
        k2[0] ^= np.uint32(1)
        assert not np.array_equal(oracle.philox(ctr, k2), o)
    m = np.mean(flips)
    assert 60 < m < 68, m  # half of 128 output bits on average


def test_philox_known_answers():
    """The published known-answer values of Philox4x32-10 (tests/golden/
    philox4x32_10_kat.txt): the oracle's generator is the published one, word
    for word, so every draw of both sides is pinned."""
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        w = [int(x, 16) for x in r]
        out = oracle.philox(w[0:4], w[4:6])
        assert [int(v) for v in out] == w[6:10], r
