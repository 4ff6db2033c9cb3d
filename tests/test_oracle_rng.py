"""Pins of the oracle's random-number layer against facts outside the oracle.

- Philox4x32-10 words against the published known-answer vectors.
- Normals: the Box-Muller identity recomputed from raw words, moments and a
  Kolmogorov-Smirnov test against scipy's normal CDF.
- Gamma (Marsaglia-Tsang): mean and variance equal the shape, KS test against
  scipy's gamma CDF, and the acceptance rate bound of the method.
"""
import math
import os

import numpy as np
import pytest
import scipy.stats as st

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    assert oracle.philox(ctr, key) == expect


def test_normal_stream_box_muller_identity():
    # normal q comes from call q//4, words (2p, 2p+1) with p = (q%4)//2:
    # z_even^2 + z_odd^2 = -2 ln u and atan2(z_odd, z_even) = 2 pi t (mod 2 pi)
    seed, c1, c2, c3 = 0x1234_5678_9ABC_DEF0, 17, 3, 2
    z = oracle.normal_stream(seed, c1, c2, c3, 0, 64)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for call in range(16):
        w = oracle.philox([call, c1, c2, c3], key)
        for p in range(2):
            u = ((w[2 * p] >> 8) + 1) * 2.0**-24
            t = (w[2 * p + 1] >> 8) * 2.0**-24
            ze, zo = z[4 * call + 2 * p], z[4 * call + 2 * p + 1]
            assert ze * ze + zo * zo == pytest.approx(-2.0 * math.log(u), rel=1e-12, abs=1e-15)
            ang = math.atan2(zo, ze) % (2 * math.pi)
            assert min(abs(ang - 2 * math.pi * t), 2 * math.pi - abs(ang - 2 * math.pi * t)) < 1e-9


def test_normal_stream_offsets_are_consistent():
    a = oracle.normal_stream(5, 1, 2, 3, 0, 40)
    b = oracle.normal_stream(5, 1, 2, 3, 13, 20)
    np.testing.assert_array_equal(a[13:33], b)


def test_normal_moments_and_ks():
    n = 400_000
    z = oracle.normal_stream(2024, 7, 0, 9, 0, n)
    se = 1.0 / math.sqrt(n)
    assert abs(z.mean()) < 5 * se
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0) * se
    assert abs(np.mean(z**4) - 3.0) < 5 * math.sqrt(96.0) * se
    assert abs(np.mean(z**3)) < 5 * math.sqrt(15.0) * se
    assert st.kstest(z, "norm").pvalue > 1e-4


def test_streams_differ_by_field():
    base = oracle.normal_stream(1, 2, 3, 4, 0, 8)
    for args in [(2, 2, 3, 4), (1, 3, 3, 4), (1, 2, 4, 4), (1, 2, 3, 5)]:
        other = oracle.normal_stream(*args, 0, 8)
        assert not np.allclose(base, other)


@pytest.mark.parametrize("shape", [1.0, 2.5, 10.0, 1000.0])
def test_gamma_moments(shape):
    n = 20_000
    x = np.array([oracle.gamma(99, shape, c1, 5, 6)[0] for c1 in range(n)])
    se = math.sqrt(shape / n)
    assert abs(x.mean() - shape) < 5 * se
    # Var = shape; the variance of the sample variance is (kurtosis-1) var^2/n
    kurt = 3.0 + 6.0 / shape
    assert abs(x.var() - shape) < 5 * math.sqrt((kurt - 1.0) / n) * shape


def test_gamma_ks_and_acceptance():
    shape = 2.5
    draws = [oracle.gamma(3, shape, c1, 0, 7) for c1 in range(20_000)]
    x = np.array([d[0] for d in draws])
    att = np.array([d[1] for d in draws])
    assert st.kstest(x, "gamma", args=(shape,)).pvalue > 1e-4
    # Marsaglia-Tsang accepts with probability > 0.95 for shape >= 1
    assert (1.0 / att.mean()) > 0.9


def test_chi_square_via_gamma():
    # chi^2(m) = 2 Gamma(m/2): mean m, variance 2m
    m = 7.0
    x = 2.0 * np.array([oracle.gamma(11, m / 2, c1, 1, 7)[0] for c1 in range(20_000)])
    assert abs(x.mean() - m) < 5 * math.sqrt(2 * m / 20_000)
    assert st.kstest(x, "chi2", args=(m,)).pvalue > 1e-4
