"""Pins for oracle.sampling: the CDT against a float64 evaluation of the same
distribution, sample moments, and the support / range of every sampler."""
import math

import numpy as np

from oracle import sampling
from oracle.philox import DOMAIN_MASK, philox4x64


def test_cdt_table_matches_float64():
    tab = sampling.cdt_table(3.2)
    xs = np.arange(-19, 20, dtype=np.float64)
    rho = np.exp(-xs ** 2 / (2 * 3.2 ** 2))
    p = rho / rho.sum()
    cum = [p[19 - j:19 + j + 1].sum() for j in range(19)]
    assert len(tab) == 19
    for tj, cj in zip(tab, cum):
        assert abs(tj / 2.0 ** 63 - cj) < 1e-13
    assert all(a < b for a, b in zip(tab, tab[1:]))
    assert tab[-1] < 2 ** 63


def test_cdt_sample_edges():
    tab = sampling.cdt_table(3.2)
    assert sampling.cdt_sample(0, tab) == 0
    assert sampling.cdt_sample(tab[0], tab) == 1                # first step
    assert sampling.cdt_sample(tab[0] | (1 << 63), tab) == -1
    assert sampling.cdt_sample((1 << 63) - 1, tab) == 19        # tail
    assert sampling.cdt_sample((1 << 64) - 1, tab) == -19


def test_gaussian_moments():
    e = []
    for ct in range(40):
        e.extend(sampling.gaussian_error(seed=7, ct=ct, n=4096))
    e = np.array(e, dtype=np.float64)
    assert abs(e.mean()) < 0.03
    assert abs(e.var() - 3.2 ** 2) < 0.15
    assert np.abs(e).max() <= 19


def test_ternary_uniform():
    s = np.array(sampling.ternary_secret(11, 1 << 15))
    assert set(np.unique(s)) == {-1, 0, 1}
    counts = np.bincount(s + 1)
    assert np.all(np.abs(counts / len(s) - 1 / 3) < 0.01)


def test_uniform_a_range_and_stream():
    q = 0xfffffffffffc001
    a = sampling.uniform_a(3, ct=5, limb=1, n=64, q=q)
    assert all(0 <= x < q for x in a)
    w = philox4x64((0, 5, 1, 0), (3, 2))
    assert a[0] == ((w[0] << 64) | w[1]) % q and a[1] == ((w[2] << 64) | w[3]) % q
    mean = np.mean([x / q for x in sampling.uniform_a(9, 0, 0, 1 << 14, q)])
    assert abs(mean - 0.5) < 0.01


def test_mask_streams():
    t = 1 << 41
    m = sampling.mask_elements(13, 10, t)
    assert m == [sampling.mask_element(13, i, t) for i in range(10)]
    assert m[5] == philox4x64((1, 0, 0, 0), (13, DOMAIN_MASK))[1] % t
    pad = sampling.mask_pad(13, 2, 16, t)
    assert len(pad) == 16 and all(0 <= x < t for x in pad)
