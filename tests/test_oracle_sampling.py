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


def _numpy_block(counter, key):
    """Philox4x64-10 block from numpy's independent implementation (numpy
    advances its counter by one before producing a block)."""
    c = sum(int(x) << (64 * i) for i, x in enumerate(counter))
    k = sum(int(x) << (64 * i) for i, x in enumerate(key))
    return [int(x) for x in np.random.Philox(counter=(c - 1) % (1 << 256), key=k).random_raw(4)]


def test_uniform_a_range_and_stream():
    q = 0xfffffffffffc001
    a = sampling.uniform_a(3, ct=5, limb=1, n=64, q=q)
    assert all(0 <= x < q for x in a)
    # one 64-bit word per coefficient, four per block (no word of this block is rejected:
    # the bound 16 q is 2^64 - 16 (2^60 - q), rejections have probability 2^-46)
    for blk in (0, 7, 15):
        w = _numpy_block((blk, 5, 1, 0), (3, 2))
        assert all(x < 16 * q for x in w)
        assert a[4 * blk: 4 * blk + 4] == [x % q for x in w]
    mean = np.mean([x / q for x in sampling.uniform_a(9, 0, 0, 1 << 14, q)])
    assert abs(mean - 0.5) < 0.01


def test_uniform_a_rejection_fallback():
    """With a modulus just above 2^63 the bound is q itself and about half of the
    words are rejected: each rejected position takes word 0 of the fallback
    blocks (i, ct, limb, 1), (i, ct, limb, 2), ... (numpy's words), in order."""
    q = (1 << 63) + 29
    a = sampling.uniform_a(4, ct=2, limb=3, n=32, q=q)
    rejected = 0
    for blk in range(8):
        w = _numpy_block((blk, 2, 3, 0), (4, 2))
        for r in range(4):
            i, x, attempt = 4 * blk + r, w[r], 0
            if x >= q:
                rejected += 1
            while x >= q:
                attempt += 1
                x = _numpy_block((i, 2, 3, attempt), (4, 2))[0]
            assert a[i] == x
    assert rejected > 4
    # the values are exactly uniform on [0, q): the mean of many is near q / 2
    big = sampling.uniform_a(5, 0, 0, 1 << 13, q)
    assert abs(np.mean([x / q for x in big]) - 0.5) < 0.02


def test_mask_streams():
    t = 1 << 41
    m = sampling.mask_elements(13, 10, t)
    assert m == [sampling.mask_element(13, i, t) for i in range(10)]
    assert m[5] == philox4x64((1, 0, 0, 0), (13, DOMAIN_MASK))[1] % t
    pad = sampling.mask_pad(13, 2, 16, t)
    assert len(pad) == 16 and all(0 <= x < t for x in pad)
