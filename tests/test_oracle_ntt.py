"""Pins for oracle.ntt / oracle.ring: the O(N^2) definition, the radix-2 loop,
the convolution theorem against the schoolbook product, and a hand-checked
N = 4 product (X^4 = -1)."""
import random

import pytest

from oracle.ntt import intt_definition, intt_radix2, ntt_definition, ntt_radix2
from oracle.params import min_primitive_root_2n, ntt_primes
from oracle.ring import negacyclic_schoolbook


def _setup(n, bits=60):
    q = ntt_primes(bits, 1, 2 * n)[0]
    return q, min_primitive_root_2n(q, 2 * n)


def test_schoolbook_n4_by_hand():
    q = 97
    # (1 + 2X + 3X^2 + 4X^3)(5 + 6X + 7X^2 + 8X^3) with X^4 = -1
    # coefficients of the full product: 5, 16, 34, 60, 61, 52, 32
    # X^4 -> -1, X^5 -> -X, X^6 -> -X^2
    want = [(5 - 61) % q, (16 - 52) % q, (34 - 32) % q, 60 % q]
    assert negacyclic_schoolbook([1, 2, 3, 4], [5, 6, 7, 8], q) == want
    # X^3 * X = X^4 = -1
    assert negacyclic_schoolbook([0, 0, 0, 1], [0, 1, 0, 0], q) == [q - 1, 0, 0, 0]


@pytest.mark.parametrize("n", [8, 16, 64, 256])
def test_radix2_equals_definition(n):
    q, psi = _setup(n)
    r = random.Random(n)
    a = [r.randrange(q) for _ in range(n)]
    assert list(ntt_radix2(a, q, psi)) == ntt_definition(a, q, psi)
    assert list(intt_radix2(a, q, psi)) == intt_definition(a, q, psi)


@pytest.mark.parametrize("n", [8, 32, 128])
def test_definition_inverse(n):
    q, psi = _setup(n, 54)
    r = random.Random(n + 1)
    a = [r.randrange(q) for _ in range(n)]
    assert intt_definition(ntt_definition(a, q, psi), q, psi) == a


@pytest.mark.parametrize("n", [1024, 4096, 8192])
def test_radix2_roundtrip(n):
    q, psi = _setup(n)
    r = random.Random(n)
    a = [r.randrange(q) for _ in range(n)]
    assert list(intt_radix2(ntt_radix2(a, q, psi), q, psi)) == a


@pytest.mark.parametrize("n", [8, 16, 64, 1024])
def test_convolution_theorem(n):
    q, psi = _setup(n)
    r = random.Random(3 * n)
    a = [r.randrange(q) for _ in range(n)]
    b = [r.randrange(q) for _ in range(n)]
    prod = [x * y % q for x, y in zip(ntt_radix2(a, q, psi), ntt_radix2(b, q, psi))]
    assert list(intt_radix2(prod, q, psi)) == negacyclic_schoolbook(a, b, q)


def test_monomial_evaluation_points():
    # NTT(X) lists the evaluation points psi^(2 brv(i) + 1); they are the N distinct roots of X^N + 1
    n = 16
    q, psi = _setup(n)
    pts = list(ntt_radix2([0, 1] + [0] * (n - 2), q, psi))
    assert len(set(pts)) == n
    for x in pts:
        assert pow(x, n, q) == q - 1
    assert pts[0] == psi          # brv(0) = 0
    assert pts[1] == pow(psi, n + 1, q)   # brv(1) = N/2 -> exponent N + 1
