"""Pins for oracle.params: primes and roots against sympy (an independent library)."""
import pytest
import sympy

from oracle.params import BfvParams, is_prime, min_primitive_root_2n, ntt_primes

CASES = [(4096, 54, 2), (8192, 60, 3), (4096, 60, 4), (16384, 60, 4), (64, 60, 3)]


@pytest.mark.parametrize("n,bits,count", CASES)
def test_primes_are_largest_ntt_friendly(n, bits, count):
    qs = ntt_primes(bits, count, 2 * n)
    assert qs == sorted(qs, reverse=True)
    top = (1 << bits)
    # every candidate = 1 mod 2N in (q_last, 2^bits) is either listed or composite (sympy)
    cand = (top - 1) // (2 * n) * (2 * n) + 1
    seen = []
    while cand >= qs[-1]:
        if cand < top and sympy.isprime(cand):
            seen.append(cand)
        cand -= 2 * n
    assert seen == qs
    for q in qs:
        assert q % (2 * n) == 1 and q < top


def test_workload_primes():
    # the moduli of the two workloads: N = 4096 with two primes below 2^54, N = 8192 with three below 2^60
    assert ntt_primes(54, 2, 8192) == [0x3ffffffffd6001, 0x3ffffffffd2001]
    assert ntt_primes(60, 3, 16384) == [0xfffffffffffc001, 0xffffffffffe8001, 0xffffffffffd8001]


def test_miller_rabin_matches_sympy():
    import random
    r = random.Random(5)
    for _ in range(3000):
        n = r.randrange(2, 1 << 64)
        assert is_prime(n) == sympy.isprime(n)
    for n in range(2, 5000):
        assert is_prime(n) == sympy.isprime(n)


@pytest.mark.parametrize("n,bits,count", CASES)
def test_psi_order_and_minimality(n, bits, count):
    for q in ntt_primes(bits, count, 2 * n):
        psi = min_primitive_root_2n(q, 2 * n)
        assert sympy.n_order(psi, q) == 2 * n
        # all primitive 2N-th roots are g^((q-1)/2N * k), k odd, for a generator g (sympy)
        g = sympy.primitive_root(q)
        base = pow(g, (q - 1) // (2 * n), q)
        roots = [pow(base, k, q) for k in range(1, 2 * n, 2)]
        assert psi == min(roots)


def test_psi_bruteforce_small_prime():
    # q = 97, 2N = 16: brute force over every element of Z_97^*
    q, two_n = 97, 16
    psi = min_primitive_root_2n(q, two_n)
    orders = {x: sympy.n_order(x, q) for x in range(1, q)}
    assert psi == min(x for x, o in orders.items() if o == two_n)


def test_params_delta():
    p = BfvParams(log_n=12, num_primes=2, prime_bits=54)
    assert p.delta == p.q // (1 << 41)
    assert p.q == p.primes[0] * p.primes[1]
