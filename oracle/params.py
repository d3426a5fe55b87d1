"""BFV / RNS parameters (oracle; test infrastructure only).

Sec. 2.2: BFV is parameterised by {N, t, q}; the plaintext ring is
Z_t[X]/(X^N+1), ciphertexts live in (Z_q[X]/(X^N+1))^2.  Sec. 5 ("RNS
Decomposition"): q = q_1 ... q_L with every q_i < 2^64, arithmetic per limb.
Sec. 5 ("NTT"): products in the ring become pointwise after a negacyclic NTT,
which needs q_i = 1 mod 2N and a primitive 2N-th root of unity psi_i.

Readings (the paper leaves these open):
* primes are the largest q_i < 2^bits with q_i = 1 mod 2N, in descending order;
* psi_i is the numerically smallest primitive 2N-th root of unity mod q_i;
* Delta = floor(q / t)  (the usual BFV scaling factor); messages are scaled as
  round(q m / t) = Delta m + round((q mod t) m / t) (see bfv.py).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

# Deterministic Miller-Rabin bases: correct for every n < 3.3e24 (> 2^64).
_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin primality test for n < 3.3e24."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def ntt_primes(bits: int, count: int, two_n: int) -> List[int]:
    """The `count` largest primes q < 2^bits with q = 1 (mod two_n), descending."""
    out = []
    q = ((1 << bits) - 1) // two_n * two_n + 1
    if q >= (1 << bits):
        q -= two_n
    while len(out) < count:
        if q <= two_n:
            raise ValueError("ran out of candidates")
        if is_prime(q):
            out.append(q)
        q -= two_n
    return out


def min_primitive_root_2n(q: int, two_n: int) -> int:
    """Smallest psi in [1, q) whose multiplicative order mod q is exactly two_n.

    two_n is a power of two, so psi has order two_n iff psi^(two_n/2) = -1.
    Any one such root psi0 generates all of them as psi0^k for odd k.
    """
    assert (q - 1) % two_n == 0
    half = two_n // 2
    exp = (q - 1) // two_n
    g = 2
    while True:
        psi0 = pow(g, exp, q)
        if pow(psi0, half, q) == q - 1:
            break
        g += 1
    best = psi0
    sq = psi0 * psi0 % q
    cur = psi0
    for _ in range(half - 1):
        cur = cur * sq % q
        if cur < best:
            best = cur
    return best


def bit_reverse(i: int, bits: int) -> int:
    r = 0
    for _ in range(bits):
        r = (r << 1) | (i & 1)
        i >>= 1
    return r


@dataclass
class BfvParams:
    """BFV instance {N, t, q = prod q_i} (Sec. 2.2) with per-limb NTT roots."""

    log_n: int
    num_primes: int
    prime_bits: int
    t_bits: int = 41
    sigma: float = 3.2
    primes: List[int] = field(default_factory=list)
    psis: List[int] = field(default_factory=list)

    def __post_init__(self):
        n = 1 << self.log_n
        if not self.primes:
            self.primes = ntt_primes(self.prime_bits, self.num_primes, 2 * n)
        if not self.psis:
            self.psis = [min_primitive_root_2n(q, 2 * n) for q in self.primes]

    @property
    def n(self) -> int:
        return 1 << self.log_n

    @property
    def t(self) -> int:
        return 1 << self.t_bits

    @property
    def q(self) -> int:
        out = 1
        for p in self.primes:
            out *= p
        return out

    @property
    def delta(self) -> int:
        """Delta = floor(q / t)."""
        return self.q // self.t
