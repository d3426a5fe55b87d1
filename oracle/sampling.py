"""Randomness of the protocol, drawn from fixed Philox streams (oracle).

Sec. 2.2 (BFV): encryption of m is (c0, c1) = (-a*s + e + [q m / t], a) with a
uniform, s the secret key and e a small error.  Alg. 1 step 3 (and Alg. 2
step 3): the model owner draws a uniform mask s in Z_t.

Readings (the paper fixes none of these): the secret key is ternary; e is a
discrete Gaussian with sigma = 3.2, tail-cut at |e| <= 19 (~6 sigma), sampled
by inversion of its cumulative table (CDT) at 63-bit resolution; a is drawn
directly as an NTT-domain value, exactly uniform mod q_i: one 64-bit word per
coefficient, kept when it lies below the largest multiple of q_i under 2^64
(then reduced mod q_i), else replaced by a word from a fallback counter.
"""
from __future__ import annotations

from functools import lru_cache
from typing import List

import mpmath

from .philox import (DOMAIN_A, DOMAIN_E, DOMAIN_MASK, DOMAIN_MASK_PAD, DOMAIN_FLOOD,
                     DOMAIN_PK_U, DOMAIN_SECRET, philox4x64)

CDT_TAIL = 19
CDT_BITS = 63


@lru_cache(maxsize=None)
def cdt_table(sigma: float = 3.2, tail: int = CDT_TAIL) -> tuple:
    """T[j] = floor(2^63 * P(|E| <= j)) for j = 0 .. tail-1.

    E is the discrete Gaussian on the integers of [-tail, tail] with
    P(E = x) proportional to exp(-x^2 / (2 sigma^2)).  Evaluated at 60 digits
    with mpmath, then floored.  sigma is passed as its decimal string so the
    value 3.2 is exact.
    """
    mpmath.mp.dps = 60
    s = mpmath.mpf(repr(sigma))
    rho = [mpmath.exp(-(mpmath.mpf(x) ** 2) / (2 * s * s)) for x in range(tail + 1)]
    z = rho[0] + 2 * sum(rho[1:])
    out = []
    acc = rho[0]
    for j in range(tail):
        if j > 0:
            acc += 2 * rho[j]
        out.append(int(mpmath.floor(acc / z * (mpmath.mpf(2) ** CDT_BITS))))
    return tuple(out)


def cdt_sample(w: int, table) -> int:
    """Map one 64-bit word to a signed error: |e| = #{j : T[j] <= u}, u = w mod 2^63,
    sign = top bit of w."""
    u = w & ((1 << CDT_BITS) - 1)
    mag = 0
    for tj in table:
        if u >= tj:
            mag += 1
    return -mag if (w >> 63) else mag


def ternary_secret(seed: int, n: int) -> List[int]:
    """Secret key coefficients s_i = (w_i mod 3) - 1 in {-1, 0, 1}."""
    out = []
    for blk in range(n // 4):
        w = philox4x64((blk, 0, 0, 0), (seed, DOMAIN_SECRET))
        out.extend((x % 3) - 1 for x in w)
    return out


def uniform_a(seed: int, ct: int, limb: int, n: int, q: int, domain: int = DOMAIN_A) -> List[int]:
    """Encryption mask a for (ciphertext ct, limb), already in NTT form (the
    public key's a with domain DOMAIN_PK_A, ct = 0).  Coefficient i takes word
    i % 4 of the block at counter (i / 4, ct, limb, 0); a word w is accepted when
    w < floor(2^64 / q) q, and then a_i = w mod q (every residue equally likely);
    a rejected word is replaced by word 0 of the block at counter (i, ct, limb, r)
    for r = 1, 2, ... until one is accepted (the fourth counter word is never 0
    there, so these blocks are disjoint from the main ones)."""
    bound = ((1 << 64) // q) * q
    out = []
    for blk in range(n // 4):
        w = philox4x64((blk, ct, limb, 0), (seed, domain))
        for r in range(4):
            i, x, attempt = 4 * blk + r, w[r], 0
            while x >= bound:
                attempt += 1
                x = philox4x64((i, ct, limb, attempt), (seed, domain))[0]
            out.append(x % q)
    return out


def gaussian_error(seed: int, ct: int, n: int, sigma: float = 3.2, domain: int = DOMAIN_E) -> List[int]:
    """Encryption error e for ciphertext ct (one integer polynomial, all limbs);
    the public key's error and public-key encryption's e2 use their own domains."""
    table = cdt_table(sigma)
    out = []
    for blk in range(n // 4):
        w = philox4x64((blk, ct, 0, 0), (seed, domain))
        out.extend(cdt_sample(x, table) for x in w)
    return out


def ternary_u(seed: int, ct: int, n: int) -> List[int]:
    """Public-key encryption's u for ciphertext ct: (w_i mod 3) - 1 in {-1, 0, 1}."""
    out = []
    for blk in range(n // 4):
        w = philox4x64((blk, ct, 0, 0), (seed, DOMAIN_PK_U))
        out.extend((x % 3) - 1 for x in w)
    return out


def mask_element(seed: int, flat: int, t: int) -> int:
    """Model owner's mask for output element `flat` (row-major over the output)."""
    return philox4x64((flat // 4, 0, 0, 0), (seed, DOMAIN_MASK))[flat % 4] % t


def mask_elements(seed: int, count: int, t: int) -> List[int]:
    out = []
    for blk in range((count + 3) // 4):
        out.extend(x % t for x in philox4x64((blk, 0, 0, 0), (seed, DOMAIN_MASK)))
    return out[:count]


def mask_pad(seed: int, ct_out: int, n: int, t: int) -> List[int]:
    """Mask for the coefficients of output ciphertext ct_out that carry no output."""
    out = []
    for blk in range(n // 4):
        out.extend(x % t for x in philox4x64((blk, ct_out, 0, 0), (seed, DOMAIN_MASK_PAD)))
    return out


def flood_noise(seed: int, ct_out: int, n: int, bits: int) -> List[int]:
    """Flooding noise added to returned ciphertext ct_out: coefficient i is
    (w mod 2^(bits+1)) - 2^bits, uniform in [-2^bits, 2^bits), w = Philox word
    (key (seed, DOMAIN_FLOOD), counter (i / 4, ct_out, 0, 0)) i % 4."""
    out = []
    for blk in range(n // 4):
        out.extend((x % (1 << (bits + 1))) - (1 << bits)
                   for x in philox4x64((blk, ct_out, 0, 0), (seed, DOMAIN_FLOOD)))
    return out
