"""Negacyclic number-theoretic transform (oracle; test infrastructure only).

Sec. 5 ("NTT"): the NTT is a bijection between Z_q[X]/(X^N+1) and Z_q^N under
which ring multiplication becomes element-wise multiplication.  With psi a
primitive 2N-th root of unity, X^N + 1 = prod_i (X - psi^(2i+1)), so the
transform evaluates a polynomial at the odd powers of psi.

Reading (order of the evaluation points, which the paper leaves open): slot i
holds a(psi^(2*brv(i)+1)), brv = bit reversal on log2(N) bits.  This is the
order a Cooley-Tukey loop with in-place butterflies produces, so a GPU
transform can write its result without a final permutation.

`ntt_definition` / `intt_definition` are the O(N^2) sums themselves.
`ntt_radix2` / `intt_radix2` are plain butterfly loops, checked against the
definition and against the schoolbook product (convolution theorem) in
tests/test_oracle_ntt.py.  Both work on Python integers (numpy object arrays),
exactly.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np

from .params import bit_reverse


def _log2(n: int) -> int:
    b = n.bit_length() - 1
    assert 1 << b == n
    return b


def ntt_definition(a, q: int, psi: int):
    """hat_a[i] = sum_j a_j * psi^((2 brv(i) + 1) j) mod q."""
    n = len(a)
    bits = _log2(n)
    out = []
    for i in range(n):
        root = pow(psi, 2 * bit_reverse(i, bits) + 1, q)
        acc, p = 0, 1
        for j in range(n):
            acc += int(a[j]) * p
            p = p * root % q
        out.append(acc % q)
    return out


def intt_definition(ahat, q: int, psi: int):
    """a_j = N^{-1} sum_i hat_a[i] * psi^(-(2 brv(i) + 1) j) mod q."""
    n = len(ahat)
    bits = _log2(n)
    psi_inv = pow(psi, -1, q)
    n_inv = pow(n, -1, q)
    out = [0] * n
    for i in range(n):
        root = pow(psi_inv, 2 * bit_reverse(i, bits) + 1, q)
        p = 1
        v = int(ahat[i])
        for j in range(n):
            out[j] += v * p
            p = p * root % q
    return [x * n_inv % q for x in out]


@lru_cache(maxsize=None)
def _twiddles(n: int, q: int, psi: int):
    """psi^brv(k) and psi^-brv(k) for k in [0, n), as object arrays."""
    bits = _log2(n)
    psi_inv = pow(psi, -1, q)
    fwd = np.array([pow(psi, bit_reverse(k, bits), q) for k in range(n)], dtype=object)
    inv = np.array([pow(psi_inv, bit_reverse(k, bits), q) for k in range(n)], dtype=object)
    return fwd, inv


def ntt_radix2(a, q: int, psi: int):
    """Cooley-Tukey, natural order in, bit-reversed evaluation order out.

    Stage with m blocks of width 2t: block i pairs (x, x + t) under twiddle
    psi^brv(m + i): (x, y) -> (x + w y, x - w y).  Accepts shape (..., N).
    """
    a = np.array(a, dtype=object)
    n = a.shape[-1]
    lead = a.shape[:-1]
    fwd, _ = _twiddles(n, q, psi)
    m, t = 1, n // 2
    while m < n:
        v = a.reshape(lead + (m, 2, t))
        w = fwd[m:2 * m].reshape((m, 1))
        x = v[..., 0, :]
        y = v[..., 1, :] * w % q
        v = np.stack(((x + y) % q, (x - y) % q), axis=-2)
        a = v.reshape(lead + (n,))
        m, t = 2 * m, t // 2
    return a


def intt_radix2(ahat, q: int, psi: int):
    """Gentleman-Sande inverse of `ntt_radix2`, then scaling by N^{-1}."""
    a = np.array(ahat, dtype=object)
    n = a.shape[-1]
    lead = a.shape[:-1]
    _, inv = _twiddles(n, q, psi)
    m, t = n // 2, 1
    while m >= 1:
        v = a.reshape(lead + (m, 2, t))
        w = inv[m:2 * m].reshape((m, 1))
        x = v[..., 0, :]
        y = v[..., 1, :]
        v = np.stack(((x + y) % q, (x - y) * w % q), axis=-2)
        a = v.reshape(lead + (n,))
        m, t = m // 2, 2 * t
    n_inv = pow(n, -1, q)
    return a * n_inv % q
