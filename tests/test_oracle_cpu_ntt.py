"""The plain CPU NTT build agrees with the oracle's NTT (itself pinned to the
O(N^2) definition) and inverts itself."""
import numpy as np
import pytest

from oracle.cpu_ntt import CpuNtt, max_threads
from oracle.ntt import intt_radix2, ntt_radix2
from oracle.params import min_primitive_root_2n, ntt_primes


@pytest.mark.parametrize("log_n", [6, 10, 13])
def test_cpu_ntt_matches_oracle(log_n):
    n = 1 << log_n
    q = ntt_primes(60, 1, 2 * n)[0]
    psi = min_primitive_root_2n(q, 2 * n)
    g = np.random.default_rng(log_n)
    a = g.integers(0, q, size=(3, n), dtype=np.uint64)
    a[0] = q - 1
    c = CpuNtt(q, psi, log_n)
    b = a.copy()
    c.run(b, threads=2)
    for i in range(3):
        assert [int(v) for v in b[i]] == list(ntt_radix2([int(v) for v in a[i]], q, psi))
    c.run(b, inverse=True)
    assert (b == a).all()
    d = a.copy()
    c.run(d, inverse=True, threads=1)
    assert [int(v) for v in d[1]] == list(intt_radix2([int(v) for v in a[1]], q, psi))
    assert max_threads() >= 1
