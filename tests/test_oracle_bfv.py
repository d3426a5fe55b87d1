"""Pins for oracle.bfv: Dec(Enc(m)) = m, homomorphic plaintext product against
the schoolbook product over Z_t, re-masking Dec(W Enc(r) - s) + s = W r, and
the noise check flagging a corrupted ciphertext."""
import random

import numpy as np
import pytest

from oracle import bfv
from oracle.params import BfvParams
from oracle.ring import negacyclic_schoolbook


@pytest.fixture(scope="module", params=[(6, 2, 54), (7, 3, 60)])
def params(request):
    log_n, L, bits = request.param
    return BfvParams(log_n=log_n, num_primes=L, prime_bits=bits)


def test_roundtrip(params):
    p = params
    sk = bfv.keygen(p, 1)
    r = random.Random(2)
    for idx in range(3):
        m = [r.randrange(p.t) for _ in range(p.n)]
        ct = bfv.encrypt(p, sk, m, seed=9, ct_index=idx)
        assert bfv.decrypt(p, sk, ct) == m
        assert bfv.noise_budget_ok(p, sk, ct)


def test_encrypt_is_randomised_by_index(params):
    p = params
    sk = bfv.keygen(p, 1)
    m = [0] * p.n
    a = bfv.encrypt(p, sk, m, seed=9, ct_index=0)
    b = bfv.encrypt(p, sk, m, seed=9, ct_index=1)
    assert not (a == b).all()


def test_plain_product_and_mask(params):
    p = params
    sk = bfv.keygen(p, 3)
    r = random.Random(4)
    x = [r.randrange(p.t) for _ in range(p.n)]
    w = [r.randrange(-(1 << 15), 1 << 15) for _ in range(p.n)]
    s = [r.randrange(p.t) for _ in range(p.n)]
    ct = bfv.encrypt(p, sk, x, seed=5, ct_index=0)
    out = bfv.sub_plain(p, bfv.mul_plain(p, ct, bfv.encode_plain(p, [v % p.t for v in w])), s)
    dec = bfv.decrypt(p, sk, out)
    want = negacyclic_schoolbook(x, [v % p.t for v in w], p.t)
    assert [(d + si) % p.t for d, si in zip(dec, s)] == want


def test_add_plain(params):
    p = params
    sk = bfv.keygen(p, 3)
    r = random.Random(6)
    x1 = [r.randrange(p.t) for _ in range(p.n)]
    x0 = [r.randrange(p.t) for _ in range(p.n)]
    ct = bfv.add_plain(p, bfv.encrypt(p, sk, x1, seed=5, ct_index=2), x0)
    assert bfv.decrypt(p, sk, ct) == [(a + b) % p.t for a, b in zip(x0, x1)]


def test_noise_check_flags_corruption():
    p = BfvParams(log_n=6, num_primes=2, prime_bits=54)
    sk = bfv.keygen(p, 1)
    ct = bfv.encrypt(p, sk, [1] * p.n, seed=1, ct_index=0)
    bad = ct.copy()
    bad[0, 0, 3] = (bad[0, 0, 3] + p.primes[0] // 3) % p.primes[0]
    assert bfv.noise_budget_ok(p, sk, ct)
    assert not bfv.noise_budget_ok(p, sk, bad)


def test_uniform_product_at_paper_parameters_decrypts():
    """t = 2^59, q ~ 2^180 (Sec. 6): Dec(w * Enc(m) - s) + s = w * m mod t for
    UNIFORM w and m in Z_t (Alg. 2's cross terms multiply two shares).  With the
    plain Delta m scaling the (q mod t) x overflow term of this product exceeds
    Delta / 2 and decryption fails; with round(q m / t) it does not."""
    p = BfvParams(log_n=10, num_primes=3, prime_bits=60, t_bits=59)
    sk = bfv.keygen(p, 17)
    g = np.random.default_rng(5)
    m = [int(v) for v in g.integers(0, p.t, p.n, dtype=np.uint64)]
    w = [int(v) for v in g.integers(0, p.t, p.n, dtype=np.uint64)]
    s = [int(v) for v in g.integers(0, p.t, p.n, dtype=np.uint64)]
    ct = bfv.mul_plain(p, bfv.encrypt(p, sk, m, 3, 0), bfv.encode_plain(p, w))
    ct = bfv.sub_plain(p, ct, s)
    assert bfv.noise_budget_ok(p, sk, ct)
    got = bfv.decrypt(p, sk, ct)
    want = negacyclic_schoolbook([bfv.centered(v, p.t) for v in w], m, p.t)
    assert [(a + b) % p.t for a, b in zip(got, s)] == [int(v) % p.t for v in want]


def _negacyclic_int(a, b):
    """Exact negacyclic product of two small integer polynomials (int64)."""
    n = len(a)
    full = np.convolve(np.asarray(a, dtype=np.int64), np.asarray(b, dtype=np.int64))
    out = full[:n].copy()
    out[:n - 1] -= full[n:]
    return out


def test_public_key_relation(params):
    """p0 + p1 s = -e: the key's phase is exactly the negated error of its own
    stream (coefficient form), so p0 carries -(a s) with the right sign."""
    from oracle import sampling
    from oracle.philox import DOMAIN_PK_E
    p = params
    sk = bfv.keygen(p, 3)
    pk = bfv.pk_keygen(p, sk, 11)
    e = sampling.gaussian_error(11, 0, p.n, p.sigma, DOMAIN_PK_E)
    phase = bfv.from_ntt(p, np.stack([(pk.p0[i] + pk.p1[i] * sk.s_hat[i]) % q for i, q in enumerate(p.primes)]))
    for i, q in enumerate(p.primes):
        assert [int(v) for v in phase[i]] == [(-x) % q for x in e]
    assert any(e)


def test_public_key_encryption_phase_and_roundtrip(params):
    """Enc_pk: c0 + c1 s - round(q m / t) = e1 - u e + e2 s exactly, every
    product recomputed as a schoolbook negacyclic convolution over the
    integers (no NTT), and Dec recovers m."""
    from oracle import sampling
    from oracle.philox import DOMAIN_PK_E, DOMAIN_PK_E2
    p = params
    sk = bfv.keygen(p, 3)
    pk = bfv.pk_keygen(p, sk, 11)
    r = random.Random(4)
    for idx in (0, 2):
        m = [r.randrange(p.t) for _ in range(p.n)]
        ct = bfv.encrypt_pk(p, pk, m, seed=21, ct_index=idx)
        assert bfv.decrypt(p, sk, ct) == m
        assert bfv.noise_budget_ok(p, sk, ct)
        u = sampling.ternary_u(21, idx, p.n)
        e = sampling.gaussian_error(11, 0, p.n, p.sigma, DOMAIN_PK_E)
        e1 = sampling.gaussian_error(21, idx, p.n, p.sigma)
        e2 = sampling.gaussian_error(21, idx, p.n, p.sigma, DOMAIN_PK_E2)
        noise = np.asarray(e1, dtype=np.int64) - _negacyclic_int(u, e) + _negacyclic_int(e2, sk.s)
        got = bfv.decrypt_phase(p, sk, ct)
        for j in range(p.n):
            want = (p.q * m[j] + p.t // 2) // p.t + int(noise[j])
            assert got[j] == want % p.q, j
    assert set(u) == {-1, 0, 1}
    # independent ciphertexts of the same message differ
    assert not (bfv.encrypt_pk(p, pk, m, 21, 0) == bfv.encrypt_pk(p, pk, m, 21, 1)).all()
