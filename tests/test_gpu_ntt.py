"""GPU parity: parameters, batched NTT / INTT (pencil_ntt_batch) against the oracle."""
import numpy as np
import pytest
import torch

from oracle.ntt import intt_radix2, ntt_radix2
from oracle.params import BfvParams
from tests.gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu

CFGS = [(12, 2, 54), (13, 3, 60), (14, 4, 60), (13, 1, 50), (12, 4, 60)]


@pytest.fixture(scope="module")
def he():
    from paper_2403_11166_gb300 import he
    return he


@pytest.mark.parametrize("cfg", CFGS)
def test_primes_and_roots(he, cfg):
    ctx = he.Context(*cfg)
    p = BfvParams(log_n=cfg[0], num_primes=cfg[1], prime_bits=cfg[2])
    q, psi = ctx.primes()
    assert q == p.primes and psi == p.psis


def _random_polys(p, count, seed):
    g = np.random.default_rng(seed)
    a = np.zeros((count, p.num_primes, p.n), dtype=np.uint64)
    for j, q in enumerate(p.primes):
        a[:, j] = g.integers(0, q, size=(count, p.n), dtype=np.uint64)
    # adversarial rows: all zero, all q-1, a single spike
    if count >= 3:
        a[0] = 0
        for j, q in enumerate(p.primes):
            a[1, j] = q - 1
        a[2] = 0
        a[2, :, 7] = 1
    return a


@pytest.mark.parametrize("cfg", CFGS)
def test_ntt_matches_oracle(he, cfg):
    ctx = he.Context(*cfg)
    p = BfvParams(log_n=cfg[0], num_primes=cfg[1], prime_bits=cfg[2])
    a = _random_polys(p, 5, cfg[0])
    d = to_dev(a)
    he.pencil_ntt_batch(ctx, d, inverse=False)
    got = to_np(d)
    for i in range(a.shape[0]):
        for j, (q, psi) in enumerate(zip(p.primes, p.psis)):
            want = ntt_radix2([int(x) for x in a[i, j]], q, psi)
            assert (got[i, j] == np.array(list(want), dtype=object).astype(np.uint64)).all(), (i, j)
    he.pencil_ntt_batch(ctx, d, inverse=True)
    assert (to_np(d) == a).all()


@pytest.mark.parametrize("cfg", CFGS[:3])
def test_intt_matches_oracle(he, cfg):
    ctx = he.Context(*cfg)
    p = BfvParams(log_n=cfg[0], num_primes=cfg[1], prime_bits=cfg[2])
    a = _random_polys(p, 2, 100 + cfg[0])
    d = to_dev(a)
    he.pencil_ntt_batch(ctx, d, inverse=True)
    got = to_np(d)
    for i in range(a.shape[0]):
        for j, (q, psi) in enumerate(zip(p.primes, p.psis)):
            want = intt_radix2([int(x) for x in a[i, j]], q, psi)
            assert (got[i, j] == np.array(list(want), dtype=object).astype(np.uint64)).all()


@pytest.mark.parametrize("log_n,radix", [(14, 4), (14, 5), (13, 5), (12, 5)])
def test_both_register_radices_match_oracle(he, log_n, radix):
    """The NTT radix knob (2^4 or 2^5 coefficients per thread) changes only the
    schedule: forward and inverse transforms equal the oracle's for either."""
    cfg = (log_n, 2, 60)
    ctx = he.Context(*cfg)
    ctx.tune(he.TUNE_NTT_LOG_RADIX, radix)
    p = BfvParams(log_n=log_n, num_primes=2, prime_bits=60)
    a = _random_polys(p, 2, 300 + log_n + radix)
    d = to_dev(a)
    he.pencil_ntt_batch(ctx, d, inverse=False)
    got = to_np(d)
    for i in range(a.shape[0]):
        for j, (q, psi) in enumerate(zip(p.primes, p.psis)):
            want = ntt_radix2([int(x) for x in a[i, j]], q, psi)
            assert (got[i, j] == np.array(list(want), dtype=object).astype(np.uint64)).all(), (i, j)
    d = to_dev(a)
    he.pencil_ntt_batch(ctx, d, inverse=True)
    got = to_np(d)
    for i in range(a.shape[0]):
        for j, (q, psi) in enumerate(zip(p.primes, p.psis)):
            want = intt_radix2([int(x) for x in a[i, j]], q, psi)
            assert (got[i, j] == np.array(list(want), dtype=object).astype(np.uint64)).all(), (i, j)


def test_large_batch_roundtrip(he):
    """Full-size sweep shape (N = 8192, 3 limbs) on a batch that spans many waves:
    INTT(NTT(a)) = a everywhere, NTT spot-checked against the oracle."""
    ctx = he.Context(13, 3, 60)
    p = BfvParams(log_n=13, num_primes=3, prime_bits=60)
    a = _random_polys(p, 1000, 7)
    d = to_dev(a)
    he.pencil_ntt_batch(ctx, d, inverse=False)
    got = to_np(d)
    for i in (0, 517, 999):
        j = i % 3
        want = ntt_radix2([int(x) for x in a[i, j]], p.primes[j], p.psis[j])
        assert (got[i, j] == np.array(list(want), dtype=object).astype(np.uint64)).all()
    he.pencil_ntt_batch(ctx, d, inverse=True)
    assert torch.equal(d, to_dev(a))


@pytest.mark.parametrize("log_n,L,radix", [(13, 3, 4), (13, 3, 5), (14, 4, 4), (14, 4, 5), (12, 4, 4), (12, 2, 5)])
@pytest.mark.parametrize("arith", [0, 1])
def test_butterfly_arithmetic_knob_matches_oracle(he, log_n, L, radix, arith):
    """Both butterfly arithmetics (Shoup / Harvey and the pseudo-Mersenne folds
    with lazily growing values) give the oracle's transforms for every radix,
    including the all-(q - 1) and single-spike rows."""
    ctx = he.Context(log_n, L, 60)
    ctx.tune(he.TUNE_NTT_ARITH, arith)
    ctx.tune(he.TUNE_NTT_LOG_RADIX, radix)
    assert ctx.get_tune(he.TUNE_NTT_ARITH) == arith
    p = BfvParams(log_n=log_n, num_primes=L, prime_bits=60)
    a = _random_polys(p, 4, 500 + log_n + radix + 7 * arith)
    d = to_dev(a)
    he.pencil_ntt_batch(ctx, d, inverse=False)
    fwd = to_np(d)
    d2 = to_dev(a)
    he.pencil_ntt_batch(ctx, d2, inverse=True)
    inv = to_np(d2)
    for i in (1, 2, 3):
        j = i % L
        q, psi = p.primes[j], p.psis[j]
        want = ntt_radix2([int(x) for x in a[i, j]], q, psi)
        assert (fwd[i, j] == np.array(list(want), dtype=object).astype(np.uint64)).all(), (i, j)
        want = intt_radix2([int(x) for x in a[i, j]], q, psi)
        assert (inv[i, j] == np.array(list(want), dtype=object).astype(np.uint64)).all(), (i, j)
    he.pencil_ntt_batch(ctx, d, inverse=True)
    assert (to_np(d) == a).all()


def test_fold_arithmetic_needs_pseudo_mersenne_primes(he):
    """54-bit primes are not 2^60 - c: the fold butterflies are refused there and
    the context keeps the Shoup arithmetic."""
    ctx = he.Context(12, 2, 54)
    assert ctx.get_tune(he.TUNE_NTT_ARITH) == 0
    with pytest.raises(he.PencilError):
        ctx.tune(he.TUNE_NTT_ARITH, 1)
    assert he.Context(13, 3, 60).get_tune(he.TUNE_NTT_ARITH) == 1
