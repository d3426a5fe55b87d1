"""Pins for oracle.protocol: Alg. 1 reconstructs W o X + b, the grad_X role
reconstructs the input gradient, Alg. 2 reconstructs grad_W -- each against
the direct ring operators -- and decoded shares do not depend on the partition."""
import numpy as np
import pytest

from oracle import bfv, protocol
from oracle.packing import Partition
from oracle.params import BfvParams
from oracle.protocol import DGRAD, FWD, WGRAD, Layer
from paper_2403_11166_gb300 import inputs

P_SMALL = BfvParams(log_n=7, num_primes=2, prime_bits=54)     # weights small: q ~ 2^108 suffices
P_BIG = BfvParams(log_n=7, num_primes=3, prime_bits=60)       # uniform shares as multipliers


def _mask(x, t_bits=41):
    return np.asarray(x).astype(np.uint64) & np.uint64((1 << t_bits) - 1)


def _add(a, b):
    with np.errstate(over="ignore"):
        return _mask(np.asarray(a, dtype=np.uint64) + np.asarray(b, dtype=np.uint64))


FC = Layer("fc", B=3, Ci=10, Co=5)
CONV = Layer("conv", B=2, Ci=3, Co=2, h=5, w=4, s=3, pad=1)


@pytest.mark.parametrize("layer,part", [
    (FC, Partition(2, 4, 3, 1, 1, 1, 1)),
    (CONV, Partition(1, 2, 1, 3, 2, 3, 3)),
])
def test_forward_reconstructs(layer, part):
    p = P_SMALL
    g = inputs.rng(0)
    sk = bfv.keygen(p, 1)
    W = inputs.gaussian_fixed(g, layer.w_shape())
    x = inputs.gaussian_fixed(g, layer.x_shape())
    b = inputs.gaussian_fixed(g, (layer.Co,), frac_bits=24)
    x0, x1 = inputs.split_shares(g, x)
    y0, y1, *_ = protocol.he_linear(p, sk, layer, FWD, part, W, x1, x0, 11, 12, bias=b)
    want = _add(protocol.ring_op(layer, FWD, W, x, 41).reshape(layer.y_shape()),
                np.asarray(b).astype(np.int64).view(np.uint64).reshape((1, -1) + (1,) * (len(layer.y_shape()) - 2)))
    assert (_add(y0, y1) == want).all()


@pytest.mark.parametrize("layer,part", [
    (FC, Partition(3, 2, 4, 1, 1, 1, 1)),
    (CONV, Partition(1, 1, 2, 2, 3, 3, 3)),
])
def test_dgrad_reconstructs(layer, part):
    p = P_SMALL
    g = inputs.rng(1)
    sk = bfv.keygen(p, 2)
    W = inputs.gaussian_fixed(g, layer.w_shape())
    gy = inputs.gaussian_fixed(g, layer.y_shape())
    gy0, gy1 = inputs.split_shares(g, gy)
    gx0, gx1, *_ = protocol.he_linear(p, sk, layer, DGRAD, part, W, gy1, gy0, 21, 22)
    want = protocol.ring_op(layer, DGRAD, W, gy, 41).reshape(layer.x_shape())
    assert (_add(gx0, gx1) == want).all()


@pytest.mark.parametrize("layer,part", [
    (FC, Partition(4, 2, 3, 1, 1, 1, 1)),
    (CONV, Partition(1, 1, 1, 3, 3, 2, 2)),
])
def test_wgrad_reconstructs(layer, part):
    p = P_BIG
    g = inputs.rng(2)
    sk = bfv.keygen(p, 3)
    x = inputs.gaussian_fixed(g, layer.x_shape())
    gy = inputs.gaussian_fixed(g, layer.y_shape())
    x0, x1 = inputs.split_shares(g, x)
    gy0, gy1 = inputs.split_shares(g, gy)
    gw, tilde, s = protocol.he_wgrad(p, sk, layer, part, gy0, gy1, x0, x1, 31, 32, 33)
    want = protocol.ring_op(layer, WGRAD, gy, x, 41).reshape(layer.w_shape())
    assert (gw == want).all()


def test_partition_independence():
    p = P_SMALL
    g = inputs.rng(3)
    sk = bfv.keygen(p, 4)
    layer = CONV
    W = inputs.gaussian_fixed(g, layer.w_shape())
    x = inputs.gaussian_fixed(g, layer.x_shape())
    x0, x1 = inputs.split_shares(g, x)
    a = protocol.he_linear(p, sk, layer, FWD, Partition(1, 3, 2, 3, 2, 3, 3), W, x1, x0, 1, 2)
    b = protocol.he_linear(p, sk, layer, FWD, Partition(2, 1, 1, 2, 2, 3, 3), W, x1, x0, 5, 2)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()


def test_simulator_view_zero_input_gives_minus_mask():
    """MO's view with Enc(0) in place of Enc(<X>_1) (and <X>_0 = 0): the protocol
    still runs and the DO decrypts exactly -s."""
    p = P_SMALL
    g = inputs.rng(4)
    sk = bfv.keygen(p, 5)
    layer = FC
    W = inputs.gaussian_fixed(g, layer.w_shape())
    zero = np.zeros(layer.x_shape(), dtype=np.uint64)
    y0, y1, *_ = protocol.he_linear(p, sk, layer, FWD, Partition(1, 5, 5, 1, 1, 1, 1), W, zero, zero, 7, 8)
    assert (_add(y0, y1) == 0).all()


def test_noise_flooding_keeps_shares_and_adds_exactly_the_flood_polynomial():
    """Flooding a returned ciphertext (circuit privacy; the paper is silent): the
    flooded ciphertext minus the unflooded one is NTT(f) with f uniform in
    [-2^B, 2^B), and the decrypted shares are unchanged."""
    from oracle import bfv as obfv, sampling
    from oracle.packing import Partition as Pt
    from oracle.params import BfvParams as BP
    p = BP(log_n=10, num_primes=3, prime_bits=60)
    sk = obfv.keygen(p, 2)
    L = Layer("conv", B=1, Ci=2, Co=2, h=4, w=4, s=3, pad=1)
    part = Pt(1, 2, 2, 4, 4, 3, 3)
    g = np.random.default_rng(3)
    W = g.integers(-2000, 2000, L.w_shape())
    x1 = g.integers(0, 1 << 41, L.x_shape(), dtype=np.uint64)
    x0 = g.integers(0, 1 << 41, L.x_shape(), dtype=np.uint64)
    plain = protocol.he_linear(p, sk, L, "fwd", part, W, x1, x0, 5, 6)
    flooded = protocol.he_linear(p, sk, L, "fwd", part, W, x1, x0, 5, 6, flood_bits=62)
    assert (np.asarray(plain[0]) == np.asarray(flooded[0])).all()
    assert (np.asarray(plain[1]) == np.asarray(flooded[1])).all()
    f = sampling.flood_noise(6, 0, p.n, 62)
    assert min(f) >= -(1 << 62) and max(f) < (1 << 62) and max(abs(v) for v in f) > (1 << 60)
    diff = obfv.add_noise(p, plain[4][0], f)
    assert (diff == flooded[4][0]).all()
    assert not (plain[4][0] == flooded[4][0]).all()


@pytest.mark.parametrize("kind,role", [("conv", "fwd"), ("conv", "dgrad"), ("fc", "fwd"), ("conv", "wgrad")])
def test_compact_return_form_decrypts_to_the_same_share(kind, role):
    """Dropping the coefficients that carry no output before sending: decrypting
    the send form (c1 in NTT form, c0 only at output coefficients) gives exactly
    the DO share that decrypting the whole ciphertexts gives, and the send form
    is smaller by one c0 per ciphertext minus one word per output and limb."""
    from oracle import bfv as obfv
    from oracle.packing import Partition as Pt, counts
    from oracle.params import BfvParams as BP
    p = BP(log_n=10, num_primes=3, prime_bits=60)
    sk = obfv.keygen(p, 2)
    g = np.random.default_rng(5)
    if kind == "conv":
        L = Layer("conv", B=2, Ci=3, Co=2, h=5, w=4, s=3, pad=1)
        part = Pt(1, 2, 2, 4, 4, 3, 3) if role != "wgrad" else Pt(1, 2, 2, 4, 4, 4, 4)
    else:
        L = Layer("fc", B=3, Ci=20, Co=7, h=1, w=1, s=1, pad=0)
        part = Pt(2, 8, 4, 1, 1, 1, 1)
    t = 1 << 41
    if role in ("fwd", "dgrad"):
        W = g.integers(-2000, 2000, L.w_shape())
        shape = L.x_shape() if role == "fwd" else L.y_shape()
        v1 = g.integers(0, t, shape, dtype=np.uint64)
        v0 = g.integers(0, t, shape, dtype=np.uint64)
        _, y1, _, _, ct_out = protocol.he_linear(p, sk, L, role, part, W, v1, v0, 5, 6)
    else:
        x0, x1 = (g.integers(0, t, L.x_shape(), dtype=np.uint64) for _ in range(2))
        gy0, gy1 = (g.integers(0, t, L.y_shape(), dtype=np.uint64) for _ in range(2))
        _, y1, _ = protocol.he_wgrad(p, sk, L, part, gy0, gy1, x0, x1, 5, 6, 7)
        c = counts(protocol.geometry(L, WGRAD), part)
        cx = protocol.encrypt_inputs(p, sk, L, WGRAD, part, x1, 5)
        cg = protocol.encrypt_kernel_operand(p, sk, L, WGRAD, part, gy1, 6)
        pg = protocol.encode_kernel(p, L, WGRAD, part, gy0)
        px = protocol.encode_input(p, L, WGRAD, part, x0)
        ct_out = {i: protocol.mo_wgrad_ct(p, L, part, cx, pg, cg, px, 7, i) for i in range(c.ct_out)}
    c1s, c0c = protocol.compact_returned(p, L, role, part, ct_out)
    got = protocol.decrypt_compact(p, sk, L, role, part, c1s, c0c)
    assert (got == np.asarray(y1, dtype=np.uint64).reshape(-1)).all()
    words = sum(v.size for v in c1s.values()) + c0c.size
    assert protocol.send_bytes(p, L, role, part, True) == 8 * words
    assert protocol.send_bytes(p, L, role, part, True) < protocol.send_bytes(p, L, role, part, False)
    # a c0 coefficient carrying no output really is dropped: changing one leaves the share unchanged
    idx = next(iter(ct_out))
    from oracle.packing import decode_positions
    used = {e for e, _ in decode_positions(protocol.geometry(L, role), part, idx // counts(
        protocol.geometry(L, role), part).NC, idx % counts(protocol.geometry(L, role), part).NC)}
    free = [e for e in range(p.n) if e not in used]
    if free:
        bad = {k: v.copy() for k, v in ct_out.items()}
        coeff = obfv.from_ntt(p, bad[idx][0])
        for li, qi in enumerate(p.primes):
            coeff[li, free[0]] = (coeff[li, free[0]] + qi // 3) % qi
        bad[idx][0] = obfv.to_ntt(p, coeff)
        c1b, c0b = protocol.compact_returned(p, L, role, part, bad)
        assert (protocol.decrypt_compact(p, sk, L, role, part, c1b, c0b) == got).all()
