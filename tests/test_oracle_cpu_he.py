"""The plain CPU build of the HE pipeline (oracle/cpu_he.c, the timed CPU
baseline) reaches exactly the oracle's protocol: raw ciphertexts, plaintexts,
output ciphertexts and both shares of Alg. 1 (forward and input-gradient
roles, conv and FC, ragged partitions) and of Alg. 2, bit for bit, with one
thread and with several."""
import numpy as np
import pytest

from oracle import bfv, protocol
from oracle.cpu_he import CpuHe
from oracle.packing import Partition
from oracle.params import BfvParams
from oracle.protocol import DGRAD, FWD, WGRAD, Layer
from paper_2403_11166_gb300 import inputs

P = BfvParams(log_n=12, num_primes=2, prime_bits=54)


@pytest.fixture(scope="module")
def keys():
    return bfv.keygen(P, 5), CpuHe(P, 5)


def _as_u64(d, idx):
    return np.array(d[idx], dtype=object).astype(np.uint64)


@pytest.mark.parametrize("L,role,part,threads", [
    (Layer("conv", B=3, Ci=3, Co=4, h=6, w=5, s=3, pad=1), FWD, (2, 2, 3, 4, 3, 3, 2), 1),
    (Layer("conv", B=3, Ci=3, Co=4, h=6, w=5, s=3, pad=1), DGRAD, (2, 3, 2, 3, 3, 3, 3), 3),
    (Layer("fc", B=5, Ci=20, Co=7), FWD, (2, 8, 3, 1, 1, 1, 1), 2),
    (Layer("fc", B=5, Ci=20, Co=7), DGRAD, (3, 4, 8, 1, 1, 1, 1), 1),
])
def test_alg1_matches_oracle(keys, L, role, part, threads):
    osk, che = keys
    part = Partition(*part)
    assert part.fits(P.n)
    g = inputs.rng(7)
    W = inputs.gaussian_fixed(g, L.w_shape())
    x = inputs.gaussian_fixed(g, L.x_shape() if role == FWD else L.y_shape())
    x0, x1 = inputs.split_shares(g, x)
    bias = inputs.uniform_zt(g, (L.Co,)) if role == FWD else None
    y0, y1, ct_in, pts, ct_out = protocol.he_linear(P, osk, L, role, part, W, x1, x0, 11, 12, bias=bias)
    c0, c1, cin, cpt, cout = che.layer_alg1(L, role, part, W, x1, x0, 11, 12, bias=bias, threads=threads)
    for i in ct_in:
        assert (cin[i] == _as_u64(ct_in, i)).all(), ("ct_in", i)
    for i in pts:
        assert (cpt[i] == _as_u64(pts, i)).all(), ("pt", i)
    for i in ct_out:
        assert (cout[i] == _as_u64(ct_out, i)).all(), ("ct_out", i)
    assert (c0 == y0.reshape(-1)).all() and (c1 == y1.reshape(-1)).all()


@pytest.mark.parametrize("L,part", [
    (Layer("conv", B=2, Ci=3, Co=4, h=6, w=5, s=3, pad=1), (2, 1, 3, 3, 3, 3, 2)),
    (Layer("fc", B=5, Ci=20, Co=7), (3, 2, 4, 1, 1, 1, 1)),
])
def test_alg2_matches_oracle(keys, L, part):
    osk, che = keys
    part = Partition(*part)
    g = inputs.rng(9)
    x0, x1 = inputs.split_shares(g, inputs.gaussian_fixed(g, L.x_shape()))
    gy0, gy1 = inputs.split_shares(g, inputs.gaussian_fixed(g, L.y_shape()))
    gw, want_tilde, want_s = protocol.he_wgrad(P, osk, L, part, gy0, gy1, x0, x1, 31, 32, 33)
    tilde, s, ct_x1, ct_gy1, ct_out = che.layer_alg2(L, part, gy0, gy1, x0, x1, 31, 32, 33, threads=2)
    want_x1 = protocol.encrypt_inputs(P, osk, L, WGRAD, part, x1, 31)
    for i, ct in want_x1.items():
        assert (ct_x1[i] == np.array(ct, dtype=object).astype(np.uint64)).all()
    want_g1 = protocol.encrypt_kernel_operand(P, osk, L, WGRAD, part, gy1, 32)
    for i, ct in want_g1.items():
        assert (ct_gy1[i] == np.array(ct, dtype=object).astype(np.uint64)).all()
    assert (s == want_s.reshape(-1)).all() and (tilde == want_tilde.reshape(-1)).all()
