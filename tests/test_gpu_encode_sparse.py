"""GPU parity of plaintext encoding for short supports.

A kernel block with few weights (one 3x3 kernel per plaintext, a 1x1 kernel,
a small FC block) packs into the first few coefficients of its polynomial;
the forward transform then skips the stages that only copy (round 0 whole and
the first j stages of round 1 for supports <= T / 2^j).  Every case here is
compared with the oracle's encoding, polynomial by polynomial, across the
thresholds of j (0 .. radix), just above T (the dense path), for both radices
and N = 4096, 8192, 16384."""
import numpy as np
import pytest

from oracle import protocol
from oracle.packing import Partition, counts
from oracle.params import BfvParams
from oracle.protocol import FWD, Layer
from paper_2403_11166_gb300 import inputs
from tests.gpu_util import as_u64, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def he():
    from paper_2403_11166_gb300 import he
    return he


def _he_layer(he, L):
    kind = he.FC if L.kind == "fc" else he.CONV
    return he.Layer(kind, L.B, L.Ci, L.Co, L.h, L.w, L.s, L.pad)


def _support(L, part, n, operand):
    """1 + the highest packed position (host restatement of Appendix A's index maps)."""
    g = protocol.geometry(L, FWD)
    p = Partition(*part)
    h, w = p.window()
    if operand == "kernel":
        O = (p.cib - 1) * h * w + (p.kth - 1) * w + p.ktw - 1
        return O + (p.cob - 1) * p.cib * h * w + 1
    return (p.bb - 1) * p.cob * p.cib * h * w + (p.cib - 1) * h * w + (h - 1) * w + w


CASES = [
    # (cfg, layer, partition, operand)
    ((13, 3, 60), Layer("conv", B=2, Ci=2, Co=2, h=32, w=32, s=3, pad=1), (1, 1, 1, 32, 32, 3, 3), "kernel"),  # 71
    ((13, 3, 60), Layer("conv", B=2, Ci=3, Co=2, h=8, w=8, s=1, pad=0), (1, 1, 1, 8, 8, 1, 1), "kernel"),      # 1
    ((13, 3, 60), Layer("fc", B=4, Ci=64, Co=16), (1, 32, 16, 1, 1, 1, 1), "kernel"),                          # 512
    ((13, 3, 60), Layer("fc", B=4, Ci=64, Co=16), (1, 16, 16, 1, 1, 1, 1), "kernel"),                          # 256
    ((13, 3, 60), Layer("fc", B=4, Ci=66, Co=16), (1, 33, 16, 1, 1, 1, 1), "kernel"),                          # 528
    ((13, 3, 60), Layer("fc", B=4, Ci=64, Co=16), (1, 8, 8, 1, 1, 1, 1), "kernel"),                            # 64
    ((13, 3, 60), Layer("fc", B=4, Ci=64, Co=16), (1, 8, 4, 1, 1, 1, 1), "kernel"),                            # 32
    ((13, 3, 60), Layer("fc", B=4, Ci=64, Co=16), (1, 64, 2, 1, 1, 1, 1), "input"),                            # 64
    ((13, 3, 60), Layer("conv", B=1, Ci=2, Co=3, h=3, w=200, s=3, pad=0), (1, 1, 1, 1, 128, 3, 3), "kernel"),  # 263
    ((12, 2, 60), Layer("conv", B=2, Ci=2, Co=2, h=16, w=16, s=3, pad=1), (1, 1, 1, 16, 16, 3, 3), "kernel"),  # 39
    ((12, 2, 60), Layer("fc", B=4, Ci=64, Co=16), (1, 16, 16, 1, 1, 1, 1), "kernel"),                          # 256
    ((14, 3, 60), Layer("conv", B=2, Ci=2, Co=2, h=32, w=32, s=3, pad=1), (1, 1, 1, 32, 32, 3, 3), "kernel"),  # 71
    ((14, 3, 60), Layer("fc", B=4, Ci=64, Co=16), (1, 32, 16, 1, 1, 1, 1), "kernel"),                          # 512
]


@pytest.mark.parametrize("radix", [4, 5])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_sparse_encode_matches_oracle(he, case, radix):
    cfg, L, part, operand = CASES[case]
    p = BfvParams(log_n=cfg[0], num_primes=cfg[1], prime_bits=cfg[2])
    ctx = he.Context(*cfg)
    ctx.tune(he.TUNE_NTT_LOG_RADIX, radix)
    assert ctx.get_tune(he.TUNE_NTT_ARITH) == 1          # the pseudo-Mersenne engine runs these primes
    plan = he.Plan(ctx, _he_layer(he, L), he.ROLE_FWD, part)
    assert plan.part == part
    g = inputs.rng(40 + case)
    c = counts(protocol.geometry(L, FWD), Partition(*part))
    sup = _support(L, part, p.n, operand)
    assert 0 < sup <= p.n
    if operand == "kernel":
        vals = inputs.gaussian_fixed(g, L.w_shape())
        pt = plan.new_pt(plan.sizes.pt)
        he.encode_weights(ctx, plan, he.OPERAND_KERNEL, to_dev(vals), pt)
        want = protocol.encode_kernel(p, L, FWD, Partition(*part), vals)
        got = to_np(pt)
        idx = range(c.pt)
    else:
        vals = inputs.gaussian_fixed(g, L.x_shape())
        pt = plan.new_pt(plan.sizes.ct_in)
        he.encode_weights(ctx, plan, he.OPERAND_INPUT, to_dev(vals), pt)
        want = protocol.encode_input(p, L, FWD, Partition(*part), vals)
        got = to_np(pt)
        idx = range(c.ct_in)
    assert ctx.sync_status() == 0
    for i in idx:
        assert (got[i].reshape(want[i].shape) == as_u64(want[i])).all(), (i, sup)
