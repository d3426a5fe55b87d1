"""GPU edge cases of the HE linear layer against the oracle: degenerate layer
shapes (batch 1, single channels, n_i or n_o = 1, a kernel covering the whole
input, 1x1 convolutions, the widest padding), the largest ring (N = 16384),
extreme share values (all zero, all t - 1), and the weight gradient at batch 1
(a reduction of length one)."""
import numpy as np
import pytest
import torch

from oracle import bfv, protocol
from oracle.packing import Partition
from oracle.params import BfvParams
from oracle.protocol import DGRAD, FWD, WGRAD, Layer
from paper_2403_11166_gb300 import inputs
from tests.gpu_util import to_dev, to_np
from tests.test_gpu_linear import _add, _he_layer, check_forward

pytestmark = pytest.mark.gpu
T_BITS = 41


@pytest.fixture(scope="module")
def he():
    from paper_2403_11166_gb300 import he
    return he


SHAPES = [
    ("fc_1x1x1", Layer("fc", B=1, Ci=1, Co=1), (12, 2, 54)),
    ("fc_no_1", Layer("fc", B=1, Ci=3000, Co=1), (12, 2, 54)),
    ("fc_ni_1", Layer("fc", B=5, Ci=1, Co=70), (12, 2, 54)),
    ("conv_scalar", Layer("conv", B=1, Ci=1, Co=1, h=1, w=1, s=1, pad=0), (12, 2, 54)),
    ("conv_kernel_covers_input", Layer("conv", B=2, Ci=3, Co=2, h=5, w=5, s=5, pad=0), (12, 2, 54)),
    ("conv_widest_pad_rect", Layer("conv", B=1, Ci=2, Co=3, h=7, w=4, s=3, pad=2), (12, 2, 54)),
    ("conv_1x1", Layer("conv", B=3, Ci=5, Co=4, h=6, w=5, s=1, pad=0), (13, 3, 60)),
    ("conv_n16384", Layer("conv", B=4, Ci=3, Co=4, h=16, w=16, s=3, pad=1), (14, 3, 60)),
]


@pytest.mark.parametrize("name,L,cfg", SHAPES, ids=[s[0] for s in SHAPES])
@pytest.mark.parametrize("role", [FWD, DGRAD])
def test_degenerate_shapes(he, name, L, cfg, role):
    check_forward(he, cfg, L, role, None, 40, sample_in=[], sample_pt=[], sample_out=[0],
                  with_bias=(role == FWD))


@pytest.mark.parametrize("fill", ["zero", "t_minus_1"])
def test_extreme_shares(he, fill):
    """The DO's share all zero or all t - 1 (the MO holds the rest): shares
    reconstruct the direct operator and the MO share is the oracle's."""
    cfg = (12, 2, 54)
    L = Layer("conv", B=2, Ci=3, Co=4, h=6, w=6, s=3, pad=1)
    ctx = he.Context(*cfg)
    sk = ctx.keygen(3)
    g = inputs.rng(44)
    W = inputs.gaussian_fixed(g, L.w_shape())
    x = inputs.gaussian_fixed(g, L.x_shape())
    tmask = np.uint64((1 << T_BITS) - 1)
    x1 = np.zeros(L.x_shape(), dtype=np.uint64) if fill == "zero" else np.full(L.x_shape(), tmask, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x0 = (np.asarray(x).astype(np.int64).view(np.uint64) - x1) & tmask
    plan = he.Plan(ctx, _he_layer(he, L), he.ROLE_FWD, None)
    S = plan.sizes
    ws = plan.new_ws(max(S.ws_encrypt, S.ws_forward, S.ws_decrypt))
    pt, ct_in, ct_out = plan.new_pt(S.pt), plan.new_ct(S.ct_in), plan.new_ct(S.ct_out)
    y0 = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    y1 = torch.empty_like(y0)
    he.encode_weights(ctx, plan, he.OPERAND_KERNEL, to_dev(W), pt)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, to_dev(x1), 5, ct_in, ws)
    he.he_linear_forward(ctx, plan, ct_in, pt, to_dev(x0), None, 6, ct_out, y0, ws)
    he.decrypt_to_share(ctx, sk, plan, ct_out, y1, True, ws)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    p = BfvParams(log_n=12, num_primes=2, prime_bits=54)
    assert (to_np(y0) == protocol.mo_share(p, L, FWD, 6).reshape(-1)).all()
    assert (_add(to_np(y0), to_np(y1)) == protocol.ring_op(L, FWD, W, x, T_BITS).reshape(-1)).all()


WG = [("conv_b1", Layer("conv", B=1, Ci=1, Co=1, h=3, w=3, s=3, pad=1)),
      ("conv_b1_rect", Layer("conv", B=1, Ci=2, Co=3, h=5, w=4, s=3, pad=1)),
      ("fc_b1", Layer("fc", B=1, Ci=40, Co=7)),
      ("fc_co1", Layer("fc", B=6, Ci=33, Co=1))]


@pytest.mark.parametrize("name,L", WG, ids=[w[0] for w in WG])
def test_weight_gradient_degenerate(he, name, L):
    cfg = (12, 3, 60)
    ctx = he.Context(*cfg)
    p = BfvParams(log_n=12, num_primes=3, prime_bits=60)
    sk = ctx.keygen(5)
    osk = bfv.keygen(p, 5)
    g = inputs.rng(45)
    x = inputs.gaussian_fixed(g, L.x_shape())
    gy = inputs.gaussian_fixed(g, L.y_shape())
    x0, x1 = inputs.split_shares(g, x)
    gy0, gy1 = inputs.split_shares(g, gy)
    plan = he.Plan(ctx, _he_layer(he, L), he.ROLE_WGRAD, None)
    S = plan.sizes
    ws = plan.new_ws(max(S.ws_encrypt, S.ws_backward, S.ws_decrypt))
    ct_x1, ct_g1, ct_gw = plan.new_ct(S.ct_in), plan.new_ct(S.pt), plan.new_ct(S.ct_out)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, to_dev(x1), 31, ct_x1, ws)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_KERNEL, to_dev(gy1), 32, ct_g1, ws)
    gw_mask = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    tilde = torch.empty_like(gw_mask)
    he.he_linear_backward(ctx, None, plan, None, None, ct_x1, ct_g1, to_dev(gy0), to_dev(x0), 0, 33,
                          None, None, ct_gw, gw_mask, ws)
    he.decrypt_to_share(ctx, sk, plan, ct_gw, tilde, True, ws)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    gw, want_tilde, want_s = protocol.he_wgrad(p, osk, L, Partition(*plan.part), gy0, gy1, x0, x1, 31, 32, 33)
    assert (to_np(gw_mask) == want_s.reshape(-1)).all()
    assert (to_np(tilde) == want_tilde.reshape(-1)).all()
    assert (gw == protocol.ring_op(L, WGRAD, gy, x, T_BITS)).all()
