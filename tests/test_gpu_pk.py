"""GPU parity of public-key BFV (pencil_pk_keygen, encrypt_share_pk) against
the oracle: ciphertexts bit-exact for both operand kinds, and Alg. 1 / Alg. 2
run on public-key-encrypted shares reconstruct the ring products exactly."""
import numpy as np
import pytest
import torch

from oracle import bfv, protocol
from oracle.packing import Partition
from oracle.params import BfvParams
from oracle.protocol import FWD, WGRAD, Layer
from paper_2403_11166_gb300 import inputs
from tests.gpu_util import as_u64, to_dev, to_np

pytestmark = pytest.mark.gpu
T_BITS = 41
TMASK = np.uint64((1 << T_BITS) - 1)


@pytest.fixture(scope="module")
def he():
    from paper_2403_11166_gb300 import he
    return he


def _he_layer(he, L):
    kind = he.FC if L.kind == "fc" else he.CONV
    return he.Layer(kind, L.B, L.Ci, L.Co, L.h, L.w, L.s, L.pad)


def _add(a, b):
    with np.errstate(over="ignore"):
        return (np.asarray(a, dtype=np.uint64) + np.asarray(b, dtype=np.uint64)) & TMASK


@pytest.mark.parametrize("cfg", [(12, 2, 54), (13, 3, 60)])
def test_pk_encrypt_and_forward(he, cfg):
    L = Layer("conv", B=3, Ci=5, Co=4, h=9, w=7, s=3, pad=1)
    ctx = he.Context(*cfg)
    p = BfvParams(log_n=cfg[0], num_primes=cfg[1], prime_bits=cfg[2])
    sk = ctx.keygen(5)
    pk = ctx.pk_keygen(sk, 11)
    osk = bfv.keygen(p, 5)
    opk = bfv.pk_keygen(p, osk, 11)
    g = inputs.rng(41)
    W = inputs.gaussian_fixed(g, L.w_shape())
    x = inputs.gaussian_fixed(g, L.x_shape())
    x0, x1 = inputs.split_shares(g, x)
    plan = he.Plan(ctx, _he_layer(he, L), he.ROLE_FWD, None)
    S = plan.sizes
    assert S.ws_encrypt_pk > S.ws_encrypt
    ws = plan.new_ws(max(S.ws_encrypt_pk, S.ws_forward, S.ws_decrypt))
    pt, ct_in, ct_out = plan.new_pt(S.pt), plan.new_ct(S.ct_in), plan.new_ct(S.ct_out)
    he.encode_weights(ctx, plan, he.OPERAND_KERNEL, to_dev(W), pt)
    he.encrypt_share_pk(ctx, pk, plan, he.OPERAND_INPUT, to_dev(x1), 21, ct_in, ws)
    y0 = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    y1 = torch.empty_like(y0)
    he.he_linear_forward(ctx, plan, ct_in, pt, to_dev(x0), None, 22, ct_out, y0, ws)
    he.decrypt_to_share(ctx, sk, plan, ct_out, y1, True, ws)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    part = Partition(*plan.part)
    idx = sorted({0, S.ct_in // 2, S.ct_in - 1})
    want = protocol.encrypt_inputs(p, osk, L, FWD, part, x1, 21, indices=idx, pk=opk)
    got = to_np(ct_in)
    for i in idx:
        assert (got[i] == as_u64(want[i])).all(), i
    ref = protocol.ring_op(L, FWD, W, x, T_BITS).reshape(-1)
    assert (_add(to_np(y0), to_np(y1)) == ref).all()


def test_pk_kernel_operand_and_wgrad(he):
    """Alg. 2 with both DO operands public-key encrypted (Enc(<X>_1) at input
    positions, Enc(<gY>_1) at kernel positions)."""
    cfg = (12, 3, 60)
    L = Layer("conv", B=2, Ci=3, Co=4, h=6, w=6, s=3, pad=1)
    ctx = he.Context(*cfg)
    p = BfvParams(log_n=cfg[0], num_primes=cfg[1], prime_bits=cfg[2])
    sk = ctx.keygen(6)
    pk = ctx.pk_keygen(sk, 12)
    osk = bfv.keygen(p, 6)
    opk = bfv.pk_keygen(p, osk, 12)
    g = inputs.rng(42)
    x = inputs.gaussian_fixed(g, L.x_shape())
    gy = inputs.gaussian_fixed(g, L.y_shape())
    x0, x1 = inputs.split_shares(g, x)
    gy0, gy1 = inputs.split_shares(g, gy)
    plan = he.Plan(ctx, _he_layer(he, L), he.ROLE_WGRAD, None)
    S = plan.sizes
    ws = plan.new_ws(max(S.ws_encrypt_pk, S.ws_backward, S.ws_decrypt))
    ct_x1, ct_g1, ct_gw = plan.new_ct(S.ct_in), plan.new_ct(S.pt), plan.new_ct(S.ct_out)
    he.encrypt_share_pk(ctx, pk, plan, he.OPERAND_INPUT, to_dev(x1), 31, ct_x1, ws)
    he.encrypt_share_pk(ctx, pk, plan, he.OPERAND_KERNEL, to_dev(gy1), 32, ct_g1, ws)
    gw_mask = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    tilde = torch.empty_like(gw_mask)
    he.he_linear_backward(ctx, None, plan, None, None, ct_x1, ct_g1, to_dev(gy0), to_dev(x0), 0, 33,
                          None, None, ct_gw, gw_mask, ws)
    he.decrypt_to_share(ctx, sk, plan, ct_gw, tilde, True, ws)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    part = Partition(*plan.part)
    want = protocol.encrypt_kernel_operand(p, osk, L, WGRAD, part, gy1, 32, indices=[S.pt - 1], pk=opk)
    assert (to_np(ct_g1)[S.pt - 1] == as_u64(want[S.pt - 1])).all()
    local = _add(protocol.ring_op(L, WGRAD, gy1, x1, T_BITS), protocol.ring_op(L, WGRAD, gy0, x0, T_BITS))
    gw = _add(_add(to_np(tilde), to_np(gw_mask)), local.reshape(-1))
    assert (gw == protocol.ring_op(L, WGRAD, gy, x, T_BITS).reshape(-1)).all()


def test_pk_validation(he):
    ctx = he.Context(12, 2, 54)
    other = he.Context(12, 2, 54)
    sk = ctx.keygen(1)
    with pytest.raises(he.PencilError):
        other.pk_keygen(sk, 1)                   # key of another context
    pk = ctx.pk_keygen(sk, 1)
    L = Layer("fc", B=2, Ci=8, Co=3, h=1, w=1, s=1, pad=0)
    plan = he.Plan(ctx, _he_layer(he, L), he.ROLE_FWD, None)
    S = plan.sizes
    x = torch.zeros(2 * 8, dtype=torch.int64, device="cuda")
    ct = plan.new_ct(S.ct_in)
    small = plan.new_ws(S.ws_encrypt_pk - 256)
    with pytest.raises(he.PencilError):
        he.encrypt_share_pk(ctx, pk, plan, he.OPERAND_INPUT, x, 1, ct, small)
