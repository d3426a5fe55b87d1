"""GPU parity of the compact send form of returned ciphertexts
(compact_returned, decrypt_compact_to_share) against the oracle: c0 at the
output coefficients bit-exact, and decrypting the compact form gives the same
DO share as decrypting the whole ciphertexts, for the forward, input-gradient
and weight-gradient roles and for plan slices."""
import numpy as np
import pytest
import torch

from oracle import bfv, protocol
from oracle.packing import Partition
from oracle.params import BfvParams
from oracle.protocol import DGRAD, FWD, WGRAD, Layer
from paper_2403_11166_gb300 import inputs
from tests.gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def he():
    from paper_2403_11166_gb300 import he
    return he


def _he_layer(he, L):
    kind = he.FC if L.kind == "fc" else he.CONV
    return he.Layer(kind, L.B, L.Ci, L.Co, L.h, L.w, L.s, L.pad)


CASES = [(Layer("conv", B=2, Ci=3, Co=4, h=6, w=5, s=3, pad=1), FWD),
         (Layer("fc", B=5, Ci=70, Co=9, h=1, w=1, s=1, pad=0), FWD),
         (Layer("conv", B=2, Ci=4, Co=3, h=6, w=6, s=3, pad=1), DGRAD),
         (Layer("conv", B=2, Ci=3, Co=2, h=5, w=5, s=3, pad=1), WGRAD)]


@pytest.mark.parametrize("L,role", CASES)
def test_compact_form_matches_oracle(he, L, role):
    cfg = (12, 3, 60)
    ctx = he.Context(*cfg)
    p = BfvParams(log_n=12, num_primes=3, prime_bits=60)
    sk = ctx.keygen(8)
    osk = bfv.keygen(p, 8)
    g = inputs.rng(61)
    W = inputs.gaussian_fixed(g, L.w_shape())
    x0, x1 = inputs.split_shares(g, inputs.gaussian_fixed(g, L.x_shape()))
    gy0, gy1 = inputs.split_shares(g, inputs.gaussian_fixed(g, L.y_shape()))
    hrole = {FWD: he.ROLE_FWD, DGRAD: he.ROLE_DGRAD, WGRAD: he.ROLE_WGRAD}[role]
    plan = he.Plan(ctx, _he_layer(he, L), hrole, None)
    S = plan.sizes
    part = Partition(*plan.part)
    ws = plan.new_ws(max(S.ws_encrypt, S.ws_forward, S.ws_backward, S.ws_decrypt))
    ct_out = plan.new_ct(S.ct_out)
    y0 = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    if role in (FWD, DGRAD):
        v0, v1 = (x0, x1) if role == FWD else (gy0, gy1)
        pt, ct_in = plan.new_pt(S.pt), plan.new_ct(S.ct_in)
        he.encode_weights(ctx, plan, he.OPERAND_KERNEL, to_dev(W), pt)
        he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, to_dev(v1), 5, ct_in, ws)
        if role == FWD:
            he.he_linear_forward(ctx, plan, ct_in, pt, to_dev(v0), None, 6, ct_out, y0, ws)
        else:
            he.he_linear_backward(ctx, plan, None, ct_in, pt, None, None, to_dev(v0), None, 6, 0, ct_out, y0,
                                  None, None, ws)
        _, _, _, _, want_ct = protocol.he_linear(p, osk, L, role, part, W, v1, v0, 5, 6)
    else:
        ct_x1, ct_g1 = plan.new_ct(S.ct_in), plan.new_ct(S.pt)
        he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, to_dev(x1), 5, ct_x1, ws)
        he.encrypt_share(ctx, sk, plan, he.OPERAND_KERNEL, to_dev(gy1), 7, ct_g1, ws)
        he.he_linear_backward(ctx, None, plan, None, None, ct_x1, ct_g1, to_dev(gy0), to_dev(x0), 0, 6,
                              None, None, ct_out, y0, ws)
        from oracle.packing import counts
        c = counts(protocol.geometry(L, WGRAD), part)
        cx = protocol.encrypt_inputs(p, osk, L, WGRAD, part, x1, 5)
        cg = protocol.encrypt_kernel_operand(p, osk, L, WGRAD, part, gy1, 7)
        pg = protocol.encode_kernel(p, L, WGRAD, part, gy0)
        px = protocol.encode_input(p, L, WGRAD, part, x0)
        want_ct = {i: protocol.mo_wgrad_ct(p, L, part, cx, pg, cg, px, 6, i) for i in range(c.ct_out)}
    c0c = torch.full((3, S.out_elems), -1, dtype=torch.int64, device="cuda")
    he.compact_returned(ctx, plan, ct_out, c0c)
    y1 = torch.empty_like(y0)
    y1c = torch.empty_like(y0)
    he.decrypt_to_share(ctx, sk, plan, ct_out, y1, True, ws)
    he.decrypt_compact_to_share(ctx, sk, plan, ct_out, c0c, y1c, True, ws)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    _, want_c0c = protocol.compact_returned(p, L, role, part, want_ct)
    assert (to_np(c0c) == np.asarray(want_c0c, dtype=np.uint64)).all()
    assert torch.equal(y1, y1c)
    want_y1 = protocol.decrypt_compact(p, osk, L, role, part, {i: v[1] for i, v in want_ct.items()}, want_c0c)
    assert (to_np(y1c) == want_y1).all()


def test_compact_form_by_slices(he):
    """Slices compact and decrypt their own output rows; together they give the
    whole plan's c0c and share."""
    ctx = he.Context(12, 2, 54)
    sk = ctx.keygen(9)
    L = Layer("conv", B=6, Ci=3, Co=4, h=8, w=8, s=3, pad=1)
    plan = he.Plan(ctx, _he_layer(he, L), he.ROLE_FWD, (1, 3, 4, 8, 8, 3, 3))
    S = plan.sizes
    assert plan.rows >= 3
    g = inputs.rng(62)
    W = inputs.gaussian_fixed(g, L.w_shape())
    x0, x1 = inputs.split_shares(g, inputs.gaussian_fixed(g, L.x_shape()))
    ws = plan.new_ws(max(S.ws_encrypt, S.ws_forward, S.ws_decrypt))
    pt, ct_in, ct_out = plan.new_pt(S.pt), plan.new_ct(S.ct_in), plan.new_ct(S.ct_out)
    y0 = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    he.encode_weights(ctx, plan, he.OPERAND_KERNEL, to_dev(W), pt)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, to_dev(x1), 5, ct_in, ws)
    he.he_linear_forward(ctx, plan, ct_in, pt, to_dev(x0), None, 6, ct_out, y0, ws)
    whole = torch.full((2, S.out_elems), -1, dtype=torch.int64, device="cuda")
    he.compact_returned(ctx, plan, ct_out, whole)
    y_whole = torch.empty_like(y0)
    he.decrypt_compact_to_share(ctx, sk, plan, ct_out, whole, y_whole, True, ws)
    parts = torch.full_like(whole, -1)
    y_parts = torch.full_like(y0, -1)
    cuts = [0, 1, plan.rows // 2, plan.rows]
    for a, b in zip(cuts[:-1], cuts[1:]):
        if b > a:
            sl = plan.slice(a, b - a)
            he.compact_returned(ctx, sl, ct_out, parts)
            he.decrypt_compact_to_share(ctx, sk, sl, ct_out, parts, y_parts, True, ws)
    y_ref = torch.empty_like(y0)
    he.decrypt_to_share(ctx, sk, plan, ct_out, y_ref, True, ws)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    assert torch.equal(parts, whole)
    assert torch.equal(y_parts, y_whole) and torch.equal(y_whole, y_ref)
