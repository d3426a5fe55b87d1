"""GPU parity at the paper's single-layer shapes (Table V; batch 64, N = 8192,
three 60-bit primes, t = 2^41), with the planner's partitions, as the bench
times them: FC 256->100, 512->10, 2048->1001; conv 64->64 16x16 k5, 3->64
56x56 k3, 64->3 56x56 k3 (padding k // 2).  For each layer and role (forward
and input gradient of Alg. 1, weight gradient of Alg. 2): the reconstruction
equals the direct ring operator (every element for FC, sampled elements
including both corners for conv), and the last output ciphertext, whose blocks
are the ragged ones, is bit-exact with the oracle's Alg. 1 / Alg. 2 evaluation."""
import numpy as np
import pytest
import torch

from oracle import bfv, protocol, ring
from oracle.packing import Partition, counts
from oracle.params import BfvParams
from oracle.protocol import DGRAD, FWD, WGRAD, Layer
from paper_2403_11166_gb300 import inputs
from tests.gpu_util import as_u64, to_dev, to_np

pytestmark = pytest.mark.gpu
CFG = (13, 3, 60)
T_BITS = 41
TMASK = np.uint64((1 << T_BITS) - 1)
B = 64
LAYERS = [("fc", 256, 100, 1, 1), ("fc", 512, 10, 1, 1), ("fc", 2048, 1001, 1, 1),
          ("conv", 64, 64, 16, 5), ("conv", 3, 64, 56, 3), ("conv", 64, 3, 56, 3)]


def _layer(kind, ci, co, hw, ks):
    if kind == "fc":
        return Layer("fc", B=B, Ci=ci, Co=co)
    return Layer("conv", B=B, Ci=ci, Co=co, h=hw, w=hw, s=ks, pad=ks // 2)


def _he_layer(he, L):
    if L.kind == "fc":
        return he.Layer(he.FC, L.B, L.Ci, L.Co)
    return he.Layer(he.CONV, L.B, L.Ci, L.Co, L.h, L.w, L.s, L.pad)


def _add(*arrs):
    with np.errstate(over="ignore"):
        acc = np.zeros_like(np.asarray(arrs[0], dtype=np.uint64))
        for a in arrs:
            acc = acc + np.asarray(a, dtype=np.uint64)
    return acc & TMASK


def _sample_idx(shape, count, seed):
    r = np.random.default_rng(seed)
    idx = [tuple(int(r.integers(d)) for d in shape) for _ in range(count)]
    return idx + [(0,) * len(shape), tuple(d - 1 for d in shape)]


def _flat(shape, idx):
    return [int(np.ravel_multi_index(i, shape)) for i in idx]


@pytest.fixture(scope="module")
def env():
    from paper_2403_11166_gb300 import he
    ctx = he.Context(*CFG)
    p = BfvParams(log_n=CFG[0], num_primes=CFG[1], prime_bits=CFG[2])
    return he, ctx, ctx.keygen(41), p, bfv.keygen(p, 41)


@pytest.mark.parametrize("spec", LAYERS, ids=lambda s: f"{s[0]}{s[1]}-{s[2]}" + (f"-{s[3]}k{s[4]}" if s[0] == "conv" else ""))
@pytest.mark.parametrize("role", [FWD, DGRAD])
def test_table5_alg1_roles(env, spec, role):
    he, ctx, sk, p, osk = env
    L = _layer(*spec)
    g = inputs.rng(100 + 10 * LAYERS.index(spec) + (role == DGRAD))
    W = inputs.gaussian_fixed(g, L.w_shape())
    v = inputs.gaussian_fixed(g, L.x_shape() if role == FWD else L.y_shape())
    v0, v1 = inputs.split_shares(g, v)
    enc_seed, mask_seed = 71, 72
    plan = he.Plan(ctx, _he_layer(he, L), he.ROLE_FWD if role == FWD else he.ROLE_DGRAD, None)
    S = plan.sizes
    pt = plan.new_pt(S.pt)
    he.encode_weights(ctx, plan, he.OPERAND_KERNEL, to_dev(W), pt)
    ws = plan.new_ws(max(S.ws_encrypt, S.ws_forward, S.ws_decrypt))
    ct_in = plan.new_ct(S.ct_in)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, to_dev(v1), enc_seed, ct_in, ws)
    ct_out = plan.new_ct(S.ct_out)
    y0 = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    y1 = torch.empty_like(y0)
    if role == FWD:
        he.he_linear_forward(ctx, plan, ct_in, pt, to_dev(v0), None, mask_seed, ct_out, y0, ws)
    else:
        he.he_linear_backward(ctx, plan, None, ct_in, pt, None, None, to_dev(v0), None, mask_seed, 0,
                              ct_out, y0, None, None, ws)
    he.decrypt_to_share(ctx, sk, plan, ct_out, y1, True, ws)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    rec = _add(to_np(y0), to_np(y1))
    shape = protocol.output_shape(L, role)
    if L.kind == "fc":
        assert (rec == protocol.ring_op(L, role, W, v, T_BITS).reshape(-1)).all()
    else:
        idx = _sample_idx(shape, 40, 3)
        fn = ring.ring_conv2d_at if role == FWD else ring.ring_conv2d_dgrad_at
        assert [int(rec[f]) for f in _flat(shape, idx)] == fn(W, v, L.pad, T_BITS, idx)
    # the last output ciphertext through the oracle's Alg. 1, bit-exact
    part = Partition(*plan.part)
    c = counts(protocol.geometry(L, role), part)
    assert (S.ct_in, S.pt, S.ct_out) == (c.ct_in, c.pt, c.ct_out)
    o = c.ct_out - 1
    m, nn = divmod(o, c.NC)
    cts = protocol.encrypt_inputs(p, osk, L, role, part, v1, enc_seed, indices=[m * c.K + k for k in range(c.K)])
    pts = protocol.encode_kernel(p, L, role, part, W, indices=[k * c.NC + nn for k in range(c.K)])
    want = protocol.mo_forward_ct(p, L, role, part, cts, pts, v0, mask_seed, o)
    assert (to_np(ct_out)[o] == as_u64(want)).all()


@pytest.mark.parametrize("spec", LAYERS, ids=lambda s: f"{s[0]}{s[1]}-{s[2]}" + (f"-{s[3]}k{s[4]}" if s[0] == "conv" else ""))
def test_table5_alg2_weight_gradient(env, spec):
    he, ctx, sk, p, osk = env
    L = _layer(*spec)
    g = inputs.rng(200 + 10 * LAYERS.index(spec))
    x = inputs.gaussian_fixed(g, L.x_shape())
    gy = inputs.gaussian_fixed(g, L.y_shape())
    x0, x1 = inputs.split_shares(g, x)
    gy0, gy1 = inputs.split_shares(g, gy)
    plan = he.Plan(ctx, _he_layer(he, L), he.ROLE_WGRAD, None)
    S = plan.sizes
    ws = plan.new_ws(max(S.ws_encrypt, S.ws_backward, S.ws_decrypt))
    ct_x1 = plan.new_ct(S.ct_in)
    ct_gy1 = plan.new_ct(S.pt)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, to_dev(x1), 81, ct_x1, ws)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_KERNEL, to_dev(gy1), 82, ct_gy1, ws)
    ct_gw = plan.new_ct(S.ct_out)
    gw_mask = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    tilde = torch.empty_like(gw_mask)
    he.he_linear_backward(ctx, None, plan, None, None, ct_x1, ct_gy1, to_dev(gy0), to_dev(x0), 0, 83,
                          None, None, ct_gw, gw_mask, ws)
    he.decrypt_to_share(ctx, sk, plan, ct_gw, tilde, True, ws)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    cross = _add(to_np(tilde), to_np(gw_mask))
    shape = protocol.output_shape(L, WGRAD)
    if L.kind == "fc":
        local = _add(ring.ring_matmul_wgrad(gy0, x0, T_BITS), ring.ring_matmul_wgrad(gy1, x1, T_BITS))
        assert (_add(cross, local.reshape(-1)) == ring.ring_matmul_wgrad(gy, x, T_BITS).reshape(-1)).all()
    else:
        idx = _sample_idx(shape, 30, 5)
        fl = _flat(shape, idx)
        at = lambda a, b: ring.ring_conv2d_wgrad_at(a, b, L.pad, L.s, T_BITS, idx)
        got = [int(v) for v in _add(cross[fl], at(gy0, x0), at(gy1, x1))]
        assert got == at(gy, x)
    part = Partition(*plan.part)
    c = counts(protocol.geometry(L, WGRAD), part)
    o = c.ct_out - 1
    m, nn = divmod(o, c.NC)
    ins = [m * c.K + k for k in range(c.K)]
    kers = [k * c.NC + nn for k in range(c.K)]
    want = protocol.mo_wgrad_ct(p, L, part,
                                protocol.encrypt_inputs(p, osk, L, WGRAD, part, x1, 81, indices=ins),
                                protocol.encode_kernel(p, L, WGRAD, part, gy0, indices=kers),
                                protocol.encrypt_kernel_operand(p, osk, L, WGRAD, part, gy1, 82, indices=kers),
                                protocol.encode_input(p, L, WGRAD, part, x0, indices=ins), 83, o)
    assert (to_np(ct_gw)[o] == as_u64(want)).all()
