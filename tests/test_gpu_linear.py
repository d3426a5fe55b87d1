"""GPU parity of the HE linear layer (through the C ABI) against the oracle:
raw ciphertexts / plaintexts bit-exact on the same seeds and partition, shares
bit-exact, and reconstruction = the direct ring operator.  Covers the FC and
conv workloads at full size (FC 784->100 B=32 N=4096; conv 3x3 16->16 32x32
B=64 N=8192) plus small ragged cases of the grad_X and grad_W roles."""
import numpy as np
import pytest
import torch

from oracle import bfv, protocol
from oracle.packing import Partition
from oracle.params import BfvParams
from oracle.protocol import DGRAD, FWD, WGRAD, Layer
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


def gpu_forward(he, ctx, sk, L, role, part, kernel, x1, x0, bias, enc_seed, mask_seed):
    plan = he.Plan(ctx, _he_layer(he, L), role, part)
    S = plan.sizes
    pt = plan.new_pt(S.pt)
    he.encode_weights(ctx, plan, he.OPERAND_KERNEL, to_dev(kernel), pt)
    ws = plan.new_ws(max(S.ws_encrypt, S.ws_forward, S.ws_decrypt))
    ct_in = plan.new_ct(S.ct_in)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, to_dev(x1), enc_seed, ct_in, ws)
    ct_out = plan.new_ct(S.ct_out)
    y0 = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    y1 = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    if role == he.ROLE_FWD:
        he.he_linear_forward(ctx, plan, ct_in, pt, to_dev(x0), None if bias is None else to_dev(bias), mask_seed,
                             ct_out, y0, ws)
    else:
        he.he_linear_backward(ctx, plan, None, ct_in, pt, None, None, to_dev(x0), None, mask_seed, 0,
                              ct_out, y0, None, None, ws)
    he.decrypt_to_share(ctx, sk, plan, ct_out, y1, True, ws)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    return plan, to_np(pt), to_np(ct_in), to_np(ct_out), to_np(y0), to_np(y1)


def check_forward(he, cfg, L, role, part, seed, sample_in, sample_pt, sample_out, with_bias):
    ctx = he.Context(*cfg)
    p = BfvParams(log_n=cfg[0], num_primes=cfg[1], prime_bits=cfg[2])
    sk = ctx.keygen(seed + 1)
    osk = bfv.keygen(p, seed + 1)
    g = inputs.rng(seed)
    W = inputs.gaussian_fixed(g, L.w_shape())
    if role == FWD:
        x = inputs.gaussian_fixed(g, L.x_shape())
        bias = inputs.gaussian_fixed(g, (L.Co,), frac_bits=24) if with_bias else None
    else:
        x = inputs.gaussian_fixed(g, L.y_shape())
        bias = None
    x0, x1 = inputs.split_shares(g, x)
    enc_seed, mask_seed = 1000 + seed, 2000 + seed
    he_role = he.ROLE_FWD if role == FWD else he.ROLE_DGRAD
    plan, pt, ct_in, ct_out, y0, y1 = gpu_forward(he, ctx, sk, L, he_role, part, W, x1, x0, bias,
                                                  enc_seed, mask_seed)
    opart = Partition(*plan.part)
    if part is not None:
        assert plan.part == tuple(part)
    from oracle.packing import counts
    c = counts(protocol.geometry(L, role), opart)
    K, NC = c.K, c.NC
    assert (plan.sizes.ct_in, plan.sizes.pt, plan.sizes.ct_out) == (c.ct_in, c.pt, c.ct_out)
    # raw ciphertexts and plaintexts
    ins = sorted(set([0, c.ct_in - 1] + list(sample_in)))
    want_in = protocol.encrypt_inputs(p, osk, L, role, opart, x1, enc_seed, indices=ins)
    for i in ins:
        assert (ct_in[i] == as_u64(want_in[i])).all(), ("ct_in", i)
    pts_idx = sorted(set([0, c.pt - 1] + list(sample_pt)))
    want_pt = protocol.encode_kernel(p, L, role, opart, W, indices=pts_idx)
    for i in pts_idx:
        assert (pt[i] == as_u64(want_pt[i])).all(), ("pt", i)
    for o in sorted(set([c.ct_out - 1] + list(sample_out))):
        m, nn = divmod(o, NC)
        need_in = [m * K + k for k in range(K)]
        need_pt = [k * NC + nn for k in range(K)]
        cts = protocol.encrypt_inputs(p, osk, L, role, opart, x1, enc_seed, indices=need_in)
        pts = protocol.encode_kernel(p, L, role, opart, W, indices=need_pt)
        want = protocol.mo_forward_ct(p, L, role, opart, cts, pts, x0, mask_seed, o)
        assert (ct_out[o] == as_u64(want)).all(), ("ct_out", o)
        # decryption of that ciphertext by the oracle lands in y1
        dec = protocol.decrypt_outputs(p, osk, L, role, opart, {o: want})
        from oracle.packing import decode_positions
        for e, (b, oc, i, j) in decode_positions(protocol.geometry(L, role), opart, m, nn):
            flat = protocol.output_flat(L, role, b, oc, i, j)
            assert y1[flat] == dec[flat]
    # shares: MO share exactly the oracle's, reconstruction = direct operator (+ bias)
    want_y0 = protocol.mo_share(p, L, role, mask_seed, bias).reshape(-1)
    assert (y0 == want_y0).all()
    if role == FWD:
        ref = protocol.ring_op(L, FWD, W, x, T_BITS)
        if bias is not None:
            ref = _add(ref, np.asarray(bias).astype(np.int64).view(np.uint64).reshape((1, -1) + (1,) * (ref.ndim - 2)))
    else:
        ref = protocol.ring_op(L, DGRAD, W, x, T_BITS)
    assert (_add(y0, y1) == ref.reshape(-1)).all()
    return plan


def test_fc_784_100_b32_n4096(he):
    L = Layer("fc", B=32, Ci=784, Co=100)
    check_forward(he, (12, 2, 54), L, FWD, (1, 128, 32, 1, 1, 1, 1), 1,
                  sample_in=[6, 13, 100], sample_pt=[3, 27], sample_out=[0, 5], with_bias=True)


def test_fc_784_100_planner(he):
    """Planner-chosen partition: shares and reconstruction still exact."""
    L = Layer("fc", B=32, Ci=784, Co=100)
    check_forward(he, (12, 2, 54), L, FWD, None, 2, sample_in=[], sample_pt=[], sample_out=[0], with_bias=True)


def test_conv_16_16_32x32_b64_n8192(he):
    L = Layer("conv", B=64, Ci=16, Co=16, h=32, w=32, s=3, pad=1)
    check_forward(he, (13, 3, 60), L, FWD, (1, 2, 3, 32, 32, 3, 3), 3,
                  sample_in=[9], sample_pt=[5], sample_out=[7], with_bias=False)


def test_conv_16_16_benched_partition(he):
    """The headline layer at the partition bench.py times (the planner's choice
    with default knobs: 7 samples per batch block, so the last block holds one
    sample): raw ciphertexts of the first and last blocks, output ciphertexts
    of the first, a middle and the ragged last batch block, every decoded
    element, the MO share and the reconstruction, all against the oracle."""
    import bench
    Lb = bench.LAYER
    L = Layer("conv", B=Lb["batch"], Ci=Lb["c_in"], Co=Lb["c_out"], h=Lb["h"], w=Lb["w"], s=Lb["s"], pad=Lb["pad"])
    plan = check_forward(he, (bench.LOG_N, bench.L, bench.PRIME_BITS), L, FWD, None, 4,
                         sample_in=[17, 144, 150], sample_pt=[255], sample_out=[0, 77, 144, 150], with_bias=True)
    assert plan.part == (7, 1, 1, 32, 32, 3, 3)
    assert (plan.sizes.ct_in, plan.sizes.pt, plan.sizes.ct_out, plan.sizes.products) == (160, 256, 160, 2560)


@pytest.mark.parametrize("L,part,cfg", [
    (Layer("conv", B=2, Ci=3, Co=4, h=6, w=5, s=3, pad=1), (1, 2, 2, 4, 3, 3, 3), (12, 2, 54)),
    (Layer("conv", B=3, Ci=2, Co=3, h=5, w=5, s=3, pad=0), (2, 1, 2, 2, 3, 3, 3), (13, 3, 60)),
    (Layer("fc", B=5, Ci=20, Co=7), (2, 3, 8, 1, 1, 1, 1), (12, 2, 54)),
])
def test_dgrad_small(he, L, part, cfg):
    # grad_X role: the shares are grad_Y's, the kernel operand is the layer's weights
    assert Partition(*part).fits(1 << cfg[0])
    check_forward(he, cfg, L, DGRAD, part, 11, sample_in=[1], sample_pt=[1], sample_out=[0, 1], with_bias=False)


@pytest.mark.parametrize("L,part,knobs", [
    (Layer("conv", B=2, Ci=3, Co=4, h=6, w=5, s=3, pad=1), (2, 1, 3, 3, 3, 3, 2), None),
    (Layer("fc", B=5, Ci=20, Co=7), (3, 2, 4, 1, 1, 1, 1), None),
    (Layer("conv", B=2, Ci=3, Co=4, h=6, w=5, s=3, pad=1), (2, 1, 3, 3, 3, 3, 2), (8, 1)),
    (Layer("fc", B=5, Ci=20, Co=7), (3, 2, 4, 1, 1, 1, 1), (4, 1)),
    (Layer("fc", B=5, Ci=20, Co=7), (3, 2, 4, 1, 1, 1, 1), (0, 0)),
])
def test_wgrad_small(he, L, part, knobs):
    cfg = (12, 3, 60)
    ctx = he.Context(*cfg)
    if knobs is not None:   # (MAC columns, staging): the other multiply-accumulate forms of Alg. 2
        ctx.tune(he.TUNE_MAC_COLUMNS, knobs[0])
        ctx.tune(he.TUNE_MAC_STAGING, knobs[1])
    p = BfvParams(log_n=cfg[0], num_primes=cfg[1], prime_bits=cfg[2])
    sk = ctx.keygen(5)
    osk = bfv.keygen(p, 5)
    g = inputs.rng(21)
    x = inputs.gaussian_fixed(g, L.x_shape())
    gy = inputs.gaussian_fixed(g, L.y_shape())
    x0, x1 = inputs.split_shares(g, x)
    gy0, gy1 = inputs.split_shares(g, gy)
    plan = he.Plan(ctx, _he_layer(he, L), he.ROLE_WGRAD, part)
    S = plan.sizes
    ws = plan.new_ws(max(S.ws_encrypt, S.ws_backward, S.ws_decrypt))
    ct_x1 = plan.new_ct(S.ct_in)
    ct_gy1 = plan.new_ct(S.pt)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, to_dev(x1), 31, ct_x1, ws)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_KERNEL, to_dev(gy1), 32, ct_gy1, ws)
    ct_gw = plan.new_ct(S.ct_out)
    gw_mask = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    tilde = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    he.he_linear_backward(ctx, None, plan, None, None, ct_x1, ct_gy1, to_dev(gy0), to_dev(x0), 0, 33,
                          None, None, ct_gw, gw_mask, ws)
    he.decrypt_to_share(ctx, sk, plan, ct_gw, tilde, True, ws)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    opart = Partition(*part)
    gw, want_tilde, want_s = protocol.he_wgrad(p, osk, L, opart, gy0, gy1, x0, x1, 31, 32, 33)
    # raw operands
    want_x1 = protocol.encrypt_inputs(p, osk, L, WGRAD, opart, x1, 31)
    for i, ct in want_x1.items():
        assert (to_np(ct_x1)[i] == as_u64(ct)).all()
    want_gy1 = protocol.encrypt_kernel_operand(p, osk, L, WGRAD, opart, gy1, 32)
    for i, ct in want_gy1.items():
        assert (to_np(ct_gy1)[i] == as_u64(ct)).all()
    assert (to_np(gw_mask) == want_s.reshape(-1)).all()
    assert (to_np(tilde) == want_tilde.reshape(-1)).all()
    # Alg. 2 reconstruction with the two local terms gives grad_W exactly
    local = _add(protocol.ring_op(L, WGRAD, gy1, x1, T_BITS), protocol.ring_op(L, WGRAD, gy0, x0, T_BITS))
    assert (_add(_add(to_np(tilde), to_np(gw_mask)), local.reshape(-1)) == gw.reshape(-1)).all()
    assert (gw == protocol.ring_op(L, WGRAD, gy, x, T_BITS)).all()
    # ... and the same reconstruction on the GPU: DO adds its local term to the
    # decrypted value (step 4), MO adds the mask and its own local term (step 6)
    tilde_do = torch.empty_like(tilde)
    he.pencil_ring_linear(ctx, plan, to_dev(gy1), to_dev(x1), tilde, tilde_do)
    gw_dev = torch.empty_like(tilde)
    he.pencil_ring_linear(ctx, plan, to_dev(gy0), to_dev(x0), tilde_do, gw_dev, addend2=gw_mask)
    assert (to_np(gw_dev) == gw.reshape(-1)).all()


def test_noise_check_flags_corrupted_ciphertext(he):
    cfg = (12, 2, 54)
    ctx = he.Context(*cfg)
    sk = ctx.keygen(3)
    L = Layer("fc", B=4, Ci=16, Co=8)
    plan = he.Plan(ctx, _he_layer(he, L), he.ROLE_FWD, (1, 16, 8, 1, 1, 1, 1))
    S = plan.sizes
    g = inputs.rng(4)
    W = inputs.gaussian_fixed(g, L.w_shape())
    x0, x1 = inputs.split_shares(g, inputs.gaussian_fixed(g, L.x_shape()))
    pt = plan.new_pt(S.pt)
    he.encode_weights(ctx, plan, he.OPERAND_KERNEL, to_dev(W), pt)
    ws = plan.new_ws(max(S.ws_encrypt, S.ws_forward, S.ws_decrypt))
    ct_in = plan.new_ct(S.ct_in)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, to_dev(x1), 1, ct_in, ws)
    ct_out = plan.new_ct(S.ct_out)
    y0 = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    y1 = torch.empty_like(y0)
    he.he_linear_forward(ctx, plan, ct_in, pt, to_dev(x0), None, 2, ct_out, y0, ws)
    he.decrypt_to_share(ctx, sk, plan, ct_out, y1, True, ws)
    assert ctx.sync_status() == 0
    q0 = ctx.primes()[0][0]
    bad = to_np(ct_out).copy()
    bad[1, 0, 0, 5] = (bad[1, 0, 0, 5] + np.uint64(q0 // 3)) % np.uint64(q0)
    he.decrypt_to_share(ctx, sk, plan, to_dev(bad), y1, True, ws)
    assert ctx.sync_status() == -5
    assert ctx.sync_status() == 0


def test_host_validation(he):
    ctx = he.Context(12, 2, 54)
    L = he.Layer(he.FC, 4, 16, 8)
    with pytest.raises(he.PencilError) as e:
        he.Plan(ctx, L, he.ROLE_FWD, (1, 16, 8, 2, 1, 1, 1))   # th > Ho
    assert e.value.code == -4
    with pytest.raises(he.PencilError) as e:
        he.Plan(ctx, he.Layer(he.FC, 4, 64, 64), he.ROLE_FWD, (2, 64, 64, 1, 1, 1, 1))   # > N
    assert e.value.code == -4
    plan = he.Plan(ctx, L, he.ROLE_FWD, (1, 16, 8, 1, 1, 1, 1))
    sk = ctx.keygen(1)
    small = plan.new_ws(8)
    with pytest.raises(he.PencilError) as e:
        he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, torch.zeros(64, dtype=torch.int64, device="cuda"), 1,
                         plan.new_ct(plan.sizes.ct_in), small)
    assert e.value.code == -4
    wplan = he.Plan(ctx, L, he.ROLE_WGRAD, None)
    with pytest.raises(he.PencilError) as e:
        he.he_linear_forward(ctx, wplan, plan.new_ct(1), plan.new_pt(1), torch.zeros(64, dtype=torch.int64,
                             device="cuda"), None, 1, plan.new_ct(1), torch.zeros(64, dtype=torch.int64,
                             device="cuda"), plan.new_ws(1 << 20))
    assert e.value.code == -1


@pytest.mark.parametrize("radix,cols,staging", [(4, 2, 0), (5, 4, 0), (4, 8, 0), (5, 8, 0), (5, 0, 0), (4, 0, 0),
                                                (4, 2, 1), (5, 4, 1), (4, 8, 1)])
def test_tuning_knobs_do_not_change_results(he, radix, cols, staging):
    """Every NTT radix / MAC column setting gives bit-identical ciphertexts and shares
    (the default setting is checked against the oracle above)."""
    cfg = (13, 3, 60)
    L = Layer("conv", B=3, Ci=5, Co=7, h=9, w=8, s=3, pad=1)
    part = (1, 2, 3, 5, 4, 3, 3)
    outs = []
    for setting in (None, (radix, cols, staging)):
        ctx = he.Context(*cfg)
        if setting:
            ctx.tune(he.TUNE_NTT_LOG_RADIX, setting[0])
            ctx.tune(he.TUNE_MAC_COLUMNS, setting[1])
            ctx.tune(he.TUNE_MAC_STAGING, setting[2])
            assert ctx.get_tune(he.TUNE_MAC_COLUMNS) == setting[1]
            assert ctx.get_tune(he.TUNE_MAC_STAGING) == setting[2]
        sk = ctx.keygen(5)
        g = inputs.rng(8)
        W = inputs.gaussian_fixed(g, L.w_shape())
        x0, x1 = inputs.split_shares(g, inputs.gaussian_fixed(g, L.x_shape()))
        outs.append(gpu_forward(he, ctx, sk, L, he.ROLE_FWD, part, W, x1, x0, None, 3, 4)[1:])
    for a, b in zip(*outs):
        assert (a == b).all()


@pytest.mark.parametrize("cfg,cols,staging", [((12, 2, 54), None, 0), ((13, 3, 60), 4, 0), ((13, 3, 60), 0, 0),
                                              ((13, 3, 60), 8, 1)])
def test_prepare_apply_equals_forward(he, cfg, cols, staging):
    """he_linear_forward_prepare on one stream, encrypt on another, then
    he_linear_forward_apply: ciphertexts and shares bit-identical to he_linear_forward
    (generic, split and shared-memory staged multiply-accumulate)."""
    L = Layer("conv", B=3, Ci=5, Co=7, h=9, w=8, s=3, pad=1)
    part = (1, 2, 3, 5, 4, 3, 3)
    ctx = he.Context(*cfg)
    if cols is not None:
        ctx.tune(he.TUNE_MAC_COLUMNS, cols)
    ctx.tune(he.TUNE_MAC_STAGING, staging)
    sk = ctx.keygen(5)
    g = inputs.rng(8)
    W = inputs.gaussian_fixed(g, L.w_shape())
    x0, x1 = inputs.split_shares(g, inputs.gaussian_fixed(g, L.x_shape()))
    bias = inputs.uniform_zt(g, (L.Co,))
    _, _, _, ct_ref, y0_ref, y1_ref = gpu_forward(he, ctx, sk, L, he.ROLE_FWD, part, W, x1, x0, bias, 3, 4)
    plan = he.Plan(ctx, _he_layer(he, L), he.ROLE_FWD, part)
    S = plan.sizes
    ws_mo = plan.new_ws(S.ws_forward)
    ws_do = plan.new_ws(max(S.ws_encrypt, S.ws_decrypt))
    pt, ct_in, ct_out = plan.new_pt(S.pt), plan.new_ct(S.ct_in), plan.new_ct(S.ct_out)
    y0 = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    y1 = torch.empty_like(y0)
    Wd, x0d, x1d, bd = to_dev(W), to_dev(x0), to_dev(x1), to_dev(bias)
    mo, do = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    he.encode_weights(ctx, plan, he.OPERAND_KERNEL, Wd, pt, stream=mo)
    he.he_linear_forward_prepare(ctx, plan, x0d, bd, 4, y0, ws_mo, stream=mo)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, x1d, 3, ct_in, ws_do, stream=do)
    do.wait_stream(mo)
    he.he_linear_forward_apply(ctx, plan, ct_in, pt, ct_out, ws_mo, stream=do)
    he.decrypt_to_share(ctx, sk, plan, ct_out, y1, True, ws_do, stream=do)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    assert (to_np(ct_out) == ct_ref).all()
    assert (to_np(y0) == y0_ref).all() and (to_np(y1) == y1_ref).all()
    # the prepared workspace is only read: a second apply gives the same ciphertexts
    ct2 = plan.new_ct(S.ct_out)
    he.he_linear_forward_apply(ctx, plan, ct_in, pt, ct2, ws_mo)
    torch.cuda.synchronize()
    assert (to_np(ct2) == ct_ref).all()


def test_split_calls_validate(he):
    ctx = he.Context(12, 2, 54)
    L = Layer("fc", B=2, Ci=10, Co=3)
    plan = he.Plan(ctx, _he_layer(he, L), he.ROLE_FWD, None)
    S = plan.sizes
    small = plan.new_ws(max(1, S.ws_forward // 2))
    x0 = torch.zeros(L.B * L.Ci, dtype=torch.int64, device="cuda")
    y0 = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    with pytest.raises(he.PencilError) as e:
        he.he_linear_forward_prepare(ctx, plan, x0, None, 1, y0, small)
    assert e.value.code == -4
    with pytest.raises(he.PencilError) as e:
        he.he_linear_forward_apply(ctx, plan, None, plan.new_pt(S.pt), plan.new_ct(S.ct_out),
                                   plan.new_ws(S.ws_forward))
    assert e.value.code == -1


@pytest.mark.parametrize("role,cfg,chunks", [("fwd", (13, 3, 60), [(0, 1), (1, 2), (3, None)]),
                                             ("fwd", (12, 2, 54), [(0, 2), (2, None)]),
                                             ("dgrad", (13, 3, 60), [(0, 3), (3, None)])])
def test_slices_stream_equals_whole(he, role, cfg, chunks):
    """A layer streamed through the protocol slice by slice (encrypt / apply /
    decrypt of disjoint output-row ranges on two alternating streams) gives the
    whole-plan ciphertexts and shares bit for bit."""
    L = Layer("conv", B=7, Ci=5, Co=6, h=9, w=8, s=3, pad=1)
    part = (2, 2, 3, 5, 4, 3, 3)
    ctx = he.Context(*cfg)
    sk = ctx.keygen(5)
    g = inputs.rng(41)
    W = inputs.gaussian_fixed(g, L.w_shape())
    xs = inputs.gaussian_fixed(g, L.x_shape() if role == "fwd" else L.y_shape())
    x0, x1 = inputs.split_shares(g, xs)
    hrole = he.ROLE_FWD if role == "fwd" else he.ROLE_DGRAD
    plan = he.Plan(ctx, _he_layer(he, L), hrole, part)
    S = plan.sizes
    M = plan.rows
    assert M >= 4 and S.ct_in % M == 0 and S.ct_out % M == 0
    Wd, x0d, x1d = to_dev(W), to_dev(x0), to_dev(x1)

    def buffers():   # encryption and decryption of different slices overlap: one workspace each
        return (plan.new_pt(S.pt), plan.new_ct(S.ct_in), plan.new_ct(S.ct_out),
                torch.empty(S.out_elems, dtype=torch.int64, device="cuda"),
                torch.empty(S.out_elems, dtype=torch.int64, device="cuda"),
                plan.new_ws(S.ws_forward), plan.new_ws(S.ws_encrypt), plan.new_ws(S.ws_decrypt))
    # whole plan
    pt, ct_in, ct_out, y0, y1, ws_mo, ws_enc, ws_dec = buffers()
    he.encode_weights(ctx, plan, he.OPERAND_KERNEL, Wd, pt)
    he.he_linear_forward_prepare(ctx, plan, x0d, None, 4, y0, ws_mo)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, x1d, 3, ct_in, ws_enc)
    he.he_linear_forward_apply(ctx, plan, ct_in, pt, ct_out, ws_mo)
    he.decrypt_to_share(ctx, sk, plan, ct_out, y1, True, ws_dec)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    want = [to_np(t) for t in (ct_in, ct_out, y0, y1)]
    # streamed by slices
    pt, ct_in, ct_out, y0, y1, ws_mo, ws_enc, ws_dec = buffers()
    he.encode_weights(ctx, plan, he.OPERAND_KERNEL, Wd, pt)
    he.he_linear_forward_prepare(ctx, plan, x0d, None, 4, y0, ws_mo)
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    slices = [plan.slice(a, (M - a) if c is None else c) for a, c in chunks]
    for i, sl in enumerate(slices):
        st = streams[i % 2]
        he.encrypt_share(ctx, sk, sl, he.OPERAND_INPUT, x1d, 3, ct_in, ws_enc, stream=st)
        he.he_linear_forward_apply(ctx, sl, ct_in, pt, ct_out, ws_mo, stream=st)
        he.decrypt_to_share(ctx, sk, sl, ct_out, y1, True, ws_dec, stream=st)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    for a, b in zip(want, (to_np(t) for t in (ct_in, ct_out, y0, y1))):
        assert (a == b).all()


def test_slice_validation(he):
    ctx = he.Context(12, 2, 54)
    L = Layer("conv", B=7, Ci=5, Co=6, h=9, w=8, s=3, pad=1)
    plan = he.Plan(ctx, _he_layer(he, L), he.ROLE_FWD, (2, 2, 3, 5, 4, 3, 3))
    M = plan.rows
    for a, c, code in [(0, 0, -2), (-1, 2, -2), (M - 1, 2, -2), (M, 1, -2)]:
        with pytest.raises(he.PencilError) as e:
            plan.slice(a, c)
        assert e.value.code == code
    sl = plan.slice(1, 2)
    with pytest.raises(he.PencilError) as e:
        sl.slice(0, 1)
    assert e.value.code == -1
    sk = ctx.keygen(1)
    S = plan.sizes
    with pytest.raises(he.PencilError) as e:   # the kernel operand is not sliced
        he.encrypt_share(ctx, sk, sl, he.OPERAND_KERNEL, torch.zeros(6 * 5 * 9, dtype=torch.int64, device="cuda"), 1,
                         plan.new_ct(S.pt), plan.new_ws(S.ws_encrypt))
    assert e.value.code == -1
    pw = he.Plan(ctx, _he_layer(he, L), he.ROLE_WGRAD, None)
    with pytest.raises(he.PencilError) as e:
        pw.slice(0, 1)
    assert e.value.code == -1


# ---------------------------------------------------------------- the paper's own parameter set
# N = 8192, three 60-bit primes, t = 2^59, f = 25 (Sec. 6 training parameters).
T59 = 59


@pytest.mark.parametrize("role", [FWD, DGRAD, WGRAD])
def test_paper_parameter_set_t59_f25(he, role):
    cfg = (13, 3, 60)
    L = Layer("conv", B=3, Ci=4, Co=5, h=7, w=6, s=3, pad=1)
    ctx = he.Context(*cfg, t_bits=T59)
    p = BfvParams(log_n=13, num_primes=3, prime_bits=60, t_bits=T59)
    sk = ctx.keygen(7)
    osk = bfv.keygen(p, 7)
    g = inputs.rng(59)
    W = inputs.gaussian_fixed(g, L.w_shape(), frac_bits=25)
    x = inputs.gaussian_fixed(g, L.x_shape(), frac_bits=25)
    gy = inputs.gaussian_fixed(g, L.y_shape(), frac_bits=25)
    x0, x1 = inputs.split_shares(g, x, t_bits=T59)
    gy0, gy1 = inputs.split_shares(g, gy, t_bits=T59)
    mask = np.uint64((1 << T59) - 1)
    hrole = {FWD: he.ROLE_FWD, DGRAD: he.ROLE_DGRAD, WGRAD: he.ROLE_WGRAD}[role]
    plan = he.Plan(ctx, _he_layer(he, L), hrole, None)
    S = plan.sizes
    opart = Partition(*plan.part)
    ws = plan.new_ws(max(S.ws_encrypt, S.ws_forward, S.ws_backward, S.ws_decrypt))
    if role in (FWD, DGRAD):
        v0, v1 = (x0, x1) if role == FWD else (gy0, gy1)
        pt = plan.new_pt(S.pt)
        he.encode_weights(ctx, plan, he.OPERAND_KERNEL, to_dev(W), pt)
        ct_in, ct_out = plan.new_ct(S.ct_in), plan.new_ct(S.ct_out)
        he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, to_dev(v1), 5, ct_in, ws)
        y0 = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
        y1 = torch.empty_like(y0)
        if role == FWD:
            he.he_linear_forward(ctx, plan, ct_in, pt, to_dev(v0), None, 6, ct_out, y0, ws)
        else:
            he.he_linear_backward(ctx, plan, None, ct_in, pt, None, None, to_dev(v0), None, 6, 0, ct_out, y0, None,
                                  None, ws)
        he.decrypt_to_share(ctx, sk, plan, ct_out, y1, True, ws)
        torch.cuda.synchronize()
        assert ctx.sync_status() == 0
        oy0, oy1, _, _, oct_out = protocol.he_linear(p, osk, L, role, opart, W, v1, v0, 5, 6)
        assert (to_np(y0) == np.asarray(oy0, dtype=np.uint64).reshape(-1)).all()
        assert (to_np(y1) == np.asarray(oy1, dtype=np.uint64).reshape(-1)).all()
        o = S.ct_out - 1
        assert (to_np(ct_out)[o] == as_u64(oct_out[o])).all()
        ref = protocol.ring_op(L, role, W, x if role == FWD else gy, T59).reshape(-1)
        with np.errstate(over="ignore"):
            assert (((to_np(y0) + to_np(y1)) & mask) == ref).all()
    else:
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
        gw, want_tilde, want_s = protocol.he_wgrad(p, osk, L, opart, gy0, gy1, x0, x1, 31, 32, 33)
        assert (to_np(gw_mask) == want_s.reshape(-1)).all()
        assert (to_np(tilde) == want_tilde.reshape(-1)).all()
        assert (gw == protocol.ring_op(L, WGRAD, gy, x, T59)).all()


@pytest.mark.parametrize("role", [FWD, WGRAD])
def test_noise_flooding_matches_oracle(he, role):
    """pencil_ctx_flooding: returned ciphertexts are the oracle's flooded ones bit
    for bit, decrypted shares are unchanged, and the noise check still passes."""
    cfg = (13, 3, 60)
    L = Layer("conv", B=2, Ci=3, Co=4, h=6, w=5, s=3, pad=1)
    p = BfvParams(log_n=13, num_primes=3, prime_bits=60)
    osk = bfv.keygen(p, 4)
    g = inputs.rng(31)
    W = inputs.gaussian_fixed(g, L.w_shape())
    x0, x1 = inputs.split_shares(g, inputs.gaussian_fixed(g, L.x_shape()))
    gy0, gy1 = inputs.split_shares(g, inputs.gaussian_fixed(g, L.y_shape()))
    outs = []
    for bits in (0, 62):
        ctx = he.Context(*cfg)
        ctx.flooding(bits)
        sk = ctx.keygen(4)
        hrole = he.ROLE_FWD if role == FWD else he.ROLE_WGRAD
        plan = he.Plan(ctx, _he_layer(he, L), hrole, None)
        S = plan.sizes
        ws = plan.new_ws(max(S.ws_encrypt, S.ws_forward, S.ws_backward, S.ws_decrypt))
        y1 = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
        y0 = torch.empty_like(y1)
        ct_out = plan.new_ct(S.ct_out)
        if role == FWD:
            pt, ct_in = plan.new_pt(S.pt), plan.new_ct(S.ct_in)
            he.encode_weights(ctx, plan, he.OPERAND_KERNEL, to_dev(W), pt)
            he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, to_dev(x1), 5, ct_in, ws)
            he.he_linear_forward(ctx, plan, ct_in, pt, to_dev(x0), None, 6, ct_out, y0, ws)
        else:
            ct_x1, ct_g1 = plan.new_ct(S.ct_in), plan.new_ct(S.pt)
            he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, to_dev(x1), 5, ct_x1, ws)
            he.encrypt_share(ctx, sk, plan, he.OPERAND_KERNEL, to_dev(gy1), 7, ct_g1, ws)
            he.he_linear_backward(ctx, None, plan, None, None, ct_x1, ct_g1, to_dev(gy0), to_dev(x0), 0, 6,
                                  None, None, ct_out, y0, ws)
        he.decrypt_to_share(ctx, sk, plan, ct_out, y1, True, ws)
        torch.cuda.synchronize()
        assert ctx.sync_status() == 0
        outs.append((plan, to_np(ct_out), to_np(y0), to_np(y1)))
    (plan, ct0, a0, a1), (_, ct1, b0, b1) = outs
    assert (a0 == b0).all() and (a1 == b1).all()
    assert not (ct0 == ct1).all()
    part = Partition(*plan.part)
    o = ct1.shape[0] - 1
    if role == FWD:
        want = protocol.he_linear(p, osk, L, FWD, part, W, x1, x0, 5, 6, flood_bits=62)[4][o]
    else:
        from oracle.packing import counts
        c = counts(protocol.geometry(L, WGRAD), part)
        m, nn = divmod(o, c.NC)
        cts_x = protocol.encrypt_inputs(p, osk, L, WGRAD, part, x1, 5, indices=[m * c.K + k for k in range(c.K)])
        cts_g = protocol.encrypt_kernel_operand(p, osk, L, WGRAD, part, gy1, 7,
                                                indices=[k * c.NC + nn for k in range(c.K)])
        pg = protocol.encode_kernel(p, L, WGRAD, part, gy0, indices=[k * c.NC + nn for k in range(c.K)])
        px = protocol.encode_input(p, L, WGRAD, part, x0, indices=[m * c.K + k for k in range(c.K)])
        want = protocol.mo_wgrad_ct(p, L, part, cts_x, pg, cts_g, px, 6, o, flood_bits=62)
    assert (ct1[o] == as_u64(want)).all()
