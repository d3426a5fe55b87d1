"""GPU: many uneven layers as one fixed launch sequence (pencil_batch_*):
bit-identical to the per-layer C-ABI calls on two consecutive steps (fresh
randomness per step), inside a captured CUDA graph, and a withheld input stage
makes the persistent multiply-accumulate time out with PENCIL_E_TIMEOUT (no hang)."""
import numpy as np
import pytest
import torch

from paper_2403_11166_gb300 import inputs
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu
ENC, MASK = 1000, 5000


@pytest.fixture(scope="module")
def he():
    from paper_2403_11166_gb300 import he
    return he


def _layers(he):
    return [he.Layer(he.FC, 16, 512, 10), he.Layer(he.CONV, 4, 64, 64, 8, 8, 3, 1),
            he.Layer(he.CONV, 2, 128, 256, 4, 4, 1, 0), he.Layer(he.FC, 3, 100, 33),
            he.Layer(he.CONV, 3, 5, 7, 9, 8, 3, 1)]


def _setup(he, ctx, sk, seed=0):
    layers = _layers(he)
    plans = [he.Plan(ctx, L, he.ROLE_FWD, None) for L in layers]
    batch = he.Batch(ctx, plans)
    g = inputs.rng(seed)
    data = []
    for i, (L, p) in enumerate(zip(layers, plans)):
        wshape = (L.c_out, L.c_in) if L.kind == he.FC else (L.c_out, L.c_in, L.kernel, L.kernel)
        xshape = (L.batch, L.c_in) if L.kind == he.FC else (L.batch, L.c_in, L.height, L.width)
        W = to_dev(inputs.gaussian_fixed(g, wshape))
        x0, x1 = (to_dev(a) for a in inputs.split_shares(g, inputs.gaussian_fixed(g, xshape)))
        bias = to_dev(inputs.uniform_zt(g, (L.c_out,))) if i % 2 == 0 else None
        y0 = torch.full((p.sizes.out_elems,), -1, dtype=torch.int64, device="cuda")
        y1 = torch.full_like(y0, -1)
        batch.bind(i, W, x1, x0, bias, y0, y1)
        data.append((W, x0, x1, bias, y0, y1))
    ws = torch.empty((batch.workspace_bytes + 7) // 8, dtype=torch.int64, device="cuda")
    batch.commit(sk, ws, ENC, MASK)
    return layers, plans, batch, data


def _reference(he, ctx, sk, plan, W, x0, x1, bias, enc_seed, mask_seed):
    S = plan.sizes
    ws = plan.new_ws(max(S.ws_encrypt, S.ws_forward, S.ws_decrypt))
    pt = plan.new_pt(S.pt)
    he.encode_weights(ctx, plan, he.OPERAND_KERNEL, W, pt)
    ct_in = plan.new_ct(S.ct_in)
    he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, x1, enc_seed, ct_in, ws)
    ct_out = plan.new_ct(S.ct_out)
    y0 = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
    y1 = torch.empty_like(y0)
    he.he_linear_forward(ctx, plan, ct_in, pt, x0, bias, mask_seed, ct_out, y0, ws)
    he.decrypt_to_share(ctx, sk, plan, ct_out, y1, True, ws)
    return pt, ct_in, ct_out, y0, y1


def _check_step(he, ctx, sk, plans, batch, data, step):
    for i, (p, (W, x0, x1, bias, y0, y1)) in enumerate(zip(plans, data)):
        pt, ct_in, ct_out, r0, r1 = _reference(he, ctx, sk, p, W, x0, x1, bias, ENC + i + (step << 32),
                                               MASK + i + (step << 32))
        got_in = torch.empty_like(ct_in)
        got_out = torch.empty_like(ct_out)
        got_pt = torch.empty_like(pt)
        batch.read(i, he.BATCH_CT_IN, got_in)
        batch.read(i, he.BATCH_CT_OUT, got_out)
        batch.read(i, he.BATCH_PT, got_pt)
        torch.cuda.synchronize()
        assert torch.equal(got_pt, pt), i
        assert torch.equal(got_in, ct_in), i
        assert torch.equal(got_out, ct_out), i
        assert torch.equal(y0, r0) and torch.equal(y1, r1), i


@pytest.mark.parametrize("cols", [0, 2, 4, 8])
def test_batch_equals_per_layer_calls(he, cols):
    ctx = he.Context(13, 3, 60)
    ctx.tune(he.TUNE_MAC_COLUMNS, cols)
    sk = ctx.keygen(3)
    layers, plans, batch, data = _setup(he, ctx, sk)
    for step in (0, 1):
        batch.forward()
        torch.cuda.synchronize()
        assert ctx.sync_status() == 0
        _check_step(he, ctx, sk, plans, batch, data, step)


def test_batch_flooded_equals_per_layer_calls(he):
    """Noise flooding in the batch engine: the flood stream is re-keyed per step
    like the mask, so every step equals the flooded per-layer calls."""
    ctx = he.Context(13, 3, 60)
    ctx.flooding(60)
    sk = ctx.keygen(6)
    layers, plans, batch, data = _setup(he, ctx, sk, seed=3)
    for step in (0, 1):
        batch.forward()
        torch.cuda.synchronize()
        assert ctx.sync_status() == 0
        _check_step(he, ctx, sk, plans, batch, data, step)


def test_batch_in_cuda_graph(he):
    ctx = he.Context(13, 3, 60)
    sk = ctx.keygen(4)
    layers, plans, batch, data = _setup(he, ctx, sk, seed=1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.forward(stream=s)              # warm-up outside capture (step 0)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.forward()
    batch.set_step(5)
    graph.replay()
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    _check_step(he, ctx, sk, plans, batch, data, 5)
    graph.replay()
    torch.cuda.synchronize()
    _check_step(he, ctx, sk, plans, batch, data, 6)


def test_withheld_stage_times_out(he):
    ctx = he.Context(13, 3, 60)
    sk = ctx.keygen(5)
    layers, plans, batch, data = _setup(he, ctx, sk, seed=2)
    batch.withhold(1)
    batch.commit(sk, batch._ws, ENC, MASK)
    batch.forward()
    torch.cuda.synchronize()
    assert ctx.sync_status() == -6
    batch.withhold(-1)
    batch.commit(sk, batch._ws, ENC, MASK)
    batch.set_step(0)
    batch.forward()
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    _check_step(he, ctx, sk, plans, batch, data, 0)


def test_autotuner_choice_keeps_results(he):
    """The tuner picks knobs and partitions by timing; outputs stay bit-identical
    to the per-layer calls with the chosen partitions."""
    from paper_2403_11166_gb300 import tuner
    ctx = he.Context(13, 3, 60)
    sk = ctx.keygen(6)
    layers = [he.Layer(he.FC, 8, 96, 12), he.Layer(he.CONV, 2, 8, 6, 6, 6, 3, 1)]
    best = tuner.tune_batch(ctx, sk, layers, topk=2, reps=1, radices=(4, 5), columns=(2, 8), stagings=(0, 1))
    assert best["ntt_log_radix"] in (4, 5) and best["mac_columns"] in (2, 8) and best["mac_staging"] in (0, 1)
    assert ctx.get_tune(he.TUNE_MAC_STAGING) == best["mac_staging"]
    assert ctx.get_tune(he.TUNE_MAC_COLUMNS) == best["mac_columns"]
    gb = tuner.GraphBatch(ctx, sk, layers, best["partitions"], capture=False)
    gb.batch.set_step(0)
    gb.run()
    torch.cuda.synchronize()
    for i, (p, (W, x0, x1, y0, y1)) in enumerate(zip(gb.plans, gb.bufs)):
        assert p.part == tuple(best["partitions"][i])
        r = _reference(he, ctx, sk, p, W, x0, x1, None, 1000 + i, 5000 + i)
        assert torch.equal(y0, r[3]) and torch.equal(y1, r[4])


def _shapes(he, L):
    if L.kind == he.FC:
        return (L.c_out, L.c_in), (L.batch, L.c_in), (L.batch, L.c_out)
    ho, wo = L.height + 2 * L.pad - L.kernel + 1, L.width + 2 * L.pad - L.kernel + 1
    return ((L.c_out, L.c_in, L.kernel, L.kernel), (L.batch, L.c_in, L.height, L.width),
            (L.batch, L.c_out, ho, wo))


def _mixed_setup(he, ctx, sk, seed):
    conv = he.Layer(he.CONV, 4, 16, 8, 8, 8, 3, 1)
    fc = he.Layer(he.FC, 16, 512, 10)
    entries = [(he.ROLE_FWD, conv), (he.ROLE_DGRAD, conv), (he.ROLE_WGRAD, conv),
               (he.ROLE_FWD, fc), (he.ROLE_DGRAD, fc), (he.ROLE_WGRAD, fc)]
    plans = [he.Plan(ctx, L, r, None) for r, L in entries]
    batch = he.Batch(ctx, plans)
    g = inputs.rng(seed)
    data = []
    for i, ((r, L), p) in enumerate(zip(entries, plans)):
        wshape, xshape, yshape = _shapes(he, L)
        n = p.sizes.out_elems
        y0 = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        y1 = torch.full_like(y0, -1)
        if r == he.ROLE_WGRAD:
            x0, x1 = (to_dev(a) for a in inputs.split_shares(g, inputs.gaussian_fixed(g, xshape)))
            g0, g1 = (to_dev(a) for a in inputs.split_shares(g, inputs.gaussian_fixed(g, yshape)))
            batch.bind_wgrad(i, g0, g1, x0, x1, y0, y1)
            data.append(("wgrad", g0, g1, x0, x1, y0, y1))
        else:
            W = to_dev(inputs.gaussian_fixed(g, wshape))
            v0, v1 = (to_dev(a) for a in inputs.split_shares(
                g, inputs.gaussian_fixed(g, xshape if r == he.ROLE_FWD else yshape)))
            bias = to_dev(inputs.uniform_zt(g, (L.c_out,))) if r == he.ROLE_FWD else None
            batch.bind(i, W, v1, v0, bias, y0, y1)
            data.append(("alg1", W, v0, v1, bias, y0, y1))
    ws = torch.empty((batch.workspace_bytes + 7) // 8, dtype=torch.int64, device="cuda")
    batch.commit(sk, ws, ENC, MASK)
    return plans, batch, data


def _check_mixed_step(he, ctx, sk, plans, batch, data, step):
    for i, (p, d) in enumerate(zip(plans, data)):
        enc, mask = ENC + i + (step << 32), MASK + i + (step << 32)
        got_out = p.new_ct(p.sizes.ct_out)
        batch.read(i, he.BATCH_CT_OUT, got_out)
        if d[0] == "alg1":
            _, W, v0, v1, bias, y0, y1 = d
            pt, ct_in, ct_out, r0, r1 = _reference(he, ctx, sk, p, W, v0, v1, bias, enc, mask)
            got_in = torch.empty_like(ct_in)
            batch.read(i, he.BATCH_CT_IN, got_in)
            torch.cuda.synchronize()
            assert torch.equal(got_in, ct_in), i
        else:
            _, g0, g1, x0, x1, y0, y1 = d
            S = p.sizes
            ws = p.new_ws(max(S.ws_encrypt, S.ws_backward, S.ws_decrypt))
            ct_x1, ct_g1, ct_out = p.new_ct(S.ct_in), p.new_ct(S.pt), p.new_ct(S.ct_out)
            he.encrypt_share(ctx, sk, p, he.OPERAND_INPUT, x1, enc, ct_x1, ws)
            he.encrypt_share(ctx, sk, p, he.OPERAND_KERNEL, g1, enc + (1 << 31), ct_g1, ws)
            r0 = torch.empty(S.out_elems, dtype=torch.int64, device="cuda")
            r1 = torch.empty_like(r0)
            he.he_linear_backward(ctx, None, p, None, None, ct_x1, ct_g1, g0, x0, 0, mask, None, None, ct_out, r0, ws)
            he.decrypt_to_share(ctx, sk, p, ct_out, r1, True, ws)
            got_k = torch.empty_like(ct_g1)
            batch.read(i, he.BATCH_CT_KERNEL, got_k)
            torch.cuda.synchronize()
            assert torch.equal(got_k, ct_g1), i
        torch.cuda.synchronize()
        assert ctx.sync_status() == 0
        assert torch.equal(got_out, ct_out), i
        assert torch.equal(y0, r0) and torch.equal(y1, r1), i


def test_batch_forward_and_backward_roles(he):
    """Forward, input-gradient and weight-gradient entries of a conv and an FC
    layer in one batch: bit-identical to the per-layer calls on two steps."""
    ctx = he.Context(13, 3, 60)
    sk = ctx.keygen(8)
    plans, batch, data = _mixed_setup(he, ctx, sk, seed=4)
    for step in (0, 1):
        batch.forward()
        torch.cuda.synchronize()
        assert ctx.sync_status() == 0
        _check_mixed_step(he, ctx, sk, plans, batch, data, step)


def test_batch_backward_roles_in_cuda_graph(he):
    ctx = he.Context(13, 3, 60)
    ctx.tune(he.TUNE_MAC_COLUMNS, 2)
    sk = ctx.keygen(9)
    plans, batch, data = _mixed_setup(he, ctx, sk, seed=5)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.forward(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.forward()
    batch.set_step(3)
    graph.replay()
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    _check_mixed_step(he, ctx, sk, plans, batch, data, 3)


def test_batch_bind_checks_roles(he):
    ctx = he.Context(12, 2, 54)
    L = he.Layer(he.FC, 4, 32, 8)
    pw = he.Plan(ctx, L, he.ROLE_WGRAD, None)
    pd = he.Plan(ctx, L, he.ROLE_DGRAD, None)
    batch = he.Batch(ctx, [pw, pd])
    t = torch.zeros(4096, dtype=torch.int64, device="cuda")
    with pytest.raises(he.PencilError):
        batch.bind(0, t, t, t, None, t, t)          # a WGRAD entry takes bind_wgrad
    with pytest.raises(he.PencilError):
        batch.bind(1, t, t, t, t, t, t)             # no bias on the input gradient
    with pytest.raises(he.PencilError):
        batch.bind_wgrad(1, t, t, t, t, t, t)       # a DGRAD entry takes bind
    batch.bind(1, t, t, t, None, t, t)
    batch.bind_wgrad(0, t, t, t, t, t, t)


def test_autotuner_over_forward_and_backward_roles(he):
    """tune_batch with a training step's roles: partitions chosen per (shape,
    role), and every entry of the tuned batch reconstructs its ring product."""
    import numpy as np
    from oracle import protocol
    from oracle.protocol import Layer as OLayer
    from paper_2403_11166_gb300 import tuner
    from tests.gpu_util import to_np
    ctx = he.Context(13, 3, 60)
    sk = ctx.keygen(10)
    L = he.Layer(he.CONV, 2, 4, 3, 6, 6, 3, 1)
    roles = [he.ROLE_FWD, he.ROLE_DGRAD, he.ROLE_WGRAD]
    best = tuner.tune_batch(ctx, sk, [L] * 3, topk=2, reps=1, radices=(4,), columns=(2, 4), stagings=(1,),
                            roles=roles)
    gb = tuner.GraphBatch(ctx, sk, [L] * 3, best["partitions"], capture=False, roles=roles)
    gb.batch.set_step(0)
    gb.run()
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    ol = OLayer("conv", B=2, Ci=4, Co=3, h=6, w=6, s=3, pad=1)
    tm = np.uint64((1 << 41) - 1)

    def add(*xs):
        with np.errstate(over="ignore"):
            acc = np.zeros_like(np.asarray(xs[0], dtype=np.uint64))
            for x in xs:
                acc = acc + np.asarray(x, dtype=np.uint64)
            return acc & tm
    for p, r, part in zip(gb.plans, roles, best["partitions"]):
        assert p.part == tuple(part)
    W, x0, x1, y0, y1 = gb.bufs[0]
    x = add(to_np(x0), to_np(x1)).reshape(ol.x_shape())
    assert (add(to_np(y0), to_np(y1)) == protocol.ring_op(ol, "fwd", to_np(W), x, 41).reshape(-1)).all()
    W, x0, x1, g0, g1, y0, y1 = gb.bufs[1]
    gy = add(to_np(g0), to_np(g1)).reshape(ol.y_shape())
    assert (add(to_np(y0), to_np(y1)) == protocol.ring_op(ol, "dgrad", to_np(W), gy, 41).reshape(-1)).all()
    W, x0, x1, g0, g1, y0, y1 = gb.bufs[2]
    x = add(to_np(x0), to_np(x1)).reshape(ol.x_shape())
    gy = add(to_np(g0), to_np(g1)).reshape(ol.y_shape())
    local = add(protocol.ring_op(ol, "wgrad", to_np(g1).reshape(ol.y_shape()), to_np(x1).reshape(ol.x_shape()), 41),
                protocol.ring_op(ol, "wgrad", to_np(g0).reshape(ol.y_shape()), to_np(x0).reshape(ol.x_shape()), 41))
    assert (add(to_np(y0), to_np(y1), local.reshape(-1)) == protocol.ring_op(ol, "wgrad", gy, x, 41).reshape(-1)).all()


def test_batch_entries_match_oracle(he):
    """Forward, input-gradient and weight-gradient entries of a conv and an FC
    layer in one batch, compared with the oracle directly (not through the
    per-layer calls): the last output ciphertext of every entry is bit-exact
    with Alg. 1 / Alg. 2, the MO's shares and the DO's decrypted shares equal
    the oracle's, and the shares reconstruct the ring operators."""
    from oracle import bfv, protocol
    from oracle.packing import Partition, counts
    from oracle.params import BfvParams
    from oracle.protocol import DGRAD, FWD, WGRAD
    from oracle.protocol import Layer as OLayer
    from tests.gpu_util import as_u64, to_np
    ctx = he.Context(13, 3, 60)
    sk = ctx.keygen(12)
    p = BfvParams(log_n=13, num_primes=3, prime_bits=60)
    osk = bfv.keygen(p, 12)
    layers = [(he.Layer(he.CONV, 4, 16, 8, 8, 8, 3, 1), OLayer("conv", B=4, Ci=16, Co=8, h=8, w=8, s=3, pad=1)),
              (he.Layer(he.FC, 16, 512, 10), OLayer("fc", B=16, Ci=512, Co=10))]
    roles = ((he.ROLE_FWD, FWD), (he.ROLE_DGRAD, DGRAD), (he.ROLE_WGRAD, WGRAD))
    entries = [(hr, orole, hl, ol) for hl, ol in layers for hr, orole in roles]
    plans = [he.Plan(ctx, hl, hr, None) for hr, _, hl, _ in entries]
    batch = he.Batch(ctx, plans)
    g = inputs.rng(13)
    data = []
    for i, ((hr, orole, hl, ol), pl) in enumerate(zip(entries, plans)):
        y0 = torch.full((pl.sizes.out_elems,), -1, dtype=torch.int64, device="cuda")
        y1 = torch.full_like(y0, -1)
        if hr == he.ROLE_WGRAD:
            x0, x1 = inputs.split_shares(g, inputs.gaussian_fixed(g, ol.x_shape()))
            g0, g1 = inputs.split_shares(g, inputs.gaussian_fixed(g, ol.y_shape()))
            batch.bind_wgrad(i, to_dev(g0), to_dev(g1), to_dev(x0), to_dev(x1), y0, y1)
            data.append({"x0": x0, "x1": x1, "g0": g0, "g1": g1, "y0": y0, "y1": y1})
        else:
            W = inputs.gaussian_fixed(g, ol.w_shape())
            v0, v1 = inputs.split_shares(g, inputs.gaussian_fixed(g, ol.x_shape() if hr == he.ROLE_FWD
                                                                  else ol.y_shape()))
            bias = inputs.uniform_zt(g, (ol.Co,)) if hr == he.ROLE_FWD else None
            batch.bind(i, to_dev(W), to_dev(v1), to_dev(v0), None if bias is None else to_dev(bias), y0, y1)
            data.append({"W": W, "v0": v0, "v1": v1, "bias": bias, "y0": y0, "y1": y1})
    ws = torch.empty((batch.workspace_bytes + 7) // 8, dtype=torch.int64, device="cuda")
    batch.commit(sk, ws, ENC, MASK)
    batch.forward()
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    tm = np.uint64((1 << 41) - 1)
    for i, ((hr, orole, hl, ol), pl, d) in enumerate(zip(entries, plans, data)):
        enc, mask = ENC + i, MASK + i           # step 0 seeds of entry i
        part = Partition(*pl.part)
        c = counts(protocol.geometry(ol, orole), part)
        o = c.ct_out - 1
        m, nn = divmod(o, c.NC)
        ins = [m * c.K + k for k in range(c.K)]
        kers = [k * c.NC + nn for k in range(c.K)]
        got_t = pl.new_ct(pl.sizes.ct_out)
        batch.read(i, he.BATCH_CT_OUT, got_t)
        torch.cuda.synchronize()
        got = to_np(got_t)
        y0, y1 = to_np(d["y0"]), to_np(d["y1"])
        if hr == he.ROLE_WGRAD:
            want = protocol.mo_wgrad_ct(
                p, ol, part, protocol.encrypt_inputs(p, osk, ol, WGRAD, part, d["x1"], enc, indices=ins),
                protocol.encode_kernel(p, ol, WGRAD, part, d["g0"], indices=kers),
                protocol.encrypt_kernel_operand(p, osk, ol, WGRAD, part, d["g1"], enc + (1 << 31), indices=kers),
                protocol.encode_input(p, ol, WGRAD, part, d["x0"], indices=ins), mask, o)
            assert (y0 == protocol.mo_share(p, ol, WGRAD, mask).reshape(-1)).all(), i
            gy, x = (d["g0"] + d["g1"]) & tm, (d["x0"] + d["x1"]) & tm
            local = (protocol.ring_op(ol, WGRAD, d["g0"], d["x0"], 41) + protocol.ring_op(ol, WGRAD, d["g1"], d["x1"], 41))
            assert (((y0 + y1 + local.reshape(-1)) & tm) == protocol.ring_op(ol, WGRAD, gy, x, 41).reshape(-1)).all(), i
        else:
            cts = protocol.encrypt_inputs(p, osk, ol, orole, part, d["v1"], enc, indices=ins)
            pts = protocol.encode_kernel(p, ol, orole, part, d["W"], indices=kers)
            want = protocol.mo_forward_ct(p, ol, orole, part, cts, pts, d["v0"], mask, o)
            assert (y0 == protocol.mo_share(p, ol, orole, mask, d["bias"]).reshape(-1)).all(), i
            v = (d["v0"] + d["v1"]) & tm
            ref = protocol.ring_op(ol, orole, d["W"], v, 41)
            if d["bias"] is not None:
                ref = (ref + d["bias"].reshape((1, -1) + (1,) * (ref.ndim - 2))) & tm
            assert (((y0 + y1) & tm) == ref.reshape(-1)).all(), i
        # the DO's share at the last ciphertext's outputs = the oracle's decryption of it
        dec = protocol.decrypt_outputs(p, osk, ol, orole, part, {o: want})
        from oracle.packing import decode_positions
        flats = [protocol.output_flat(ol, orole, *pos) for _, pos in decode_positions(protocol.geometry(ol, orole), part, m, nn)]
        assert (y1[flats] == dec[flats]).all(), i
        assert (got[o].reshape(-1) == as_u64(want).reshape(-1)).all(), i
