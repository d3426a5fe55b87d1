"""Several forward steps in flight at once, as bench.py times them: each step's
encode_weights, he_linear_forward_prepare and encrypt_share on three streams,
he_linear_forward_apply and decrypt_to_share on two more, with D device buffer
sets reused every D steps under events.  Every step's shares must be
bit-identical to the same step run alone on one stream, and their sum must be
the plain ring convolution plus bias (the oracle's definition), so calls that
overlap on the GPU share no hidden state."""
import numpy as np
import pytest
import torch

from oracle import protocol
from oracle.protocol import FWD, Layer
from paper_2403_11166_gb300 import inputs
from tests.gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu
T_BITS = 41
TMASK = np.uint64((1 << T_BITS) - 1)


@pytest.fixture(scope="module")
def he():
    from paper_2403_11166_gb300 import he
    return he


def _add(a, b):
    with np.errstate(over="ignore"):
        return (np.asarray(a, dtype=np.uint64) + np.asarray(b, dtype=np.uint64)) & TMASK


@pytest.mark.parametrize("in_flight", [2, 3])
def test_steps_in_flight_equal_steps_alone(he, in_flight):
    L = Layer("conv", B=8, Ci=4, Co=4, h=8, w=8, s=3, pad=1)
    ctx = he.Context(13, 3, 60)
    sk = ctx.keygen(77)
    plan = he.Plan(ctx, he.Layer(he.CONV, L.B, L.Ci, L.Co, L.h, L.w, L.s, L.pad), he.ROLE_FWD, None)
    S = plan.sizes
    steps = 2 * in_flight + 1   # every buffer set reused at least twice
    g = inputs.rng(2024)
    data = []
    for i in range(steps):   # a different layer input, weight and bias per step
        W = inputs.gaussian_fixed(g, (L.Co, L.Ci, L.s, L.s))
        x = inputs.gaussian_fixed(g, (L.B, L.Ci, L.h, L.w))
        bias = inputs.gaussian_fixed(g, (L.Co,), frac_bits=24)
        x0, x1 = inputs.split_shares(g, x)
        data.append(dict(W=W, x=x, bias=bias, dev={"W": to_dev(W), "x0": to_dev(x0), "x1": to_dev(x1),
                                                   "bias": to_dev(bias.astype(np.uint64) & TMASK)}))

    def buffers():
        return {"pt": plan.new_pt(S.pt), "ct_in": plan.new_ct(S.ct_in), "ct_out": plan.new_ct(S.ct_out),
                "ws_mo": plan.new_ws(S.ws_forward),
                "y0": torch.empty(S.out_elems, dtype=torch.int64, device="cuda"),
                "y1": torch.empty(S.out_elems, dtype=torch.int64, device="cuda")}

    ws_enc, ws_dec = plan.new_ws(S.ws_encrypt), plan.new_ws(S.ws_decrypt)

    def one_step(i, b, st_enc, st_prep, st_ct, st_app, st_dec, ev):
        d = data[i]["dev"]
        he.encode_weights(ctx, plan, he.OPERAND_KERNEL, d["W"], b["pt"], stream=st_enc)
        ev["enc"].record(st_enc)
        he.he_linear_forward_prepare(ctx, plan, d["x0"], d["bias"], 500 + i, b["y0"], b["ws_mo"], stream=st_prep)
        ev["prep"].record(st_prep)
        he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, d["x1"], 100 + i, b["ct_in"], ws_enc, stream=st_ct)
        ev["ct"].record(st_ct)
        for e in ("enc", "prep", "ct"):
            st_app.wait_event(ev[e])
        he.he_linear_forward_apply(ctx, plan, b["ct_in"], b["pt"], b["ct_out"], b["ws_mo"], stream=st_app)
        ev["app"].record(st_app)
        st_dec.wait_event(ev["app"])
        he.decrypt_to_share(ctx, sk, plan, b["ct_out"], b["y1"], True, ws_dec, stream=st_dec)
        ev["dec"].record(st_dec)

    # each step alone, on the default stream
    s0 = torch.cuda.current_stream()
    alone = []
    b = buffers()
    ev = {k: torch.cuda.Event() for k in ("enc", "prep", "ct", "app", "dec")}
    for i in range(steps):
        one_step(i, b, s0, s0, s0, s0, s0, ev)
        torch.cuda.synchronize()
        alone.append((to_np(b["y0"]).copy(), to_np(b["y1"]).copy()))
    assert ctx.sync_status() == 0

    # the same steps with in_flight of them overlapping on five streams
    streams = [torch.cuda.Stream() for _ in range(5)]
    st_enc, st_prep, st_ct, st_app, st_dec = streams
    sets = [buffers() for _ in range(in_flight)]
    evs = [{k: torch.cuda.Event() for k in ("enc", "prep", "ct", "app", "dec")} for _ in range(in_flight)]
    used = [False] * in_flight
    out = [(torch.empty(S.out_elems, dtype=torch.int64, device="cuda"),
            torch.empty(S.out_elems, dtype=torch.int64, device="cuda")) for _ in range(steps)]
    fork = torch.cuda.Event()
    fork.record(s0)
    for st in streams:
        st.wait_event(fork)
    for i in range(steps):
        p = i % in_flight
        b, ev = sets[p], evs[p]
        if used[p]:   # step i - in_flight is done with this buffer set
            for st in (st_enc, st_prep, st_ct):
                st.wait_event(ev["app"])
            st_app.wait_event(ev["dec"])
            st_prep.wait_event(ev["dec"])   # (y0 is copied out on st_dec below)
        one_step(i, b, st_enc, st_prep, st_ct, st_app, st_dec, ev)
        with torch.cuda.stream(st_dec):   # keep this step's shares before the set is reused
            out[i][0].copy_(b["y0"])
            out[i][1].copy_(b["y1"])
        ev["dec"].record(st_dec)
        used[p] = True
    for st in streams:
        s0.wait_stream(st)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0

    for i in range(steps):
        y0, y1 = to_np(out[i][0]), to_np(out[i][1])
        assert (y0 == alone[i][0]).all() and (y1 == alone[i][1]).all(), f"step {i}"
        ref = protocol.ring_op(L, FWD, data[i]["W"], data[i]["x"], T_BITS)
        ref = _add(ref, np.asarray(data[i]["bias"]).astype(np.int64).view(np.uint64).reshape(1, -1, 1, 1))
        assert (_add(y0, y1) == ref.reshape(-1)).all(), f"step {i}"
