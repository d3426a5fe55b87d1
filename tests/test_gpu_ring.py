"""GPU parity of the plaintext ring operators over Z_2^41 (Alg. 2's local terms,
the bias gradient) against the oracle's direct operators, with uniform Z_t
operands (so every sum wraps) and both addends."""
import numpy as np
import pytest
import torch

from oracle import protocol
from oracle.protocol import DGRAD, FWD, WGRAD, Layer
from paper_2403_11166_gb300 import inputs
from tests.gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu
T = 41
MASK = np.uint64((1 << T) - 1)


@pytest.fixture(scope="module")
def he():
    from paper_2403_11166_gb300 import he
    return he


def _add(*xs):
    out = np.zeros_like(np.asarray(xs[0], dtype=np.uint64))
    with np.errstate(over="ignore"):
        for x in xs:
            out = out + np.asarray(x, dtype=np.uint64)
    return out & MASK


LAYERS = [Layer("fc", B=7, Ci=33, Co=9), Layer("conv", B=3, Ci=4, Co=5, h=9, w=7, s=3, pad=1),
          Layer("conv", B=2, Ci=3, Co=2, h=6, w=6, s=3, pad=0), Layer("conv", B=64, Ci=16, Co=32, h=32, w=32, s=3, pad=1)]


@pytest.mark.parametrize("li", range(len(LAYERS)))
@pytest.mark.parametrize("role", [FWD, DGRAD, WGRAD])
def test_ring_linear(he, li, role):
    L = LAYERS[li]
    ctx = he.Context(12, 2, 54)
    kind = he.FC if L.kind == "fc" else he.CONV
    hl = he.Layer(kind, L.B, L.Ci, L.Co, L.h, L.w, L.s, L.pad)
    hrole = {FWD: he.ROLE_FWD, DGRAD: he.ROLE_DGRAD, WGRAD: he.ROLE_WGRAD}[role]
    plan = he.Plan(ctx, hl, hrole, None)
    g = inputs.rng(40 + li)
    x = inputs.uniform_zt(g, L.x_shape())
    w = inputs.uniform_zt(g, L.w_shape())
    gy = inputs.uniform_zt(g, L.y_shape())
    if role == FWD:
        kern, inp, ref = w, x, protocol.ring_op(L, FWD, w, x, T)
    elif role == DGRAD:
        kern, inp, ref = w, gy, protocol.ring_op(L, DGRAD, w, gy, T)
    else:
        kern, inp, ref = gy, x, protocol.ring_op(L, WGRAD, gy, x, T)
    a1 = inputs.uniform_zt(g, ref.shape)
    a2 = inputs.uniform_zt(g, ref.shape)
    out = torch.empty(ref.size, dtype=torch.int64, device="cuda")
    he.pencil_ring_linear(ctx, plan, to_dev(kern), to_dev(inp), None, out)
    assert (to_np(out) == ref.reshape(-1)).all()
    he.pencil_ring_linear(ctx, plan, to_dev(kern), to_dev(inp), to_dev(a1), out, addend2=to_dev(a2))
    assert (to_np(out) == _add(ref, a1, a2).reshape(-1)).all()


@pytest.mark.parametrize("li", [0, 1, 3])
def test_bias_grad(he, li):
    L = LAYERS[li]
    ctx = he.Context(12, 2, 54)
    kind = he.FC if L.kind == "fc" else he.CONV
    plan = he.Plan(ctx, he.Layer(kind, L.B, L.Ci, L.Co, L.h, L.w, L.s, L.pad), he.ROLE_FWD, None)
    gy = inputs.uniform_zt(inputs.rng(7), L.y_shape())
    out = torch.empty(L.Co, dtype=torch.int64, device="cuda")
    he.pencil_bias_grad(ctx, plan, to_dev(gy), out)
    axes = (0,) if L.kind == "fc" else (0, 2, 3)
    want = np.zeros(L.Co, dtype=np.uint64)
    with np.errstate(over="ignore"):
        want = gy.sum(axis=axes, dtype=np.uint64) & MASK
    assert (to_np(out) == want).all()
