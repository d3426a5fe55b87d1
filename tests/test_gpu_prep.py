"""GPU: the preprocessing protocol (Alg. 3) through the C ABI -- the stacked
preprocessing evaluation (shares of every u'_i o v'_j) and the HE-free online
phase (masked operands, shares of u o v) bit-exact with the oracle, and the
online shares reconstruct u o v exactly."""
import numpy as np
import pytest
import torch

from oracle import bfv, prep as oprep, protocol
from oracle.packing import Partition
from oracle.params import BfvParams
from oracle.protocol import DGRAD, FWD, WGRAD, Layer
from paper_2403_11166_gb300 import inputs
from tests.gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu
T = 41
MASK = np.uint64((1 << T) - 1)


def _shapes(L, role):
    return {FWD: (L.w_shape(), L.x_shape()), DGRAD: (L.w_shape(), L.y_shape()),
            WGRAD: (L.y_shape(), L.x_shape()), oprep.WGRAD_REV: (L.x_shape(), L.y_shape())}[role]


@pytest.mark.parametrize("L,role,m", [
    (Layer("conv", B=2, Ci=3, Co=4, h=6, w=5, s=3, pad=1), FWD, 3),
    (Layer("conv", B=2, Ci=3, Co=4, h=6, w=5, s=3, pad=1), DGRAD, 2),
    (Layer("fc", B=3, Ci=10, Co=4), FWD, 4),
    (Layer("conv", B=2, Ci=3, Co=4, h=6, w=5, s=3, pad=1), WGRAD, 2),
    (Layer("conv", B=2, Ci=3, Co=4, h=6, w=5, s=3, pad=1), oprep.WGRAD_REV, 2),
    (Layer("fc", B=3, Ci=10, Co=4), WGRAD, 3),
    (Layer("fc", B=3, Ci=10, Co=4), FWD, 9),       # m^2 > 64: the online phase's per-j form
])
def test_prep_protocol_matches_oracle(L, role, m):
    from paper_2403_11166_gb300 import he, prep
    cfg = (13, 3, 60)
    ctx = he.Context(*cfg)
    p = BfvParams(log_n=13, num_primes=3, prime_bits=60)
    sk, osk = ctx.keygen(9), bfv.keygen(p, 9)
    g = inputs.rng(77)
    ushape, vshape = _shapes(L, role)
    u = inputs.gaussian_fixed(g, ushape) if role in (FWD, DGRAD) else inputs.uniform_zt(g, ushape)
    v = inputs.uniform_zt(g, vshape)
    um = [inputs.uniform_zt(g, ushape) for _ in range(m)]
    vm = [inputs.uniform_zt(g, vshape) for _ in range(m)]
    k = [int(a) for a in inputs.uniform_zt(g, (m,))]
    l = [int(a) for a in inputs.uniform_zt(g, (m,))]
    hrole = {FWD: he.ROLE_FWD, DGRAD: he.ROLE_DGRAD, WGRAD: he.ROLE_WGRAD, oprep.WGRAD_REV: prep.WGRAD_REV}[role]
    kind = he.FC if L.kind == "fc" else he.CONV
    pp = prep.PrepProduct(ctx, sk, he.Layer(kind, L.B, L.Ci, L.Co, L.h, L.w, L.s, L.pad), hrole, m)
    U = np.concatenate(um, axis=oprep.u_axis(role))
    V = np.concatenate(vm, axis=oprep.v_axis(role))
    pp.preprocess(to_dev(U), to_dev(V), 41, 42)
    ut, vt, z0, z1 = pp.online(to_dev(u), to_dev(v), k, l)
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0
    part = Partition(*pp.plan_s.part)
    S0, S1 = oprep.prep(p, osk, L, role, part, um, vm, 41, 42)
    assert (to_np(pp.S0) == S0.reshape(-1)).all() and (to_np(pp.S1) == S1.reshape(-1)).all()
    out, outv, oz0, oz1 = oprep.online(L, role, u, v, um, vm, S0, S1, k, l, T)
    assert (to_np(ut) == out.reshape(-1)).all() and (to_np(vt) == outv.reshape(-1)).all()
    assert (to_np(z0) == oz0.reshape(-1)).all() and (to_np(z1) == oz1.reshape(-1)).all()
    with np.errstate(over="ignore"):
        rec = (to_np(z0) + to_np(z1)) & MASK
    assert (rec == oprep.op(L, role, u, v, T).reshape(-1)).all()


def test_lincomb_rejects_bad_arguments():
    from paper_2403_11166_gb300 import he
    ctx = he.Context(12, 2, 54)
    a = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(he.PencilError) as e:
        he.pencil_lincomb(ctx, a, [1] * 65, 8, a)
    assert e.value.code == -1
    with pytest.raises(he.PencilError) as e:
        he.pencil_lincomb(ctx, a, [1], 8, a, inner=0)
    assert e.value.code == -1


@pytest.mark.parametrize("count,inner,outer,tstride,off,terms,negate,with_addend", [
    (1000, 1000, 0, 1000, 0, 8, False, False),      # contiguous terms
    (777, 64, 200, 13000, 5, 8, True, True),        # strided rows, partial last row, negated
    (70000, 16384, 65536, 16384, 3, 64, False, True),  # many rows, the maximum term count
    (5, 1, 3, 7, 2, 1, True, False),                 # one element per row
])
def test_lincomb_matches_definition(count, inner, outer, tstride, off, terms, negate, with_addend):
    """out[e] = addend[e] +/- sum_i k_i src[off + (e // inner) outer + e % inner + i tstride] mod 2^41."""
    from paper_2403_11166_gb300 import he
    ctx = he.Context(12, 2, 54)
    g = np.random.default_rng(count + terms)
    rows = -(-count // inner)
    need = off + (rows - 1) * outer + inner + (terms - 1) * tstride
    src = g.integers(0, 1 << 41, need, dtype=np.uint64)
    k = [int(x) for x in g.integers(0, 1 << 41, terms, dtype=np.uint64)]
    add = g.integers(0, 1 << 41, count, dtype=np.uint64) if with_addend else None
    out = torch.full((count,), -1, dtype=torch.int64, device="cuda")
    he.pencil_lincomb(ctx, to_dev(src), k, count, out, addend=None if add is None else to_dev(add), negate=negate,
                      src_offset=off, inner=inner, outer_stride=outer, term_stride=tstride)
    torch.cuda.synchronize()
    want = []
    for e in range(count):
        base = off + (e // inner) * outer + e % inner
        acc = sum(k[i] * int(src[base + i * tstride]) for i in range(terms))
        a = int(add[e]) if add is not None else 0
        want.append(((a - acc) if negate else (a + acc)) % (1 << 41))
    assert (to_np(out) == np.array(want, dtype=np.uint64)).all()


@pytest.mark.parametrize("count,inner,outer,t1,n1,t2,n2,off", [
    (3000, 3000, 0, 3000, 8, 24000, 8, 0),          # m x m contiguous blocks (64 scalars)
    (517, 40, 120, 40, 3, 9000, 5, 7),              # strided rows, partial last row
    (100, 100, 0, 1, 1, 100, 1, 0),                 # one term
])
def test_lincomb2_matches_definition(count, inner, outer, t1, n1, t2, n2, off):
    from paper_2403_11166_gb300 import he
    ctx = he.Context(12, 2, 54)
    g = np.random.default_rng(count + n1 * n2)
    rows = -(-count // inner)
    need = off + (rows - 1) * outer + inner + (n1 - 1) * t1 + (n2 - 1) * t2
    src = g.integers(0, 1 << 41, need, dtype=np.uint64)
    k = [int(x) for x in g.integers(0, 1 << 41, n1 * n2, dtype=np.uint64)]
    add = g.integers(0, 1 << 41, count, dtype=np.uint64)
    out = torch.full((count,), -1, dtype=torch.int64, device="cuda")
    he.pencil_lincomb2(ctx, to_dev(src), k, n1, n2, count, out, addend=to_dev(add), src_offset=off, inner=inner,
                       outer_stride=outer, term_stride=t1, term_stride2=t2)
    torch.cuda.synchronize()
    want = []
    for e in range(count):
        base = off + (e // inner) * outer + e % inner
        acc = sum(k[i2 * n1 + i] * int(src[base + i * t1 + i2 * t2]) for i2 in range(n2) for i in range(n1))
        want.append((int(add[e]) + acc) % (1 << 41))
    assert (to_np(out) == np.array(want, dtype=np.uint64)).all()
    with pytest.raises(he.PencilError):
        he.pencil_lincomb2(ctx, to_dev(src), [1] * 65, 65, 1, count, out)
    with pytest.raises(he.PencilError):
        he.pencil_lincomb2(ctx, to_dev(src), [1] * 8, 8, 0, count, out)


def test_alg4_linear_layer_with_preprocessing():
    """Alg. 4 for one conv layer: forward shares from P_Online(o, W, <X>_1) plus the
    MO's local W o <X>_0 + b reconstruct W o X + b; grad_X shares from
    P_Online((.)_x, W, <gY>_1) plus W (.)_x <gY>_0 reconstruct grad_X; grad_W from the
    two cross terms P_Online((.), <gY>_0, <X>_1), P_Online((.)_rev, <X>_0, <gY>_1)
    and both local terms <gY>_j (.) <X>_j equals grad_Y (.) X -- all exactly mod t."""
    from paper_2403_11166_gb300 import he, prep
    L = Layer("conv", B=2, Ci=3, Co=4, h=6, w=5, s=3, pad=1)
    Lh = he.Layer(he.CONV, L.B, L.Ci, L.Co, L.h, L.w, L.s, L.pad)
    m = 2
    ctx = he.Context(13, 3, 60)
    sk = ctx.keygen(3)
    g = inputs.rng(88)
    W = inputs.gaussian_fixed(g, L.w_shape())
    b = inputs.uniform_zt(g, (L.Co,))
    x, gy = inputs.gaussian_fixed(g, L.x_shape()), inputs.gaussian_fixed(g, L.y_shape())
    x0, x1 = inputs.split_shares(g, x)
    gy0, gy1 = inputs.split_shares(g, gy)

    def online(role, u, v, ushape, vshape, seed):
        pp = prep.PrepProduct(ctx, sk, Lh, role, m)
        rm = inputs.rng(seed)
        um = np.concatenate([inputs.uniform_zt(rm, ushape) for _ in range(m)],
                            axis=0 if role == he.ROLE_FWD else 1)
        vm = np.concatenate([inputs.uniform_zt(rm, vshape) for _ in range(m)],
                            axis=1 if role in (he.ROLE_WGRAD, prep.WGRAD_REV) else 0)
        pp.preprocess(to_dev(um), to_dev(vm), seed, seed + 7)
        k = [int(a) for a in inputs.uniform_zt(rm, (m,))]
        l = [int(a) for a in inputs.uniform_zt(rm, (m,))]
        _, _, z0, z1 = pp.online(to_dev(u), to_dev(v), k, l)
        return to_np(z0), to_np(z1)

    def add(*arrs):
        with np.errstate(over="ignore"):
            out = np.zeros_like(np.asarray(arrs[0], dtype=np.uint64))
            for a in arrs:
                out = out + np.asarray(a).astype(np.int64).view(np.uint64).reshape(out.shape)
            return out & MASK
    # forward
    f0, f1 = online(he.ROLE_FWD, W, x1, L.w_shape(), L.x_shape(), 100)
    local = protocol.ring_op(L, FWD, W, x0, T).reshape(-1)
    bias = np.broadcast_to(b.reshape(1, -1, 1, 1), (L.B, L.Co, L.h, L.w)).reshape(-1)
    want = add(protocol.ring_op(L, FWD, W, x, T).reshape(-1), bias)
    assert (add(f0, local, bias, f1) == want).all()
    # grad_X
    d0, d1 = online(he.ROLE_DGRAD, W, gy1, L.w_shape(), L.y_shape(), 200)
    local = protocol.ring_op(L, DGRAD, W, gy0, T).reshape(-1)
    assert (add(d0, local, d1) == protocol.ring_op(L, DGRAD, W, gy, T).reshape(-1)).all()
    # grad_W
    a0, a1 = online(he.ROLE_WGRAD, gy0, x1, L.y_shape(), L.x_shape(), 300)
    r0, r1 = online(prep.WGRAD_REV, x0, gy1, L.x_shape(), L.y_shape(), 400)
    loc0 = protocol.ring_op(L, WGRAD, gy0, x0, T).reshape(-1)
    loc1 = protocol.ring_op(L, WGRAD, gy1, x1, T).reshape(-1)
    w_hat = add(a1, r1, loc1)                         # the DO's part, sent to the MO
    gw = add(w_hat, a0, r0, loc0)                     # the MO finishes
    assert (gw == protocol.ring_op(L, WGRAD, gy, x, T).reshape(-1)).all()
    assert ctx.sync_status() == 0
