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
from oracle.protocol import DGRAD, FWD, Layer
from paper_2403_11166_gb300 import inputs
from tests.gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu
T = 41
MASK = np.uint64((1 << T) - 1)


@pytest.mark.parametrize("L,role,m", [
    (Layer("conv", B=2, Ci=3, Co=4, h=6, w=5, s=3, pad=1), FWD, 3),
    (Layer("conv", B=2, Ci=3, Co=4, h=6, w=5, s=3, pad=1), DGRAD, 2),
    (Layer("fc", B=3, Ci=10, Co=4), FWD, 4),
])
def test_prep_protocol_matches_oracle(L, role, m):
    from paper_2403_11166_gb300 import he, prep
    cfg = (13, 3, 60)
    ctx = he.Context(*cfg)
    p = BfvParams(log_n=13, num_primes=3, prime_bits=60)
    sk, osk = ctx.keygen(9), bfv.keygen(p, 9)
    g = inputs.rng(77)
    u = inputs.gaussian_fixed(g, L.w_shape())
    vshape = L.x_shape() if role == FWD else L.y_shape()
    v = inputs.uniform_zt(g, vshape)
    um = [inputs.uniform_zt(g, L.w_shape()) for _ in range(m)]
    vm = [inputs.uniform_zt(g, vshape) for _ in range(m)]
    k = [int(a) for a in inputs.uniform_zt(g, (m,))]
    l = [int(a) for a in inputs.uniform_zt(g, (m,))]
    hrole = he.ROLE_FWD if role == FWD else he.ROLE_DGRAD
    kind = he.FC if L.kind == "fc" else he.CONV
    pp = prep.PrepProduct(ctx, sk, he.Layer(kind, L.B, L.Ci, L.Co, L.h, L.w, L.s, L.pad), hrole, m)
    U = np.concatenate(um, axis=oprep.u_axis(role))
    V = np.concatenate(vm, axis=0)
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
    assert (rec == protocol.ring_op(L, role, u, v, T).reshape(-1)).all()


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
