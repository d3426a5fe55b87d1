"""CPU pins of the preprocessing protocol's operand and share descriptors
(prep.layout): for every operator of Alg. 4 each strided descriptor selects
exactly the oracle's block (i, j) of the stacked shares, mask i of the stacked
operands, and block j of the stacked ring product; the block offsets are linear
in j (the online phase combines all m^2 blocks with one j-stride)."""
import numpy as np
import pytest

from oracle import prep as oprep
from oracle import protocol
from oracle.protocol import DGRAD, FWD, WGRAD, Layer


def _he():
    from paper_2403_11166_gb300 import he, prep
    return he, prep


def _pick(flat, st, count, i):
    e = np.arange(count)
    return flat[st.off + (e // st.inner) * st.outer + e % st.inner + i * st.term]


LAYERS = [Layer("conv", B=2, Ci=3, Co=4, h=6, w=5, s=3, pad=1), Layer("fc", B=3, Ci=7, Co=5)]
ROLES = [FWD, DGRAD, WGRAD, oprep.WGRAD_REV]


@pytest.mark.parametrize("L", LAYERS, ids=["conv", "fc"])
@pytest.mark.parametrize("role", ROLES)
def test_layout_selects_the_oracle_blocks(L, role):
    he, prep = _he()
    m = 3
    hrole = {FWD: he.ROLE_FWD, DGRAD: he.ROLE_DGRAD, WGRAD: he.ROLE_WGRAD, oprep.WGRAD_REV: prep.WGRAD_REV}[role]
    kind = he.FC if L.kind == "fc" else he.CONV
    lay = prep.layout(he.Layer(kind, L.B, L.Ci, L.Co, L.h, L.w, L.s, L.pad), hrole, m)
    S = oprep.stacked_layer(L, role, m)
    assert (lay.stacked.batch, lay.stacked.c_in, lay.stacked.c_out) == (S.B, S.Ci, S.Co)
    # shares of the stacked output: block (i, j) = u'_i o v'_j
    out_role = WGRAD if role == oprep.WGRAD_REV else role
    y = np.arange(int(np.prod(protocol.output_shape(S, out_role)))).reshape(protocol.output_shape(S, out_role))
    yf = y.reshape(-1)
    b0, b1 = lay.blk(0), lay.blk(1)
    for j in range(m):
        bj = lay.blk(j)
        assert (bj.off, bj.inner, bj.outer, bj.term) == (b0.off + j * (b1.off - b0.off), b0.inner, b0.outer, b0.term)
        for i in range(m):
            want = oprep.block(y, L, role, i, j).reshape(-1)
            assert want.size == lay.n_out
            assert (_pick(yf, bj, lay.n_out, i) == want).all(), (i, j)
    # masks stacked along the operator's axes
    ushape, vshape = {FWD: (L.w_shape(), L.x_shape()), DGRAD: (L.w_shape(), L.y_shape()),
                      WGRAD: (L.y_shape(), L.x_shape()), oprep.WGRAD_REV: (L.x_shape(), L.y_shape())}[role]
    um = [np.arange(int(np.prod(ushape))).reshape(ushape) + 10 ** 6 * i for i in range(m)]
    vm = [np.arange(int(np.prod(vshape))).reshape(vshape) + 10 ** 6 * i for i in range(m)]
    U = np.concatenate(um, axis=oprep.u_axis(role)).reshape(-1)
    V = np.concatenate(vm, axis=oprep.v_axis(role)).reshape(-1)
    for i in range(m):
        assert (_pick(U, lay.u_st, lay.n_u, i) == um[i].reshape(-1)).all(), i
        assert (_pick(V, lay.v_st, lay.n_v, i) == vm[i].reshape(-1)).all(), i
    # the stacked ring product u~ o v'_j (DO): block j is the product with mask j
    RL = lay.ring_all[0]
    R_layer = Layer(L.kind, B=RL.batch, Ci=RL.c_in, Co=RL.c_out, h=L.h, w=L.w, s=L.s, pad=L.pad)
    rshape = protocol.output_shape(R_layer, out_role)
    R = np.arange(int(np.prod(rshape))).reshape(rshape)
    for j in range(m):
        if role in (FWD, DGRAD):
            want = R[j * L.B:(j + 1) * L.B]                     # batch rows of mask j
        elif role == WGRAD:
            want = R[:, j * L.Ci:(j + 1) * L.Ci]                # input channels of mask j
        else:
            want = R[j * L.Co:(j + 1) * L.Co]                   # output channels of mask j
        assert (_pick(R.reshape(-1), lay.ring_blk(j), lay.n_out, 0) == want.reshape(-1)).all(), j
