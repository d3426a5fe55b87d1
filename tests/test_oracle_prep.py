"""CPU pins of the preprocessing-protocol oracle (Alg. 3): every stacked block
is its product u'_i o v'_j; the online shares reconstruct u o v exactly; with
one mask and unit scalars the protocol is the single-mask one the paper states
first.  Small N, small layers."""
import numpy as np
import pytest

from oracle import bfv, prep, protocol
from oracle.packing import Partition
from oracle.params import BfvParams
from oracle.protocol import DGRAD, FWD, WGRAD, Layer
from paper_2403_11166_gb300 import inputs

T = 41
MASK = np.uint64((1 << T) - 1)


def _add(a, b):
    with np.errstate(over="ignore"):
        return (np.asarray(a, dtype=np.uint64) + np.asarray(b, dtype=np.uint64)) & MASK


CASES = [
    (Layer("conv", B=1, Ci=2, Co=2, h=4, w=4, s=3, pad=1), FWD, 2, Partition(2, 2, 4, 4, 4, 3, 3)),
    (Layer("conv", B=1, Ci=2, Co=2, h=4, w=4, s=3, pad=1), DGRAD, 2, Partition(2, 2, 4, 4, 4, 3, 3)),
    (Layer("fc", B=2, Ci=5, Co=3), FWD, 3, Partition(6, 5, 9, 1, 1, 1, 1)),
    (Layer("conv", B=2, Ci=2, Co=2, h=4, w=4, s=3, pad=1), WGRAD, 2, None),
    (Layer("conv", B=2, Ci=2, Co=2, h=4, w=4, s=3, pad=1), prep.WGRAD_REV, 2, None),
    (Layer("fc", B=3, Ci=4, Co=3), WGRAD, 2, None),
]


def _shapes(L, role):
    """(u shape, v shape) of the operator."""
    return {FWD: (L.w_shape(), L.x_shape()), DGRAD: (L.w_shape(), L.y_shape()),
            WGRAD: (L.y_shape(), L.x_shape()), prep.WGRAD_REV: (L.x_shape(), L.y_shape())}[role]


def _part(L, role, m, n):
    """One polynomial per (batch item, channel pair): the whole output window in one tile."""
    Ls = prep.stacked_layer(L, role, m)
    g = protocol.geometry(Ls, WGRAD if role == prep.WGRAD_REV else role)
    part = Partition(1, 1, 1, g.Ho, g.Wo, g.KH, g.KW)
    assert part.fits(n)
    return part


def _operands(L, role, m, seed):
    g = inputs.rng(seed)
    ushape, vshape = _shapes(L, role)
    u = inputs.gaussian_fixed(g, ushape) if role in (FWD, DGRAD) else inputs.uniform_zt(g, ushape)
    v = inputs.uniform_zt(g, vshape)
    u_masks = [inputs.uniform_zt(g, ushape) for _ in range(m)]
    v_masks = [inputs.uniform_zt(g, vshape) for _ in range(m)]
    k = [int(a) for a in inputs.uniform_zt(g, (m,))]
    l = [int(a) for a in inputs.uniform_zt(g, (m,))]
    return u, v, u_masks, v_masks, k, l


@pytest.mark.parametrize("L,role,m,part", CASES)
def test_prep_blocks_are_the_products_and_online_reconstructs(L, role, m, part):
    p = BfvParams(log_n=10, num_primes=3, prime_bits=60)   # room for uniform Z_t masks in the product
    if part is None:
        part = _part(L, role, m, p.n)
    assert part.fits(p.n)
    sk = bfv.keygen(p, 3)
    u, v, um, vm, k, l = _operands(L, role, m, 5)
    S0, S1 = prep.prep(p, sk, L, role, part, um, vm, 11, 12)
    for i in range(m):
        for j in range(m):
            want = prep.op(L, role, um[i], vm[j], T)
            got = _add(prep.block(S0, L, role, i, j), prep.block(S1, L, role, i, j))
            assert (got == want).all(), (i, j)
    ut, vt, z0, z1 = prep.online(L, role, u, v, um, vm, S0, S1, k, l, T)
    assert (_add(z0, z1) == prep.op(L, role, u, v, T)).all()
    # the masked operands are what the parties send: u~ + sum k u' = u, v~ + sum l v' = v
    with np.errstate(over="ignore"):
        back_u = ut.copy()
        for i in range(m):
            back_u = back_u + np.uint64(k[i]) * um[i]
        back_v = vt.copy()
        for j in range(m):
            back_v = back_v + np.uint64(l[j]) * vm[j]
    assert ((back_u & MASK) == (np.asarray(u).astype(np.int64).view(np.uint64) & MASK)).all()
    assert ((back_v & MASK) == (v & MASK)).all()


def test_one_mask_is_the_single_mask_protocol():
    """m = 1, k = l = 1: <u o v>_1 = (u - u') o v' + <u' o v'>_1 and
    <u o v>_0 = u o (v - v') + <u' o v'>_0 (the paper's first, single-mask form
    applied twice)."""
    L, role, m, part = CASES[0]
    p = BfvParams(log_n=10, num_primes=3, prime_bits=60)   # room for uniform Z_t masks in the product
    sk = bfv.keygen(p, 4)
    u, v, um, vm, _, _ = _operands(L, role, 1, 6)
    S0, S1 = prep.prep(p, sk, L, role, part, um, vm, 21, 22)
    ut, vt, z0, z1 = prep.online(L, role, u, v, um, vm, S0, S1, [1], [1], T)
    with np.errstate(over="ignore"):
        du = (np.asarray(u).astype(np.int64).view(np.uint64) - um[0]) & MASK
        dv = (v - vm[0]) & MASK
    assert (ut == du).all() and (vt == dv).all()
    assert (z1 == _add(protocol.ring_op(L, role, du, vm[0], T), S1)).all()
    assert (z0 == _add(protocol.ring_op(L, role, u, dv, T), S0)).all()


def test_stacked_layer_shapes():
    L = Layer("conv", B=2, Ci=3, Co=4, h=5, w=5, s=3, pad=1)
    assert prep.stacked_layer(L, FWD, 3) == Layer("conv", B=6, Ci=3, Co=12, h=5, w=5, s=3, pad=1)
    assert prep.stacked_layer(L, DGRAD, 3) == Layer("conv", B=6, Ci=9, Co=4, h=5, w=5, s=3, pad=1)
    y = np.arange(6 * 12 * 25).reshape(6, 12, 5, 5)
    assert (prep.block(y, L, FWD, 1, 2) == y[4:6, 4:8]).all()
