"""Pins for oracle.packing: the brute-force collision checker over many block
shapes (including the matrix encoding h = w = s = 1, rectangular kernels and
the grad_W shapes), and the closed-form identities of Appendix A evaluated
through an integer polynomial product."""
import numpy as np
import pytest

from oracle import packing
from oracle.packing import Geometry, Partition
from oracle.ring import negacyclic_schoolbook

SHAPES = [
    (64, Partition(1, 8, 8, 1, 1, 1, 1)),        # FC block n_i'=8, n_o'=8, B'=1
    (64, Partition(2, 4, 8, 1, 1, 1, 1)),        # FC with batch 2
    (128, Partition(1, 2, 2, 3, 3, 3, 3)),       # conv 3x3 on a 5x5 window
    (256, Partition(2, 2, 3, 2, 3, 3, 3)),
    (256, Partition(1, 3, 2, 4, 2, 2, 3)),       # rectangular window and kernel
    (128, Partition(1, 2, 1, 3, 3, 4, 4)),       # grad_W style: large kernel, small output
    (512, Partition(1, 1, 1, 8, 8, 8, 8)),
]


@pytest.mark.parametrize("n,part", SHAPES)
def test_collision_free(n, part):
    packing.collision_check(part, n)


def test_collision_check_catches_bad_offset():
    bad = Partition(1, 2, 2, 3, 3, 3, 3)
    orig = packing.offset_O
    try:
        packing.offset_O = lambda p: orig(p) - 1
        with pytest.raises(AssertionError):
            packing.collision_check(bad, 128)
    finally:
        packing.offset_O = orig


def _correlate(Wt, V):
    B, C, H, W = V.shape
    O, _, KH, KW = Wt.shape
    out = np.zeros((B, O, H - KH + 1, W - KW + 1), dtype=object)
    for u in range(KH):
        for v in range(KW):
            out += np.einsum("bchw,oc->bohw", V[:, :, u:u + H - KH + 1, v:v + W - KW + 1].astype(object),
                             Wt[:, :, u, v].astype(object))
    return out


@pytest.mark.parametrize("g,part,n", [
    (Geometry(3, 5, 4, 1, 1, 1, 1), Partition(2, 2, 2, 1, 1, 1, 1), 64),
    (Geometry(2, 3, 2, 6, 5, 3, 3), Partition(1, 2, 2, 2, 2, 3, 3), 128),
    (Geometry(2, 2, 3, 7, 7, 5, 4), Partition(1, 1, 2, 2, 3, 3, 2), 128),
])
def test_blockwise_products_equal_correlation(g, part, n):
    """pack every block, multiply the integer polynomials (schoolbook, q huge so no
    wrap), sum over k, decode -> the direct correlation."""
    rng = np.random.default_rng(0)
    V = rng.integers(-9, 9, size=(g.B, g.Ci, g.H, g.W))
    Wt = rng.integers(-9, 9, size=(g.Co, g.Ci, g.KH, g.KW))
    c = packing.counts(g, part)
    big = (1 << 127) - 1
    want = _correlate(Wt, V)
    got = np.zeros_like(want)
    seen = set()
    for m in range(c.M):
        for nn in range(c.NC):
            acc = [0] * n
            for k in range(c.K):
                prod = negacyclic_schoolbook(packing.pack_input(V, g, part, n, m, k),
                                             packing.pack_weight(Wt, g, part, n, k, nn), big)
                acc = [a + b for a, b in zip(acc, prod)]
            for e, (b, o, i, j) in packing.decode_positions(g, part, m, nn):
                v = acc[e] % big
                got[b, o, i, j] = v - big if v > big // 2 else v
                assert (b, o, i, j) not in seen
                seen.add((b, o, i, j))
    assert len(seen) == want.size
    assert (got == want).all()


def test_matrix_encoding_closed_form():
    """Appendix A, matrix product: y_(k n_o n_i + i n_i + n_i - 1) = sum_j W_ij v_jk."""
    n_i, n_o, B, n = 4, 3, 2, 32
    rng = np.random.default_rng(1)
    Wm = rng.integers(-5, 5, size=(n_o, n_i))
    v = rng.integers(-5, 5, size=(n_i, B))
    pv = [0] * n
    pw = [0] * n
    for j in range(n_i):
        for k in range(B):
            pv[k * n_o * n_i + j] = int(v[j, k])
    for i in range(n_o):
        for j in range(n_i):
            pw[i * n_i + n_i - 1 - j] = int(Wm[i, j])
    big = (1 << 61) - 1
    y = negacyclic_schoolbook(pv, pw, big)
    for i in range(n_o):
        for k in range(B):
            val = y[k * n_o * n_i + i * n_i + n_i - 1]
            val = val - big if val > big // 2 else val
            assert val == int((Wm @ v)[i, k])
    # and the generic geometry reproduces the same coefficient placement
    part = Partition(B, n_i, n_o, 1, 1, 1, 1)
    g = Geometry(B, n_i, n_o, 1, 1, 1, 1)
    V = v.T[:, :, None, None]
    Wt = Wm[:, :, None, None]
    assert packing.pack_input(V, g, part, n, 0, 0) == pv
    assert packing.pack_weight(Wt, g, part, n, 0, 0) == pw
