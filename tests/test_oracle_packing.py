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


def test_appendix_a_exponents_golden():
    """The oracle's encodings put every entry at the exponent App. A's formulas
    give, evaluated by hand in tests/golden/appendix_a_packing.txt (matrix
    product as the 1 x 1 case of the convolution geometry)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "appendix_a_packing.txt")
    section, part = None, None
    checked = 0
    for line in open(path):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "mat":
            n_o, n_i, B = (int(x) for x in f[1:])
            section, part = "mat", Partition(B, n_i, n_o, 1, 1, 1, 1)
            continue
        if f[0] == "conv":
            B, c_o, c_i, h, w, s = (int(x) for x in f[1:])
            section, part = "conv", Partition(B, c_i, c_o, h - s + 1, w - s + 1, s, s)
            assert part.window() == (h, w)
            continue
        idx, want = [int(x) for x in f[1:-1]], int(f[-1])
        if section == "mat":
            if f[0] == "v":      # v_jk
                got = packing.index_v(part, idx[1], idx[0], 0, 0)
            elif f[0] == "W":    # W_ij
                got = packing.index_w(part, idx[0], idx[1], 0, 0)
            else:                # y_ik
                got = packing.index_y(part, idx[1], idx[0], 0, 0)
        else:
            fn = {"v": packing.index_v, "W": packing.index_w, "y": packing.index_y}[f[0]]
            got = fn(part, *idx)
        assert got == want, line
        checked += 1
    assert checked == 31
