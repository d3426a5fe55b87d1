"""Polynomial encodings of Appendix A (oracle; test infrastructure only).

Appendix A gives two coefficient encodings so that ONE polynomial product
W * v in Z[X]/(X^N+1) carries a whole batched linear operator:

* matrix product (Iron-style): v at x^(k n_o n_i + j), W "reversed" at
  x^(i n_i + n_i - 1 - j), result y_(k n_o n_i + i n_i + n_i - 1) = sum_j W_ij v_jk;
* 2-D convolution: index_v(b,c,i,j) = b c_o c_i h w + c h w + i w + j,
  index_W(c',c,i,j) = O + c' c_i h w - c h w - i w - j with
  O = (c_i - 1) h w + (s - 1) w + s - 1, and
  index_y(b,c',i,j) = b c_o c_i h w + O + c' c_i h w + i w + j,
  valid while B c_o c_i h w <= N.

The matrix encoding is the convolution encoding with h = w = s = 1
(c_i = n_i, c_o = n_o, b = k), so one geometry covers both.

Readings:
* (i)  the printed weight index range "i, j in [h]" is read as [s];
* (ii) h, w are the spatial sizes of the zero-padded input window;
* (iii) kernels may be rectangular (kh x kw): O = (c_i-1) h w + (kh-1) w + kw-1;
* (iv) "larger inputs or weights could be partitioned" (App. A) is read as a
  block partition: batch blocks of bb, input-channel blocks of cib, output-channel
  blocks of cob, output tiles th x tw and kernel tiles kth x ktw; input windows of
  (th + kth - 1) x (tw + ktw - 1); partial sums over channel blocks and kernel
  tiles are added in the ciphertext domain.

Operator computed (cross-correlation, as PyTorch's conv2d):
    y[b, o, i, j] = sum_{c, u, v} Wt[o, c, u, v] * V[b, c, i + u, j + v]
with V of shape (B, Ci, H, W) (already padded) and Wt of shape (Co, Ci, KH, KW).

Index order (a convention this oracle and the CUDA planner both follow):
  m = (mb * MTH + mh) * MTW + mw       over batch blocks and output tiles
  k = (kc * KTH + kh) * KTW + kw       over input-channel blocks and kernel tiles
  n = nc                               over output-channel blocks
  ct_in[m * K + k], pt[k * NC + n], ct_out[m * NC + n].
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Tuple

import numpy as np


def _cdiv(a: int, b: int) -> int:
    return -(-a // b)


@dataclass(frozen=True)
class Geometry:
    B: int
    Ci: int
    Co: int
    H: int
    W: int
    KH: int
    KW: int

    @property
    def Ho(self) -> int:
        return self.H - self.KH + 1

    @property
    def Wo(self) -> int:
        return self.W - self.KW + 1


@dataclass(frozen=True)
class Partition:
    bb: int
    cib: int
    cob: int
    th: int
    tw: int
    kth: int
    ktw: int

    def window(self) -> Tuple[int, int]:
        return self.th + self.kth - 1, self.tw + self.ktw - 1

    def fits(self, n: int) -> bool:
        h, w = self.window()
        return self.bb * self.cob * self.cib * h * w <= n


@dataclass(frozen=True)
class Counts:
    MB: int
    MTH: int
    MTW: int
    KC: int
    KTH: int
    KTW: int
    NC: int

    @property
    def M(self) -> int:
        return self.MB * self.MTH * self.MTW

    @property
    def K(self) -> int:
        return self.KC * self.KTH * self.KTW

    @property
    def ct_in(self) -> int:
        return self.M * self.K

    @property
    def pt(self) -> int:
        return self.K * self.NC

    @property
    def ct_out(self) -> int:
        return self.M * self.NC

    @property
    def products(self) -> int:
        return self.M * self.K * self.NC


def counts(g: Geometry, p: Partition) -> Counts:
    return Counts(MB=_cdiv(g.B, p.bb), MTH=_cdiv(g.Ho, p.th), MTW=_cdiv(g.Wo, p.tw),
                  KC=_cdiv(g.Ci, p.cib), KTH=_cdiv(g.KH, p.kth), KTW=_cdiv(g.KW, p.ktw),
                  NC=_cdiv(g.Co, p.cob))


def split_m(c: Counts, m: int):
    mw = m % c.MTW
    mh = (m // c.MTW) % c.MTH
    mb = m // (c.MTW * c.MTH)
    return mb, mh, mw


def split_k(c: Counts, k: int):
    kw = k % c.KTW
    kh = (k // c.KTW) % c.KTH
    kc = k // (c.KTW * c.KTH)
    return kc, kh, kw


def offset_O(p: Partition) -> int:
    h, w = p.window()
    return (p.cib - 1) * h * w + (p.kth - 1) * w + p.ktw - 1


def index_v(p: Partition, b: int, c: int, i: int, j: int) -> int:
    h, w = p.window()
    return b * p.cob * p.cib * h * w + c * h * w + i * w + j


def index_w(p: Partition, co: int, c: int, u: int, v: int) -> int:
    h, w = p.window()
    return offset_O(p) + co * p.cib * h * w - c * h * w - u * w - v


def index_y(p: Partition, b: int, co: int, i: int, j: int) -> int:
    h, w = p.window()
    return b * p.cob * p.cib * h * w + offset_O(p) + co * p.cib * h * w + i * w + j


def pack_input(V: np.ndarray, g: Geometry, p: Partition, n: int, m: int, k: int) -> List[int]:
    """pi_v of the input window feeding ct_in[m, k]."""
    assert p.fits(n)
    c = counts(g, p)
    mb, mh, mw = split_m(c, m)
    kc, kh, kw = split_k(c, k)
    h, w = p.window()
    out = [0] * n
    for b in range(p.bb):
        gb = mb * p.bb + b
        if gb >= g.B:
            continue
        for ch in range(p.cib):
            gc = kc * p.cib + ch
            if gc >= g.Ci:
                continue
            for i in range(h):
                r = mh * p.th + kh * p.kth + i
                if r >= g.H:
                    continue
                for j in range(w):
                    s = mw * p.tw + kw * p.ktw + j
                    if s >= g.W:
                        continue
                    out[index_v(p, b, ch, i, j)] = int(V[gb, gc, r, s])
    return out


def pack_weight(Wt: np.ndarray, g: Geometry, p: Partition, n: int, k: int, nn: int) -> List[int]:
    """pi_W of the kernel block feeding pt[k, nn] (signed or Z_t values, as given)."""
    assert p.fits(n)
    c = counts(g, p)
    kc, kh, kw = split_k(c, k)
    out = [0] * n
    for co in range(p.cob):
        go = nn * p.cob + co
        if go >= g.Co:
            continue
        for ch in range(p.cib):
            gc = kc * p.cib + ch
            if gc >= g.Ci:
                continue
            for u in range(p.kth):
                gu = kh * p.kth + u
                if gu >= g.KH:
                    continue
                for v in range(p.ktw):
                    gv = kw * p.ktw + v
                    if gv >= g.KW:
                        continue
                    out[index_w(p, co, ch, u, v)] = int(Wt[go, gc, gu, gv])
    return out


def decode_positions(g: Geometry, p: Partition, m: int, nn: int) -> List[Tuple[int, Tuple[int, int, int, int]]]:
    """(exponent, (b, o, i, j)) for every in-range output carried by ct_out[m, nn]."""
    c = counts(g, p)
    mb, mh, mw = split_m(c, m)
    out = []
    for b in range(p.bb):
        gb = mb * p.bb + b
        if gb >= g.B:
            continue
        for co in range(p.cob):
            go = nn * p.cob + co
            if go >= g.Co:
                continue
            for i in range(p.th):
                gi = mh * p.th + i
                if gi >= g.Ho:
                    continue
                for j in range(p.tw):
                    gj = mw * p.tw + j
                    if gj >= g.Wo:
                        continue
                    out.append((index_y(p, b, co, i, j), (gb, go, gi, gj)))
    return out


def collision_check(p: Partition, n: int) -> None:
    """Brute force over one (ct_in, pt, ct_out) block: multiply every input
    coefficient by every weight coefficient, land it at its exponent modulo
    X^N + 1, and assert that each decode position receives exactly the pairs
    of the correlation and nothing else.  Raises AssertionError otherwise."""
    assert p.fits(n)
    h, w = p.window()
    landed: Dict[int, set] = {}
    for b in range(p.bb):
        for c in range(p.cib):
            for i in range(h):
                for j in range(w):
                    ev = index_v(p, b, c, i, j)
                    for co in range(p.cob):
                        for c2 in range(p.cib):
                            for u in range(p.kth):
                                for v in range(p.ktw):
                                    e = ev + index_w(p, co, c2, u, v)
                                    assert 0 <= e < 2 * n
                                    e %= n
                                    landed.setdefault(e, set()).add((b, c, i, j, co, c2, u, v))
    for b in range(p.bb):
        for co in range(p.cob):
            for i in range(p.th):
                for j in range(p.tw):
                    e = index_y(p, b, co, i, j)
                    assert 0 <= e < n
                    want = {(b, c, i + u, j + v, co, c, u, v)
                            for c in range(p.cib) for u in range(p.kth) for v in range(p.ktw)}
                    got = landed.get(e, set())
                    assert got == want, (p, (b, co, i, j), len(got), len(want))
