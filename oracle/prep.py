"""Oracle of the preprocessing protocol (Alg. 3, "Preprocessing optimization"):
P(o, u, v) = (P_Prep(o), P_Online(o, u, v)) for a linear operator o of a
layer, with m masks per party.  Test infrastructure only (see oracle/__init__).

u is the MO's operand (the layer's weights W for o = the forward product and
for (.)_x = the input gradient), v the DO's operand (X, resp. grad_Y).

P_Prep: the DO draws masks v'_j, the MO masks u'_i (i, j < m); the MO evaluates
Enc(u'_i o v'_j - s_ij) homomorphically for all i, j and the DO decrypts, so
the MO holds <u'_i o v'_j>_0 = s_ij and the DO <u'_i o v'_j>_1 = u'_i o v'_j -
s_ij.  The m^2 products are ONE Alg. 1 evaluation of the "stacked" layer whose
batch is m B (v'_j at batch rows j B ..) and whose o-output channels are m
times as many (u'_i at channels i C ..), with the MO's own share of the input
zero; block (i, j) of its output (batch rows of j, channels of i) is
u'_i o v'_j.  (Reading: the paper does not say how the m^2 evaluations are
batched nor how s_ij is drawn; the s_ij here are the stacked evaluation's
per-element masks.)

P_Online (scalars k_i from the MO, l_j from the DO):
  u~ = u - sum_i k_i u'_i,  v~ = v - sum_j l_j v'_j,
  <u o v'_j>_0 = sum_i k_i <u'_i o v'_j>_0,
  <u o v'_j>_1 = u~ o v'_j + sum_i k_i <u'_i o v'_j>_1,
  <u o v>_0 = u o v~ + sum_j l_j <u o v'_j>_0,
  <u o v>_1 = sum_j l_j <u o v'_j>_1,
all over Z_t (u64 wrap-around masked to t_bits).
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from . import protocol
from .protocol import DGRAD, FWD, Layer

_U64 = np.uint64


def _mod(a, t_bits):
    return np.asarray(a).astype(np.int64).view(_U64) & _U64((1 << t_bits) - 1)


def u_axis(role: str) -> int:
    """Axis of u (the kernel) along which the u'_i are stacked: the operator's output channel."""
    if role == FWD:
        return 0          # W[o, c, ...]: output channel o
    if role == DGRAD:
        return 1          # grad_X's channel is W's input channel
    raise ValueError(role)


def stacked_layer(layer: Layer, role: str, m: int) -> Layer:
    """The layer whose single Alg. 1 evaluation gives all m^2 products u'_i o v'_j."""
    if role == FWD:
        return replace(layer, B=m * layer.B, Co=m * layer.Co)
    if role == DGRAD:
        return replace(layer, B=m * layer.B, Ci=m * layer.Ci)
    raise ValueError(role)


def out_channels(layer: Layer, role: str) -> int:
    return layer.Co if role == FWD else layer.Ci


def block(y, layer: Layer, role: str, i: int, j: int):
    """u'_i o v'_j inside a stacked output (batch rows of j, output channels of i)."""
    B, C = layer.B, out_channels(layer, role)
    return y[j * B:(j + 1) * B, i * C:(i + 1) * C]


def prep(p, sk, layer: Layer, role: str, part, u_masks, v_masks, enc_seed: int, mask_seed: int):
    """P_Prep: returns (S0, S1), the MO's and DO's shares of the stacked output."""
    m = len(u_masks)
    assert len(v_masks) == m
    Ls = stacked_layer(layer, role, m)
    U = np.concatenate([np.asarray(u) for u in u_masks], axis=u_axis(role))
    V = np.concatenate([np.asarray(v) for v in v_masks], axis=0)
    zero = np.zeros(V.shape, dtype=_U64)
    s0, s1, _, _, _ = protocol.he_linear(p, sk, Ls, role, part, U, V, zero, enc_seed, mask_seed)
    return np.asarray(s0, dtype=_U64), np.asarray(s1, dtype=_U64)


def online(layer: Layer, role: str, u, v, u_masks, v_masks, S0, S1, k, l, t_bits: int):
    """P_Online: returns (u~, v~, <u o v>_0, <u o v>_1)."""
    m = len(u_masks)
    with np.errstate(over="ignore"):
        ut = _mod(u, t_bits)
        for i in range(m):
            ut = (ut - _U64(k[i]) * _mod(u_masks[i], t_bits)) & _U64((1 << t_bits) - 1)
        vt = _mod(v, t_bits)
        for j in range(m):
            vt = (vt - _U64(l[j]) * _mod(v_masks[j], t_bits)) & _U64((1 << t_bits) - 1)
        z0 = protocol.ring_op(layer, role, u, vt, t_bits).astype(_U64)
        z1 = np.zeros_like(z0)
        for j in range(m):
            a0 = np.zeros_like(z0)
            a1 = protocol.ring_op(layer, role, ut, v_masks[j], t_bits).astype(_U64)
            for i in range(m):
                a0 = a0 + _U64(k[i]) * block(S0, layer, role, i, j)
                a1 = a1 + _U64(k[i]) * block(S1, layer, role, i, j)
            z0 = z0 + _U64(l[j]) * a0
            z1 = z1 + _U64(l[j]) * a1
        mask = _U64((1 << t_bits) - 1)
        return ut, vt, z0 & mask, z1 & mask
