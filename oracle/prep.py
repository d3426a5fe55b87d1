"""Oracle of the preprocessing protocol (Alg. 3, "Preprocessing optimization"):
P(o, u, v) = (P_Prep(o), P_Online(o, u, v)) for a linear operator o of a
layer, with m masks per party.  Test infrastructure only (see oracle/__init__).

u is the MO's operand, v the DO's operand, for the four operators of Alg. 4:
  FWD   (o)       u = W,           v = X,           u o v = W o X;
  DGRAD ((.)_x)   u = W,           v = grad_Y,      u o v = W (.)_x grad_Y;
  WGRAD ((.))     u = <grad_Y>_0,  v = <X>_1,       u o v = u (.) v  (grad_W-shaped);
  WGRAD_REV       u = <X>_0,       v = <grad_Y>_1,  u o v = v (.) u.

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
from .protocol import DGRAD, FWD, WGRAD, Layer

WGRAD_REV = "wgrad_rev"

_U64 = np.uint64


def _mod(a, t_bits):
    return np.asarray(a).astype(np.int64).view(_U64) & _U64((1 << t_bits) - 1)


def u_axis(role: str) -> int:
    """Axis of u along which the u'_i are stacked."""
    if role == FWD:
        return 0          # W[o, c, ...]: output channel o
    if role in (DGRAD, WGRAD, WGRAD_REV):
        return 1          # W's input channel / grad_Y's channel / X's channel
    raise ValueError(role)


def v_axis(role: str) -> int:
    """Axis of v along which the v'_j are stacked (the batch, or the channel for grad_W)."""
    return 1 if role in (WGRAD, WGRAD_REV) else 0


def stacked_layer(layer: Layer, role: str, m: int) -> Layer:
    """The layer whose single evaluation gives all m^2 products u'_i o v'_j."""
    if role == FWD:
        return replace(layer, B=m * layer.B, Co=m * layer.Co)
    if role == DGRAD:
        return replace(layer, B=m * layer.B, Ci=m * layer.Ci)
    if role in (WGRAD, WGRAD_REV):
        return replace(layer, Ci=m * layer.Ci, Co=m * layer.Co)
    raise ValueError(role)


def out_channels(layer: Layer, role: str) -> int:
    return layer.Co if role == FWD else layer.Ci


def block(y, layer: Layer, role: str, i: int, j: int):
    """u'_i o v'_j inside a stacked output: FWD / DGRAD (batch rows of j, channels of i);
    WGRAD (grad_W rows of i, columns of j); WGRAD_REV (rows of j, columns of i)."""
    if role in (FWD, DGRAD):
        B, C = layer.B, out_channels(layer, role)
        return y[j * B:(j + 1) * B, i * C:(i + 1) * C]
    Co, Ci = layer.Co, layer.Ci
    r, c = (i, j) if role == WGRAD else (j, i)
    return y[r * Co:(r + 1) * Co, c * Ci:(c + 1) * Ci]


def op(layer: Layer, role: str, u, v, t_bits: int):
    """u o v over Z_t."""
    if role in (FWD, DGRAD):
        return protocol.ring_op(layer, role, u, v, t_bits)
    if role == WGRAD:
        return protocol.ring_op(layer, WGRAD, u, v, t_bits)
    return protocol.ring_op(layer, WGRAD, v, u, t_bits)


def prep(p, sk, layer: Layer, role: str, part, u_masks, v_masks, enc_seed: int, mask_seed: int):
    """P_Prep: returns (S0, S1), the MO's and DO's shares of the stacked output.
    FWD / DGRAD: Alg. 1 on the stacked layer with the MO's input share zero;
    WGRAD / WGRAD_REV: Alg. 2 on the stacked layer keeping one cross term (the
    other's MO operand zero): <gY>_0 (.) Enc(<X>_1) with gY_0 = U, X_1 = V, resp.
    Enc(<gY>_1) (.) <X>_0 with gY_1 = V, X_0 = U."""
    m = len(u_masks)
    assert len(v_masks) == m
    Ls = stacked_layer(layer, role, m)
    U = np.concatenate([np.asarray(u) for u in u_masks], axis=u_axis(role))
    V = np.concatenate([np.asarray(v) for v in v_masks], axis=v_axis(role))
    if role in (FWD, DGRAD):
        zero = np.zeros(V.shape, dtype=_U64)
        s0, s1, _, _, _ = protocol.he_linear(p, sk, Ls, role, part, U, V, zero, enc_seed, mask_seed)
        return np.asarray(s0, dtype=_U64), np.asarray(s1, dtype=_U64)
    if role == WGRAD:
        gy0, x1 = U, V
        gy1, x0 = np.zeros(U.shape, dtype=_U64), np.zeros(V.shape, dtype=_U64)
    else:
        gy1, x0 = V, U
        gy0, x1 = np.zeros(V.shape, dtype=_U64), np.zeros(U.shape, dtype=_U64)
    _, tilde, s = protocol.he_wgrad(p, sk, Ls, part, gy0, gy1, x0, x1, enc_seed, enc_seed + 1, mask_seed)
    return np.asarray(s, dtype=_U64), np.asarray(tilde, dtype=_U64)


def online(layer: Layer, role: str, u, v, u_masks, v_masks, S0, S1, k, l, t_bits: int):
    """P_Online: returns (u~, v~, <u o v>_0, <u o v>_1)."""
    m = len(u_masks)
    mask = _U64((1 << t_bits) - 1)
    with np.errstate(over="ignore"):
        ut = _mod(u, t_bits)
        for i in range(m):
            ut = (ut - _U64(k[i]) * _mod(u_masks[i], t_bits)) & mask
        vt = _mod(v, t_bits)
        for j in range(m):
            vt = (vt - _U64(l[j]) * _mod(v_masks[j], t_bits)) & mask
        z0 = op(layer, role, u, vt, t_bits).astype(_U64)
        z1 = np.zeros_like(z0)
        for j in range(m):
            a0 = np.zeros_like(z0)
            a1 = op(layer, role, ut, v_masks[j], t_bits).astype(_U64)
            for i in range(m):
                a0 = a0 + _U64(k[i]) * block(S0, layer, role, i, j)
                a1 = a1 + _U64(k[i]) * block(S1, layer, role, i, j)
            z0 = z0 + _U64(l[j]) * a0
            z1 = z1 + _U64(l[j]) * a1
        return ut, vt, z0 & mask, z1 & mask
