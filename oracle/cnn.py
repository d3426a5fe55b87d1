"""Fixed-point CNN of the training workload, written directly over Z_t (oracle;
test infrastructure only).

The decoded results of the HE protocols have a plain definition (Sec. 3.2:
<Y>_0 + <Y>_1 = W o X + b, grad_X = W (.)_x grad_Y, grad_W = grad_Y (.) X), so the
oracle of a secure training step is the fixed-point network itself:
conv3x3 -> ReLU -> conv3x3 -> AvgPool 2 -> FC, each linear layer computed with
the direct ring operators of `ring`, the glue between layers (decode, ReLU
with DReLU = 1{x >= 0}, average pooling, re-encode) in float64 on exact dyadic
values (Sec. 2.3, Appendix B).

Readings: forward values are encoded / truncated with floor(x 2^f) as Sec. 2.3
prints; gradients are encoded / truncated with round-to-nearest
floor(x 2^f + 1/2), because at f = 12 the floor's systematic half-unit bias,
summed over a convolution's batch and positions, exceeds the gradient itself
(measured: relative error above 1 for the conv weight gradients); the loss is
scaled by the caller (2^12 in the tests) before its gradient is encoded.
"""
from __future__ import annotations

import numpy as np

from . import ring


def _enc(a, frac, t_bits):
    return (np.floor(np.asarray(a, dtype=np.float64) * (1 << frac)).astype(np.int64).view(np.uint64)
            & np.uint64((1 << t_bits) - 1))


def _enc_round(a, frac, t_bits):
    return (np.floor(np.asarray(a, dtype=np.float64) * (1 << frac) + 0.5).astype(np.int64).view(np.uint64)
            & np.uint64((1 << t_bits) - 1))


def _dec(r, frac, t_bits):
    s = np.asarray(r, dtype=np.uint64).astype(np.int64)
    s = np.where(s >= (1 << (t_bits - 1)), s - (1 << t_bits), s)
    return s.astype(np.float64) / (1 << frac)


def _add(a, b, t_bits):
    with np.errstate(over="ignore"):
        return (np.asarray(a, dtype=np.uint64) + np.asarray(b, dtype=np.uint64)) & np.uint64((1 << t_bits) - 1)


def _avgpool2(h):
    B, C, H, W = h.shape
    return h.reshape(B, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5)) / 4


def _avgpool2_back(g, shape):
    return np.repeat(np.repeat(g, 2, axis=2), 2, axis=3) / 4


def _bias_sum(G, t_bits):
    axes = (0,) if G.ndim == 2 else (0, 2, 3)
    with np.errstate(over="ignore"):
        return G.sum(axis=axes, dtype=np.uint64) & np.uint64((1 << t_bits) - 1)


def train_step(params, x, dlogits, f=12, t_bits=41):
    """params: float64 arrays w1, b1, w2, b2, w3, b3 (fixed-point representable);
    x: float64 input batch; dlogits: float64 gradient of the loss w.r.t. the logits.
    Returns the ring values of every linear layer, forward and backward."""
    r = {}
    W1, W2, W3 = (_enc(params[k], f, t_bits) for k in ("w1", "w2", "w3"))
    B1, B2, B3 = (_enc(params[k], 2 * f, t_bits) for k in ("b1", "b2", "b3"))
    X1 = _enc(x, f, t_bits)
    Y1 = _add(ring.ring_conv2d(W1, X1, 1, t_bits), B1.reshape(1, -1, 1, 1), t_bits)
    y1 = _dec(Y1, 2 * f, t_bits)
    h1 = np.where(y1 >= 0, y1, 0.0)
    X2 = _enc(h1, f, t_bits)
    Y2 = _add(ring.ring_conv2d(W2, X2, 1, t_bits), B2.reshape(1, -1, 1, 1), t_bits)
    h2 = _avgpool2(_dec(Y2, 2 * f, t_bits))
    X3 = _enc(h2.reshape(h2.shape[0], -1), f, t_bits)
    Y3 = _add(ring.ring_matmul(W3, X3, t_bits), B3.reshape(1, -1), t_bits)
    r.update(X1=X1, Y1=Y1, X2=X2, Y2=Y2, X3=X3, Y3=Y3, logits=_dec(Y3, 2 * f, t_bits))

    G3 = _enc_round(dlogits, f, t_bits)
    r.update(G3=G3, GW3=ring.ring_matmul_wgrad(G3, X3, t_bits), GB3=_bias_sum(G3, t_bits))
    GX3 = ring.ring_matmul_dgrad(W3, G3, t_bits)
    gh2 = _avgpool2_back(_dec(GX3, 2 * f, t_bits).reshape(h2.shape), Y2.shape)
    G2 = _enc_round(gh2, f, t_bits)
    r.update(GX3=GX3, G2=G2, GW2=ring.ring_conv2d_wgrad(G2, X2, 1, 3, t_bits), GB2=_bias_sum(G2, t_bits))
    GX2 = ring.ring_conv2d_dgrad(W2, G2, 1, t_bits)
    gh1 = np.where(y1 >= 0, _dec(GX2, 2 * f, t_bits), 0.0)
    G1 = _enc_round(gh1, f, t_bits)
    r.update(GX2=GX2, G1=G1, GW1=ring.ring_conv2d_wgrad(G1, X1, 1, 3, t_bits), GB1=_bias_sum(G1, t_bits))
    r["grads"] = {"w1": _dec(r["GW1"], 2 * f, t_bits), "b1": _dec(r["GB1"], f, t_bits),
                  "w2": _dec(r["GW2"], 2 * f, t_bits), "b2": _dec(r["GB2"], f, t_bits),
                  "w3": _dec(r["GW3"], 2 * f, t_bits), "b3": _dec(r["GB3"], f, t_bits)}
    return r
