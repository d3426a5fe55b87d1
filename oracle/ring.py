"""Plain ring arithmetic (oracle; test infrastructure only).

* `negacyclic_schoolbook`: the product in Z_q[X]/(X^N+1) by its definition,
  c_k = sum_{i+j=k} a_i b_j - sum_{i+j=k+N} a_i b_j (Sec. 2.2, Sec. 5 "NTT":
  direct multiplication costs O(N^2)).
* `ring_matmul`, `ring_conv2d`, `ring_conv2d_wgrad`, `ring_conv2d_dgrad`: the
  linear operators of Sec. 2.4 (y = W o x + b, with o = matrix product or 2-D
  convolution) and their gradients, computed directly over Z_t with t = 2^l.
  Because t divides 2^64, uint64 wrap-around arithmetic followed by a mask is
  exact.
"""
from __future__ import annotations

import numpy as np


def negacyclic_schoolbook(a, b, q: int):
    n = len(a)
    out = [0] * n
    for i in range(n):
        ai = int(a[i])
        if ai == 0:
            continue
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += ai * int(b[j])
            else:
                out[k - n] -= ai * int(b[j])
    return [x % q for x in out]


def _u64(x):
    x = np.asarray(x)
    if x.dtype == np.uint64:
        return x
    return x.astype(np.int64).view(np.uint64)


def mod_t(x, t_bits: int):
    """Reduce int64 / uint64 values into [0, 2^t_bits) as uint64."""
    return _u64(x) & np.uint64((1 << t_bits) - 1)


def ring_matmul(w, x, t_bits: int):
    """FC layer over Z_t: y[b, o] = sum_i W[o, i] x[b, i]  (x: B x n_i, W: n_o x n_i)."""
    w = _u64(w)
    x = _u64(x)
    with np.errstate(over="ignore"):
        y = np.zeros((x.shape[0], w.shape[0]), dtype=np.uint64)
        for i in range(w.shape[1]):
            y += x[:, i:i + 1] * w[None, :, i]
    return y & np.uint64((1 << t_bits) - 1)


def _pad(x, pad: int):
    if pad == 0:
        return x
    return np.pad(x, ((0, 0), (0, 0), (pad, pad), (pad, pad)))


def ring_conv2d(w, x, pad: int, t_bits: int):
    """Stride-1 2-D convolution over Z_t (cross-correlation, as in Sec. 2.4):
    y[b, o, i, j] = sum_{c, u, v} W[o, c, u, v] * xpad[b, c, i + u, j + v]."""
    w = _u64(w)
    xp = _pad(_u64(x), pad)
    bsz, ci, h, wd = xp.shape
    co, _, s, s2 = w.shape
    ho, wo = h - s + 1, wd - s2 + 1
    y = np.zeros((bsz, co, ho, wo), dtype=np.uint64)
    with np.errstate(over="ignore"):
        for u in range(s):
            for v in range(s2):
                patch = xp[:, :, u:u + ho, v:v + wo]                # B, ci, ho, wo
                y += np.einsum("bchw,oc->bohw", patch, w[:, :, u, v], dtype=np.uint64)
    return y & np.uint64((1 << t_bits) - 1)


def ring_conv2d_dgrad(w, gy, pad: int, t_bits: int):
    """Input gradient of `ring_conv2d` w.r.t. the unpadded x:
    gx[b, c, i, j] = sum_{o, u, v} gy[b, o, i + pad - u, j + pad - v] W[o, c, u, v]."""
    w = _u64(w)
    gy = _u64(gy)
    bsz, co, ho, wo = gy.shape
    _, ci, s, s2 = w.shape
    hp, wp = ho + s - 1, wo + s2 - 1           # padded input size
    gxp = np.zeros((bsz, ci, hp, wp), dtype=np.uint64)
    with np.errstate(over="ignore"):
        for u in range(s):
            for v in range(s2):
                gxp[:, :, u:u + ho, v:v + wo] += np.einsum(
                    "bohw,oc->bchw", gy, w[:, :, u, v], dtype=np.uint64)
    gx = gxp[:, :, pad:hp - pad, pad:wp - pad]
    return np.ascontiguousarray(gx) & np.uint64((1 << t_bits) - 1)


def ring_conv2d_wgrad(gy, x, pad: int, s: int, t_bits: int):
    """Weight gradient of `ring_conv2d`:
    gW[o, c, u, v] = sum_{b, i, j} gy[b, o, i, j] * xpad[b, c, i + u, j + v]."""
    gy = _u64(gy)
    xp = _pad(_u64(x), pad)
    bsz, co, ho, wo = gy.shape
    ci = xp.shape[1]
    gw = np.zeros((co, ci, s, s), dtype=np.uint64)
    with np.errstate(over="ignore"):
        for u in range(s):
            for v in range(s):
                patch = xp[:, :, u:u + ho, v:v + wo]
                gw[:, :, u, v] = np.einsum("bohw,bchw->oc", gy, patch, dtype=np.uint64)
    return gw & np.uint64((1 << t_bits) - 1)


def ring_matmul_dgrad(w, gy, t_bits: int):
    """gx[b, i] = sum_o gy[b, o] W[o, i]."""
    return ring_matmul(np.ascontiguousarray(_u64(w).T), gy, t_bits)


def ring_matmul_wgrad(gy, x, t_bits: int):
    """gW[o, i] = sum_b gy[b, o] x[b, i]."""
    return ring_matmul(np.ascontiguousarray(_u64(x).T), np.ascontiguousarray(_u64(gy).T), t_bits)


# ---------------------------------------------------------------------------
# The same operators evaluated at chosen output elements only (for checks at
# sizes where the full operator is too slow): each element is its defining sum.
def ring_conv2d_at(w, x, pad: int, t_bits: int, idx):
    """y[b, o, i, j] of `ring_conv2d` for each (b, o, i, j) in idx."""
    w = _u64(w)
    xp = _pad(_u64(x), pad)
    s = w.shape[2]
    out = []
    with np.errstate(over="ignore"):
        for b, o, i, j in idx:
            out.append(int((w[o] * xp[b, :, i:i + s, j:j + s]).sum(dtype=np.uint64)) & ((1 << t_bits) - 1))
    return out


def ring_conv2d_dgrad_at(w, gy, pad: int, t_bits: int, idx):
    """gx[b, c, i, j] of `ring_conv2d_dgrad` for each (b, c, i, j) in idx."""
    w = _u64(w)
    gy = _u64(gy)
    co, ci, s, _ = w.shape
    ho, wo = gy.shape[2], gy.shape[3]
    out = []
    with np.errstate(over="ignore"):
        for b, c, i, j in idx:
            acc = np.uint64(0)
            for u in range(s):
                for v in range(s):
                    r, q = i + pad - u, j + pad - v
                    if 0 <= r < ho and 0 <= q < wo:
                        acc += (gy[b, :, r, q] * w[:, c, u, v]).sum(dtype=np.uint64)
            out.append(int(acc) & ((1 << t_bits) - 1))
    return out


def ring_conv2d_wgrad_at(gy, x, pad: int, s: int, t_bits: int, idx):
    """gW[o, c, u, v] of `ring_conv2d_wgrad` for each (o, c, u, v) in idx."""
    gy = _u64(gy)
    xp = _pad(_u64(x), pad)
    ho, wo = gy.shape[2], gy.shape[3]
    out = []
    with np.errstate(over="ignore"):
        for o, c, u, v in idx:
            out.append(int((gy[:, o] * xp[:, c, u:u + ho, v:v + wo]).sum(dtype=np.uint64)) & ((1 << t_bits) - 1))
    return out
