"""The linear-layer protocols over shares (oracle; test infrastructure only).

* Alg. 1 (forward): DO sends Enc(<X>_1); MO evaluates
  Enc(W o X) = W o (Enc(<X>_1) + <X>_0), subtracts a fresh mask s, returns the
  ciphertext; DO decrypts <Y>_1 = W o X - s; MO keeps <Y>_0 = s + b.
* Sec. 3.2.2 grad_X: the same protocol with the operator transposed (W^T for
  FC, channel-swapped and 180-degree-rotated kernel on a (s-1-pad)-padded
  grad_Y for convolution).
* Alg. 2 (grad_W): MO evaluates the cross terms
  <gY>_0 (.) Enc(<X>_1) + Enc(<gY>_1) (.) <X>_0, subtracts a mask s; DO decrypts
  and adds its local term <gY>_1 (.) <X>_1; MO adds s and <gY>_0 (.) <X>_0.
  (Step 5's differential-privacy noise is out of scope.)

Each "role" (fwd, dgrad, wgrad) maps the user's tensors onto the one
correlation geometry of `packing` (V: input, Wt: kernel, y: output).

Readings: the MO's mask is one Z_t value per output element, drawn from
stream (mask_seed, MASK) at the element's row-major index in the user's output
layout, so decoded shares do not depend on the partition; coefficients of an
output ciphertext that carry no output get masks from stream
(mask_seed, MASK_PAD, ct_out index).  The DO's encryption randomness for
ct_in[idx] uses (enc_seed, idx).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List

import numpy as np

from . import bfv
from .packing import (Geometry, Partition, counts, decode_positions, pack_input,
                      pack_weight)
from .params import BfvParams
from .ring import (ring_conv2d, ring_conv2d_dgrad, ring_conv2d_wgrad, ring_matmul,
                   ring_matmul_dgrad, ring_matmul_wgrad)
from .sampling import flood_noise, mask_elements, mask_pad

FWD, DGRAD, WGRAD = "fwd", "dgrad", "wgrad"


@dataclass(frozen=True)
class Layer:
    kind: str        # "fc" or "conv"
    B: int
    Ci: int          # n_i for FC
    Co: int          # n_o for FC
    h: int = 1
    w: int = 1
    s: int = 1
    pad: int = 0

    @property
    def ho(self) -> int:
        return self.h + 2 * self.pad - self.s + 1

    @property
    def wo(self) -> int:
        return self.w + 2 * self.pad - self.s + 1

    def x_shape(self):
        return (self.B, self.Ci) if self.kind == "fc" else (self.B, self.Ci, self.h, self.w)

    def w_shape(self):
        return (self.Co, self.Ci) if self.kind == "fc" else (self.Co, self.Ci, self.s, self.s)

    def y_shape(self):
        return (self.B, self.Co) if self.kind == "fc" else (self.B, self.Co, self.ho, self.wo)


def geometry(layer: Layer, role: str) -> Geometry:
    L = layer
    if L.kind == "fc":
        if role == FWD:
            return Geometry(L.B, L.Ci, L.Co, 1, 1, 1, 1)
        if role == DGRAD:
            return Geometry(L.B, L.Co, L.Ci, 1, 1, 1, 1)
        return Geometry(L.Ci, L.B, L.Co, 1, 1, 1, 1)
    hp, wp = L.h + 2 * L.pad, L.w + 2 * L.pad
    if role == FWD:
        return Geometry(L.B, L.Ci, L.Co, hp, wp, L.s, L.s)
    if role == DGRAD:
        e = L.s - 1 - L.pad
        return Geometry(L.B, L.Co, L.Ci, L.ho + 2 * e, L.wo + 2 * e, L.s, L.s)
    return Geometry(L.Ci, L.B, L.Co, hp, wp, L.ho, L.wo)


def _pad4(x, p):
    return np.pad(x, ((0, 0), (0, 0), (p, p), (p, p))) if p else x


def role_input(layer: Layer, role: str, t: np.ndarray) -> np.ndarray:
    """V for the role: fwd <- X, dgrad <- grad_Y, wgrad <- X (channel/batch swapped)."""
    L = layer
    t = np.asarray(t)
    if L.kind == "fc":
        v = t[:, :, None, None]
        return np.ascontiguousarray(v.transpose(1, 0, 2, 3)) if role == WGRAD else v
    if role == FWD:
        return _pad4(t, L.pad)
    if role == DGRAD:
        return _pad4(t, L.s - 1 - L.pad)
    return np.ascontiguousarray(_pad4(t, L.pad).transpose(1, 0, 2, 3))


def role_kernel(layer: Layer, role: str, t: np.ndarray) -> np.ndarray:
    """Wt for the role: fwd <- W, dgrad <- W channel-swapped and rotated,
    wgrad <- grad_Y with batch as the input-channel axis."""
    L = layer
    t = np.asarray(t)
    if L.kind == "fc":
        if role == FWD:
            return t[:, :, None, None]
        if role == DGRAD:
            return np.ascontiguousarray(t.T)[:, :, None, None]
        return np.ascontiguousarray(t.T)[:, :, None, None]          # gY^T: (n_o, B)
    if role == FWD:
        return t
    if role == DGRAD:
        return np.ascontiguousarray(t.transpose(1, 0, 2, 3)[:, :, ::-1, ::-1])
    return np.ascontiguousarray(t.transpose(1, 0, 2, 3))           # gY: (Co, B, Ho, Wo)


def output_shape(layer: Layer, role: str):
    if role == FWD:
        return layer.y_shape()
    if role == DGRAD:
        return layer.x_shape()
    return layer.w_shape()


def output_flat(layer: Layer, role: str, b: int, o: int, i: int, j: int) -> int:
    """Row-major index in the user's output tensor of geometry output (b, o, i, j)."""
    L = layer
    if role == WGRAD:                          # y'[c, o, u, v] = gW[o, c, u, v]
        return ((o * L.Ci + b) * L.s + i) * L.s + j
    g = geometry(L, role)
    return ((b * g.Co + o) * g.Ho + i) * g.Wo + j


# ---------------------------------------------------------------------------
# Plain definitions (what the HE protocol must reach exactly).
# ---------------------------------------------------------------------------
def ring_op(layer: Layer, role: str, a, b, t_bits: int):
    """fwd: (W, X) -> W o X;  dgrad: (W, gY) -> grad_X;  wgrad: (gY, X) -> grad_W."""
    L = layer
    if L.kind == "fc":
        if role == FWD:
            return ring_matmul(a, b, t_bits)
        if role == DGRAD:
            return ring_matmul_dgrad(a, b, t_bits)
        return ring_matmul_wgrad(a, b, t_bits)
    if role == FWD:
        return ring_conv2d(a, b, L.pad, t_bits)
    if role == DGRAD:
        return ring_conv2d_dgrad(a, b, L.pad, t_bits)
    return ring_conv2d_wgrad(a, b, L.pad, L.s, t_bits)


# ---------------------------------------------------------------------------
# Step-by-step HE protocol.
# ---------------------------------------------------------------------------
def _enc(p: BfvParams, sk, pk, m, seed: int, i: int) -> np.ndarray:
    return bfv.encrypt(p, sk, m, seed, i) if pk is None else bfv.encrypt_pk(p, pk, m, seed, i)


def encrypt_inputs(p: BfvParams, sk, layer: Layer, role: str, part: Partition,
                   share, seed: int, indices=None, pk=None) -> Dict[int, np.ndarray]:
    """DO: Enc(pi_v(share)) for ct_in[m * K + k] (all, or only `indices`);
    with the secret key, or with the public key `pk` when one is given."""
    g = geometry(layer, role)
    c = counts(g, part)
    V = role_input(layer, role, share)
    idx = range(c.ct_in) if indices is None else indices
    return {i: _enc(p, sk, pk, pack_input(V, g, part, p.n, i // c.K, i % c.K), seed, i)
            for i in idx}


def encrypt_kernel_operand(p: BfvParams, sk, layer: Layer, role: str, part: Partition,
                           share, seed: int, indices=None, pk=None) -> Dict[int, np.ndarray]:
    """DO: Enc(pi_W(share)) for kernel-position operand [k * NC + n] (Alg. 2's
    Enc(<gY>_1)); secret- or public-key as encrypt_inputs."""
    g = geometry(layer, role)
    c = counts(g, part)
    Wt = role_kernel(layer, role, share)
    idx = range(c.pt) if indices is None else indices
    return {i: _enc(p, sk, pk, pack_weight(Wt, g, part, p.n, i // c.NC, i % c.NC), seed, i)
            for i in idx}


def encode_kernel(p: BfvParams, layer: Layer, role: str, part: Partition, values,
                  indices=None) -> Dict[int, np.ndarray]:
    """MO: NTT(pi_W(values)) for pt[k * NC + n] (weights, or Alg. 2's <gY>_0)."""
    g = geometry(layer, role)
    c = counts(g, part)
    Wt = role_kernel(layer, role, values)
    idx = range(c.pt) if indices is None else indices
    return {i: bfv.encode_plain(p, pack_weight(Wt, g, part, p.n, i // c.NC, i % c.NC))
            for i in idx}


def encode_input(p: BfvParams, layer: Layer, role: str, part: Partition, values,
                 indices=None) -> Dict[int, np.ndarray]:
    """MO: NTT(pi_v(values)) at input position [m * K + k] (Alg. 2's <X>_0)."""
    g = geometry(layer, role)
    c = counts(g, part)
    V = role_input(layer, role, values)
    idx = range(c.ct_in) if indices is None else indices
    return {i: bfv.encode_plain(p, pack_input(V, g, part, p.n, i // c.K, i % c.K))
            for i in idx}


def mask_polynomial(p: BfvParams, layer: Layer, role: str, part: Partition,
                    mask_seed: int, ct_out: int) -> List[int]:
    """The mask s subtracted from ct_out (Alg. 1 step 3), coefficient form."""
    g = geometry(layer, role)
    c = counts(g, part)
    poly = mask_pad(mask_seed, ct_out, p.n, p.t)
    elems = mask_elements(mask_seed, int(np.prod(output_shape(layer, role))), p.t)
    for e, (b, o, i, j) in decode_positions(g, part, ct_out // c.NC, ct_out % c.NC):
        poly[e] = elems[output_flat(layer, role, b, o, i, j)]
    return poly


def flood(p: BfvParams, ct: np.ndarray, mask_seed: int, ct_out: int, flood_bits: int) -> np.ndarray:
    """Noise flooding of a returned ciphertext (no-op for flood_bits = 0)."""
    if not flood_bits:
        return ct
    return bfv.add_noise(p, ct, flood_noise(mask_seed, ct_out, p.n, flood_bits))


def mo_forward_ct(p: BfvParams, layer: Layer, role: str, part: Partition, ct_in: Dict,
                  pts: Dict, x0, mask_seed: int, ct_out: int, flood_bits: int = 0) -> np.ndarray:
    """Alg. 1 steps 2-3 for one output ciphertext:
    sum_k (ct_in[m,k] + [q pi_v(x0) / t]) * pt[k,n] - [q s / t] (+ flooding noise)."""
    g = geometry(layer, role)
    c = counts(g, part)
    m, nn = divmod(ct_out, c.NC)
    V0 = role_input(layer, role, x0)
    acc = None
    for k in range(c.K):
        ct = bfv.add_plain(p, ct_in[m * c.K + k], pack_input(V0, g, part, p.n, m, k))
        prod = bfv.mul_plain(p, ct, pts[k * c.NC + nn])
        acc = prod if acc is None else bfv.add_ct(p, acc, prod)
    out = bfv.sub_plain(p, acc, mask_polynomial(p, layer, role, part, mask_seed, ct_out))
    return flood(p, out, mask_seed, ct_out, flood_bits)


def mo_wgrad_ct(p: BfvParams, layer: Layer, part: Partition, ct_x1: Dict, pt_gy0: Dict,
                ct_gy1: Dict, pt_x0: Dict, mask_seed: int, ct_out: int, flood_bits: int = 0) -> np.ndarray:
    """Alg. 2 steps 2-3 for one output ciphertext:
    sum_k Enc(x1)[m,k] * gy0[k,n] + Enc(gy1)[k,n] * x0[m,k] - [q s / t]."""
    g = geometry(layer, WGRAD)
    c = counts(g, part)
    m, nn = divmod(ct_out, c.NC)
    acc = None
    for k in range(c.K):
        a = bfv.mul_plain(p, ct_x1[m * c.K + k], pt_gy0[k * c.NC + nn])
        b = bfv.mul_plain(p, ct_gy1[k * c.NC + nn], pt_x0[m * c.K + k])
        term = bfv.add_ct(p, a, b)
        acc = term if acc is None else bfv.add_ct(p, acc, term)
    out = bfv.sub_plain(p, acc, mask_polynomial(p, layer, WGRAD, part, mask_seed, ct_out))
    return flood(p, out, mask_seed, ct_out, flood_bits)


def decrypt_outputs(p: BfvParams, sk, layer: Layer, role: str, part: Partition,
                    ct_outs: Dict[int, np.ndarray], out: np.ndarray | None = None) -> np.ndarray:
    """DO: decrypt every given ct_out and scatter pi_y^{-1} into the user's output layout."""
    g = geometry(layer, role)
    c = counts(g, part)
    if out is None:
        out = np.zeros(int(np.prod(output_shape(layer, role))), dtype=np.uint64)
    for idx, ct in ct_outs.items():
        msg = bfv.decrypt(p, sk, ct)
        for e, (b, o, i, j) in decode_positions(g, part, idx // c.NC, idx % c.NC):
            out[output_flat(layer, role, b, o, i, j)] = msg[e]
    return out


def compact_returned(p: BfvParams, layer: Layer, role: str, part: Partition, ct_outs: Dict[int, np.ndarray]):
    """MO: the send form of returned ciphertexts with the coefficients that
    carry no output dropped: c1 as is (NTT form), c0 in coefficient form at the
    output coefficients only, gathered as c0c[limb][flat] (flat = the output
    element's index in the user's layout).  Returns (c1 by ct index, c0c)."""
    g = geometry(layer, role)
    c = counts(g, part)
    c0c = np.zeros((len(p.primes), int(np.prod(output_shape(layer, role)))), dtype=object)
    c1s = {}
    for idx, ct in ct_outs.items():
        coeff = bfv.from_ntt(p, ct[0])
        for e, (b, o, i, j) in decode_positions(g, part, idx // c.NC, idx % c.NC):
            c0c[:, output_flat(layer, role, b, o, i, j)] = coeff[:, e]
        c1s[idx] = ct[1]
    return c1s, c0c


def decrypt_compact(p: BfvParams, sk, layer: Layer, role: str, part: Partition, c1s: Dict[int, np.ndarray],
                    c0c: np.ndarray, out: np.ndarray | None = None) -> np.ndarray:
    """DO: decrypt the send form: at an output coefficient e of ciphertext idx,
    x = INTT(c1 * NTT(s))[e] + c0c[flat] per limb, CRT, m = round(t x / q) mod t."""
    g = geometry(layer, role)
    c = counts(g, part)
    q, t = p.q, p.t
    if out is None:
        out = np.zeros(int(np.prod(output_shape(layer, role))), dtype=np.uint64)
    for idx, c1 in c1s.items():
        c1s_coeff = bfv.from_ntt(p, np.stack([c1[i] * sk.s_hat[i] % qi for i, qi in enumerate(p.primes)]))
        for e, (b, o, i, j) in decode_positions(g, part, idx // c.NC, idx % c.NC):
            flat = output_flat(layer, role, b, o, i, j)
            x = bfv.crt(p, [(int(c1s_coeff[li, e]) + int(c0c[li, flat])) % qi for li, qi in enumerate(p.primes)])
            out[flat] = ((2 * t * x + q) // (2 * q)) % t
    return out


def send_bytes(p: BfvParams, layer: Layer, role: str, part: Partition, compact: bool) -> int:
    """Bytes of the returned ciphertexts of one evaluation (64-bit words):
    2 L N per ciphertext, or L N per ciphertext + L per output element compacted."""
    c = counts(geometry(layer, role), part)
    L, n = len(p.primes), p.n
    if not compact:
        return 8 * 2 * L * n * c.ct_out
    return 8 * (L * n * c.ct_out + L * int(np.prod(output_shape(layer, role))))


def mo_share(p: BfvParams, layer: Layer, role: str, mask_seed: int, bias=None) -> np.ndarray:
    """MO's output share: s (+ b broadcast over the output channel for the forward role)."""
    shape = output_shape(layer, role)
    s = np.array(mask_elements(mask_seed, int(np.prod(shape)), p.t), dtype=np.uint64).reshape(shape)
    if bias is not None:
        b = np.asarray(bias).astype(np.int64).view(np.uint64)
        bshape = (1, -1) + (1,) * (len(shape) - 2)
        with np.errstate(over="ignore"):
            s = (s + b.reshape(bshape)) & np.uint64(p.t - 1)
    return s


def he_linear(p: BfvParams, sk, layer: Layer, role: str, part: Partition, kernel, x1, x0,
              enc_seed: int, mask_seed: int, bias=None, flood_bits: int = 0):
    """Full Alg. 1 (fwd / dgrad roles) on small shapes: returns (y0, y1, ct_in, pts, ct_out)."""
    g = geometry(layer, role)
    c = counts(g, part)
    ct_in = encrypt_inputs(p, sk, layer, role, part, x1, enc_seed)
    pts = encode_kernel(p, layer, role, part, kernel)
    ct_out = {i: mo_forward_ct(p, layer, role, part, ct_in, pts, x0, mask_seed, i, flood_bits)
              for i in range(c.ct_out)}
    y1 = decrypt_outputs(p, sk, layer, role, part, ct_out).reshape(output_shape(layer, role))
    y0 = mo_share(p, layer, role, mask_seed, bias)
    return y0, y1, ct_in, pts, ct_out


def he_wgrad(p: BfvParams, sk, layer: Layer, part: Partition, gy0, gy1, x0, x1,
             enc_seed_x: int, enc_seed_g: int, mask_seed: int, flood_bits: int = 0):
    """Full Alg. 2 on small shapes.  Returns (grad_W, DO's decrypted tilde, MO mask)."""
    g = geometry(layer, WGRAD)
    c = counts(g, part)
    ct_x1 = encrypt_inputs(p, sk, layer, WGRAD, part, x1, enc_seed_x)
    ct_gy1 = encrypt_kernel_operand(p, sk, layer, WGRAD, part, gy1, enc_seed_g)
    pt_gy0 = encode_kernel(p, layer, WGRAD, part, gy0)
    pt_x0 = encode_input(p, layer, WGRAD, part, x0)
    ct_out = {i: mo_wgrad_ct(p, layer, part, ct_x1, pt_gy0, ct_gy1, pt_x0, mask_seed, i, flood_bits)
              for i in range(c.ct_out)}
    shape = output_shape(layer, WGRAD)
    tilde = decrypt_outputs(p, sk, layer, WGRAD, part, ct_out).reshape(shape)
    s = mo_share(p, layer, WGRAD, mask_seed)
    with np.errstate(over="ignore"):
        tilde_do = (tilde + ring_op(layer, WGRAD, gy1, x1, p.t_bits)) & np.uint64(p.t - 1)
        gw = (tilde_do + s + ring_op(layer, WGRAD, gy0, x0, p.t_bits)) & np.uint64(p.t - 1)
    return gw, tilde, s
