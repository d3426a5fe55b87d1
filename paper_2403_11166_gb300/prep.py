"""The preprocessing protocol (Alg. 3) of a linear operator on the GPU, for the
four operators of Alg. 4 (u: the MO's operand, v: the DO's operand):

  he.ROLE_FWD    (o)       u = W,           v = X,           u o v = W o X
  he.ROLE_DGRAD  ((.)_x)   u = W,           v = grad_Y,      u o v = W (.)_x grad_Y
  he.ROLE_WGRAD  ((.))     u = <grad_Y>_0,  v = <X>_1,       u o v = u (.) v
  WGRAD_REV      ((.)_rev) u = <X>_0,       v = <grad_Y>_1,  u o v = v (.) u

P_Prep (HE, once): the MO's m masks u'_i and the DO's m masks v'_j are stacked
into one evaluation of a larger layer (batch or channels m times as large), so
that block (i, j) of its output is u'_i o v'_j, shared as (s_ij, u'_i o v'_j -
s_ij): Alg. 1 with the MO's own input share zero (FWD, DGRAD), or Alg. 2 with
the other cross term's MO operand zero (WGRAD, WGRAD_REV).

P_Online (no HE): masked operands and shares are linear combinations over Z_t
(`pencil_lincomb`) plus two plaintext ring operators (`pencil_ring_linear`):
  u~ = u - sum_i k_i u'_i,  v~ = v - sum_j l_j v'_j,
  A0_j = sum_i k_i S0[i, j],  A1_j = u~ o v'_j + sum_i k_i S1[i, j],
  <u o v>_0 = u o v~ + sum_j l_j A0_j,  <u o v>_1 = sum_j l_j A1_j.
All tensors are int64 storage of Z_t values in the user's layouts.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Optional, Sequence, Tuple

import torch

from . import he

WGRAD_REV = 3   # (.)_rev: Alg. 2's second cross term with the MO's X-shaped operand


@dataclass
class Strided:
    """Element e of a result read at off + (e // inner) * outer + e % inner (+ i * term for term i)."""
    off: int
    inner: int
    outer: int
    term: int


def _layer(kind, B, Ci, Co, H, W, s, pad) -> he.Layer:
    return he.Layer(kind, B, Ci, Co, H, W, s, pad)


@dataclass
class Layout:
    """Where Alg. 3's operands and shares live for one operator: the stacked
    layer of the m^2 preprocessing products, the operand / mask / share sizes,
    and strided descriptors (mask i of u at u_st + i * u_st.term; share block
    (i, j) of the stacked output at blk(j) + i * blk(j).term, blk(j).off linear
    in j; ring block j at ring_blk(j))."""
    stacked: he.Layer
    he_role: int
    n_u: int
    n_v: int
    n_out: int
    u_st: Strided
    v_st: Strided
    blk: Callable[[int], Strided]
    ring_all: tuple
    ring_blk: Callable[[int], Strided]
    ring_one: tuple


def layout(layer: he.Layer, role: int, m: int) -> Layout:
    Lr = layer
    kind, B, Ci, Co, H, W, s, pad = Lr.kind, Lr.batch, Lr.c_in, Lr.c_out, Lr.height, Lr.width, Lr.kernel, Lr.pad
    conv = kind == he.CONV
    Ho, Wo = (H + 2 * pad - s + 1, W + 2 * pad - s + 1) if conv else (1, 1)
    HW, HoWo, ss = (H * W, Ho * Wo, s * s) if conv else (1, 1, 1)
    if role == he.ROLE_FWD:
        n_u, n_v, n_out = Co * Ci * ss, B * Ci * HW, B * Co * HoWo
        return Layout(_layer(kind, m * B, Ci, m * Co, H, W, s, pad), he.ROLE_FWD, n_u, n_v, n_out,
                      Strided(0, n_u, 0, n_u), Strided(0, n_v, 0, n_v),
                      lambda j: Strided(j * B * m * Co * HoWo, Co * HoWo, m * Co * HoWo, Co * HoWo),
                      (_layer(kind, m * B, Ci, Co, H, W, s, pad), he.ROLE_FWD, "uv"),
                      lambda j: Strided(j * n_out, n_out, 0, 0), (Lr, he.ROLE_FWD, "uv"))
    if role == he.ROLE_DGRAD:
        n_u, n_v, n_out = Co * Ci * ss, B * Co * HoWo, B * Ci * HW
        return Layout(_layer(kind, m * B, m * Ci, Co, H, W, s, pad), he.ROLE_DGRAD, n_u, n_v, n_out,
                      Strided(0, Ci * ss, m * Ci * ss, Ci * ss), Strided(0, n_v, 0, n_v),
                      lambda j: Strided(j * B * m * Ci * HW, Ci * HW, m * Ci * HW, Ci * HW),
                      (_layer(kind, m * B, Ci, Co, H, W, s, pad), he.ROLE_DGRAD, "uv"),
                      lambda j: Strided(j * n_out, n_out, 0, 0), (Lr, he.ROLE_DGRAD, "uv"))
    if role == he.ROLE_WGRAD:
        n_u, n_v, n_out = B * Co * HoWo, B * Ci * HW, Co * Ci * ss
        return Layout(_layer(kind, B, m * Ci, m * Co, H, W, s, pad), he.ROLE_WGRAD, n_u, n_v, n_out,
                      Strided(0, Co * HoWo, m * Co * HoWo, Co * HoWo), Strided(0, Ci * HW, m * Ci * HW, Ci * HW),
                      lambda j: Strided(j * Ci * ss, Ci * ss, m * Ci * ss, Co * m * Ci * ss),
                      (_layer(kind, B, m * Ci, Co, H, W, s, pad), he.ROLE_WGRAD, "uv"),
                      lambda j: Strided(j * Ci * ss, Ci * ss, m * Ci * ss, 0), (Lr, he.ROLE_WGRAD, "uv"))
    if role == WGRAD_REV:
        n_u, n_v, n_out = B * Ci * HW, B * Co * HoWo, Co * Ci * ss
        return Layout(_layer(kind, B, m * Ci, m * Co, H, W, s, pad), he.ROLE_WGRAD, n_u, n_v, n_out,
                      Strided(0, Ci * HW, m * Ci * HW, Ci * HW), Strided(0, Co * HoWo, m * Co * HoWo, Co * HoWo),
                      lambda j: Strided(j * Co * m * Ci * ss, Ci * ss, m * Ci * ss, Ci * ss),
                      (_layer(kind, B, Ci, m * Co, H, W, s, pad), he.ROLE_WGRAD, "vu"),
                      lambda j: Strided(j * n_out, n_out, 0, 0), (Lr, he.ROLE_WGRAD, "vu"))
    raise ValueError(role)


class PrepProduct:
    """Alg. 3 for one operator of `layer` with m masks per party."""

    def __init__(self, ctx: he.Context, sk: he.SecretKey, layer: he.Layer, role: int, m: int,
                 part: Optional[tuple] = None):
        self.ctx, self.sk, self.layer, self.role, self.m = ctx, sk, layer, role, m
        lay = layout(layer, role, m)
        self.stacked, self.he_role = lay.stacked, lay.he_role
        self.n_u, self.n_v, self.n_out = lay.n_u, lay.n_v, lay.n_out
        self.u_st, self.v_st, self.blk = lay.u_st, lay.v_st, lay.blk
        self.ring_all, self.ring_blk, self.ring_one = lay.ring_all, lay.ring_blk, lay.ring_one
        self.plan_s = he.Plan(ctx, self.stacked, self.he_role, part)
        self.plan_all = he.Plan(ctx, self.ring_all[0], self.ring_all[1], None)
        self.plan_one = he.Plan(ctx, self.ring_one[0], self.ring_one[1], None)
        self.dev = torch.device(f"cuda:{ctx.device}")
        self.products = self.plan_s.sizes.products * (1 if self.he_role != he.ROLE_WGRAD else 2)
        self.S0 = self.S1 = self.u_masks = self.v_masks = None

    # ---------------------------------------------------------------- P_Prep
    def preprocess(self, u_masks: torch.Tensor, v_masks: torch.Tensor, enc_seed: int, mask_seed: int,
                   stream=None):
        """u_masks / v_masks: the masks stacked as the stacked layer's operands (FWD: u'_i along W's
        output channel, v'_j along the batch; DGRAD: u'_i along W's input channel, v'_j along the
        batch; WGRAD / WGRAD_REV: along the channel axis of grad_Y / X)."""
        ctx, P, sk = self.ctx, self.plan_s, self.sk
        S = P.sizes
        u_masks, v_masks = u_masks.contiguous(), v_masks.contiguous()
        ws_do = P.new_ws(max(S.ws_encrypt, S.ws_decrypt))
        S0 = torch.empty(S.out_elems, dtype=torch.int64, device=self.dev)
        S1 = torch.empty_like(S0)
        ct_out = P.new_ct(S.ct_out)
        if self.he_role != he.ROLE_WGRAD:
            pt, ct_in = P.new_pt(S.pt), P.new_ct(S.ct_in)
            ws_mo = P.new_ws(S.ws_forward if self.he_role == he.ROLE_FWD else S.ws_backward)
            zero = torch.zeros_like(v_masks)
            he.encode_weights(ctx, P, he.OPERAND_KERNEL, u_masks, pt, stream=stream)                    # MO
            he.encrypt_share(ctx, sk, P, he.OPERAND_INPUT, v_masks, enc_seed, ct_in, ws_do, stream=stream)  # DO
            if self.he_role == he.ROLE_FWD:                                                               # MO
                he.he_linear_forward(ctx, P, ct_in, pt, zero, None, mask_seed, ct_out, S0, ws_mo, stream=stream)
            else:
                he.he_linear_backward(ctx, P, None, ct_in, pt, None, None, zero, None, mask_seed, 0, ct_out, S0,
                                      None, None, ws_mo, stream=stream)
        else:
            ws_mo = P.new_ws(S.ws_backward)
            if self.role == he.ROLE_WGRAD:      # <gY>_0 (.) Enc(<X>_1): gY_0 = u', X_1 = v'
                gy0, x1 = u_masks, v_masks
                gy1, x0 = torch.zeros_like(u_masks), torch.zeros_like(v_masks)
            else:                               # Enc(<gY>_1) (.) <X>_0: gY_1 = v', X_0 = u'
                gy1, x0 = v_masks, u_masks
                gy0, x1 = torch.zeros_like(v_masks), torch.zeros_like(u_masks)
            ct_x1, ct_g1 = P.new_ct(S.ct_in), P.new_ct(S.pt)
            he.encrypt_share(ctx, sk, P, he.OPERAND_INPUT, x1, enc_seed, ct_x1, ws_do, stream=stream)   # DO
            he.encrypt_share(ctx, sk, P, he.OPERAND_KERNEL, gy1, enc_seed + 1, ct_g1, ws_do, stream=stream)
            he.he_linear_backward(ctx, None, P, None, None, ct_x1, ct_g1, gy0, x0, 0, mask_seed, None, None,
                                  ct_out, S0, ws_mo, stream=stream)                                      # MO
        he.decrypt_to_share(ctx, sk, P, ct_out, S1, True, ws_do, stream=stream)                          # DO
        self.S0, self.S1 = S0, S1
        self.u_masks, self.v_masks = u_masks, v_masks

    # ---------------------------------------------------------------- P_Online
    def _comb(self, src, scalars, count, out, st: Strided, addend=None, negate=False, stream=None):
        he.pencil_lincomb(self.ctx, src, scalars, count, out, addend=addend, negate=negate, src_offset=st.off,
                          inner=st.inner, outer_stride=st.outer, term_stride=st.term, stream=stream)

    def _ring(self, spec, plan, u_like, v_like, out, stream=None):
        """out = u_like o v_like with the operand order of the operator ("uv": kernel = u;
        "vu": kernel = v, input = u)."""
        kern, inp = (u_like, v_like) if spec[2] == "uv" else (v_like, u_like)
        he.pencil_ring_linear(self.ctx, plan, kern, inp, None, out, stream=stream)

    def online(self, u: torch.Tensor, v: torch.Tensor, k: Sequence[int], l: Sequence[int], stream=None
               ) -> Tuple[torch.Tensor, torch.Tensor, torch.Tensor, torch.Tensor]:
        """Returns (u~, v~, <u o v>_0, <u o v>_1) (flat int64 tensors of Z_t values)."""
        assert self.S0 is not None, "preprocess first"
        m, dev, n_out = self.m, self.dev, self.n_out
        u, v = u.contiguous(), v.contiguous()
        ut = torch.empty(self.n_u, dtype=torch.int64, device=dev)     # MO: u~ = u - sum_i k_i u'_i
        self._comb(self.u_masks, k, self.n_u, ut, self.u_st, addend=u, negate=True, stream=stream)
        vt = torch.empty(self.n_v, dtype=torch.int64, device=dev)     # DO: v~ = v - sum_j l_j v'_j
        self._comb(self.v_masks, l, self.n_v, vt, self.v_st, addend=v, negate=True, stream=stream)
        R = torch.empty(m * n_out, dtype=torch.int64, device=dev)
        self._ring(self.ring_all, self.plan_all, ut, self.v_masks, R, stream=stream)               # DO: u~ o v'_j
        z0 = torch.empty(n_out, dtype=torch.int64, device=dev)
        z1 = torch.empty_like(z0)
        self._ring(self.ring_one, self.plan_one, u, vt, z0, stream=stream)                          # MO: u o v~
        if m * m <= 64:
            # <u o v>_0 = u o v~ + sum_{i,j} l_j k_i S0[i, j]   (MO)
            # <u o v>_1 = sum_j l_j (u~ o v'_j) + sum_{i,j} l_j k_i S1[i, j]   (DO)
            # (the same sums as the per-j shares <u o v'_j> below, regrouped: one pass over each S)
            tm = (1 << self.ctx.t_bits) - 1
            lk = [(int(l[j]) * int(k[i])) & tm for j in range(m) for i in range(m)]
            b0, b1, r0, r1 = self.blk(0), self.blk(1), self.ring_blk(0), self.ring_blk(1)
            he.pencil_lincomb2(self.ctx, self.S0, lk, m, m, n_out, z0, addend=z0, src_offset=b0.off, inner=b0.inner,
                               outer_stride=b0.outer, term_stride=b0.term, term_stride2=b1.off - b0.off,
                               stream=stream)
            he.pencil_lincomb(self.ctx, R, l, n_out, z1, src_offset=r0.off, inner=r0.inner, outer_stride=r0.outer,
                              term_stride=r1.off - r0.off, stream=stream)
            he.pencil_lincomb2(self.ctx, self.S1, lk, m, m, n_out, z1, addend=z1, src_offset=b0.off, inner=b0.inner,
                               outer_stride=b0.outer, term_stride=b0.term, term_stride2=b1.off - b0.off,
                               stream=stream)
            return ut, vt, z0, z1
        # shares of u o v'_j for every j (j-major, each in the operator's output layout)
        A0 = torch.empty(m * n_out, dtype=torch.int64, device=dev)
        A1 = torch.empty_like(A0)
        for j in range(m):
            a0, a1 = A0[j * n_out:(j + 1) * n_out], A1[j * n_out:(j + 1) * n_out]
            self._comb(self.S0, k, n_out, a0, self.blk(j), stream=stream)                          # MO
            self._comb(R, [1], n_out, a1, self.ring_blk(j), stream=stream)                          # DO
            self._comb(self.S1, k, n_out, a1, self.blk(j), addend=a1, stream=stream)
        # shares of u o v
        he.pencil_lincomb(self.ctx, A0, l, n_out, z0, addend=z0, term_stride=n_out, stream=stream)
        he.pencil_lincomb(self.ctx, A1, l, n_out, z1, term_stride=n_out, stream=stream)            # DO
        return ut, vt, z0, z1
