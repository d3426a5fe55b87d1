"""The preprocessing protocol (Alg. 3) of a linear operator on the GPU.

P_Prep (HE, once): the MO's m masks u'_i and the DO's m masks v'_j are stacked
into one layer evaluation (batch m B with v'_j at batch rows j B.., the
operator's output channels m C with u'_i at channels i C..), so Alg. 1 on that
layer (the MO's own input share zero) yields every product u'_i o v'_j in
block (i, j) of the stacked output, as shares (s_ij, u'_i o v'_j - s_ij).

P_Online (no HE): masked operands and shares are linear combinations over Z_t
(`pencil_lincomb`) and two plaintext ring operators (`pencil_ring_linear`):
  u~ = u - sum_i k_i u'_i,  v~ = v - sum_j l_j v'_j,
  A0_j = sum_i k_i S0[i, j],  A1_j = u~ o v'_j + sum_i k_i S1[i, j],
  <u o v>_0 = u o v~ + sum_j l_j A0_j,  <u o v>_1 = sum_j l_j A1_j.

Operators: the forward product (u = W, v = X) and the input gradient
(u = W, v = grad_Y).  All tensors are int64 storage of Z_t values in the
user's layouts.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import torch

from . import he


def _stacked(layer: he.Layer, role: int, m: int) -> he.Layer:
    if role == he.ROLE_FWD:
        return he.Layer(layer.kind, m * layer.batch, layer.c_in, m * layer.c_out, layer.height, layer.width,
                        layer.kernel, layer.pad)
    if role == he.ROLE_DGRAD:
        return he.Layer(layer.kind, m * layer.batch, m * layer.c_in, layer.c_out, layer.height, layer.width,
                        layer.kernel, layer.pad)
    raise ValueError("the preprocessing protocol covers the forward and input-gradient operators")


def _spatial_out(layer: he.Layer, role: int) -> int:
    if layer.kind == he.FC:
        return 1
    if role == he.ROLE_FWD:
        return (layer.height + 2 * layer.pad - layer.kernel + 1) * (layer.width + 2 * layer.pad - layer.kernel + 1)
    return layer.height * layer.width


class PrepProduct:
    """Alg. 3 for one operator (he.ROLE_FWD: W o X, he.ROLE_DGRAD: W (.)_x grad_Y) of `layer`."""

    def __init__(self, ctx: he.Context, sk: he.SecretKey, layer: he.Layer, role: int, m: int,
                 part: Optional[tuple] = None):
        self.ctx, self.sk, self.layer, self.role, self.m = ctx, sk, layer, role, m
        self.stacked = _stacked(layer, role, m)
        self.plan_s = he.Plan(ctx, self.stacked, role, part)        # HE evaluation of all m^2 products
        self.plan = he.Plan(ctx, layer, role, None)                  # ring operator u o v~
        self.plan_vj = he.Plan(ctx, he.Layer(layer.kind, m * layer.batch, layer.c_in, layer.c_out, layer.height,
                                             layer.width, layer.kernel, layer.pad), role, None)   # u~ o v'_j
        self.C = layer.c_out if role == he.ROLE_FWD else layer.c_in     # the operator's output channels
        self.HW = _spatial_out(layer, role)
        self.out_elems = self.plan.sizes.out_elems                       # B C HW
        self.dev = torch.device(f"cuda:{ctx.device}")
        self.S0 = self.S1 = None
        self.u_masks = self.v_masks = None
        self.products = self.plan_s.sizes.products

    # ---------------------------------------------------------------- P_Prep
    def preprocess(self, u_masks: torch.Tensor, v_masks: torch.Tensor, enc_seed: int, mask_seed: int,
                   stream=None):
        """u_masks: the MO's u'_i stacked along the operator's output channel (FWD: [m Co, Ci, ..],
        DGRAD: [Co, m Ci, ..]); v_masks: the DO's v'_j stacked along the batch ([m B, ..])."""
        ctx, P = self.ctx, self.plan_s
        S = P.sizes
        pt, ct_in, ct_out = P.new_pt(S.pt), P.new_ct(S.ct_in), P.new_ct(S.ct_out)
        ws_mo = P.new_ws(S.ws_forward if self.role == he.ROLE_FWD else S.ws_backward)
        ws_do = P.new_ws(max(S.ws_encrypt, S.ws_decrypt))
        zero = torch.zeros_like(v_masks)
        S0 = torch.empty(S.out_elems, dtype=torch.int64, device=self.dev)
        S1 = torch.empty_like(S0)
        he.encode_weights(ctx, P, he.OPERAND_KERNEL, u_masks.contiguous(), pt, stream=stream)          # MO
        he.encrypt_share(ctx, self.sk, P, he.OPERAND_INPUT, v_masks.contiguous(), enc_seed, ct_in, ws_do,
                         stream=stream)                                                                  # DO
        if self.role == he.ROLE_FWD:                                                                     # MO
            he.he_linear_forward(ctx, P, ct_in, pt, zero, None, mask_seed, ct_out, S0, ws_mo, stream=stream)
        else:
            he.he_linear_backward(ctx, P, None, ct_in, pt, None, None, zero, None, mask_seed, 0, ct_out, S0,
                                  None, None, ws_mo, stream=stream)
        he.decrypt_to_share(ctx, self.sk, P, ct_out, S1, True, ws_do, stream=stream)                   # DO
        self.S0, self.S1 = S0, S1
        self.u_masks, self.v_masks = u_masks.contiguous(), v_masks.contiguous()

    # ---------------------------------------------------------------- P_Online
    def _block_comb(self, S: torch.Tensor, k: Sequence[int], out: torch.Tensor, addend=None, stream=None):
        """out (j-stacked [m B, C, HW]) = addend + sum_i k_i S[block (i, j)]."""
        inner = self.C * self.HW
        he.pencil_lincomb(self.ctx, S, k, out.numel(), out, addend=addend, inner=inner,
                          outer_stride=self.m * inner, term_stride=inner, stream=stream)

    def online(self, u: torch.Tensor, v: torch.Tensor, k: Sequence[int], l: Sequence[int], stream=None):
        """Returns (u~, v~, <u o v>_0, <u o v>_1) (flat int64 tensors of Z_t values)."""
        ctx, m = self.ctx, self.m
        assert self.S0 is not None, "preprocess first"
        u, v = u.contiguous(), v.contiguous()
        un, vn = u.numel(), v.numel()
        # MO: u~ = u - sum_i k_i u'_i (the u'_i stacked along the output channel of the operator)
        ut = torch.empty(un, dtype=torch.int64, device=self.dev)
        if self.role == he.ROLE_FWD:   # [m Co, Ci, ..]: mask i is a contiguous block
            he.pencil_lincomb(ctx, self.u_masks, k, un, ut, addend=u, negate=True, term_stride=un, stream=stream)
        else:                          # [Co, m Ci, ..]: mask i at channel offset i Ci in every row o
            inner = self.layer.c_in * self.layer.kernel * self.layer.kernel
            he.pencil_lincomb(ctx, self.u_masks, k, un, ut, addend=u, negate=True, inner=inner,
                              outer_stride=m * inner, term_stride=inner, stream=stream)
        # DO: v~ = v - sum_j l_j v'_j (batch-stacked: mask j is a contiguous block)
        vt = torch.empty(vn, dtype=torch.int64, device=self.dev)
        he.pencil_lincomb(ctx, self.v_masks, l, vn, vt, addend=v, negate=True, term_stride=vn, stream=stream)
        # shares of u o v'_j for every j, j-stacked
        A0 = torch.empty(m * self.out_elems, dtype=torch.int64, device=self.dev)
        A1 = torch.empty_like(A0)
        self._block_comb(self.S0, k, A0, stream=stream)                                                # MO
        he.pencil_ring_linear(ctx, self.plan_vj, ut, self.v_masks, None, A1, stream=stream)              # DO
        self._block_comb(self.S1, k, A1, addend=A1, stream=stream)
        # shares of u o v
        z0 = torch.empty(self.out_elems, dtype=torch.int64, device=self.dev)
        z1 = torch.empty_like(z0)
        he.pencil_ring_linear(ctx, self.plan, u, vt, None, z0, stream=stream)                           # MO
        he.pencil_lincomb(ctx, A0, l, self.out_elems, z0, addend=z0, term_stride=self.out_elems, stream=stream)
        he.pencil_lincomb(ctx, A1, l, self.out_elems, z1, term_stride=self.out_elems, stream=stream)    # DO
        return ut, vt, z0, z1
