"""torch.autograd wrappers of the secure linear layers (Sec. 3.1-3.2).

`HeLinearFn` is a `torch.autograd.Function` whose forward pass is Algorithm 1
and whose backward pass is the input-gradient protocol of Sec. 3.2.2 plus
Algorithm 2, all through the C ABI (`he.py`).  It takes and returns float64
tensors holding fixed-point values: the fixed-point encoding, the additive
sharing of the inputs and the reconstruction of the outputs stand in for the
2PC machinery around the linear layers (the OT-based non-linear protocols of
Appendix B are outside this hot path and are simulated on reconstructed
plaintext, exactly: see `SecureCNN`).

Fixed point (Sec. 2.3): x -> floor(x 2^f) mod t; a product carries 2f fractional
bits; the next layer's encode floor(y 2^f) is the exact arithmetic right shift
by f of the signed product (the truncation of Appendix B without its 1-bit
error).  Gradients are encoded with round-to-nearest floor(g 2^f + 1/2): at
f = 12 the floor's half-unit bias, summed over a convolution's batch and
positions, would exceed the gradient itself; callers scale the loss (e.g. by
2^10) as in mixed-precision training.  Scales: y, grad_X, grad_W at 2f bits;
grad_b at f bits.
"""
from __future__ import annotations

from typing import Dict, Optional, Tuple

import torch

from . import he


class HeSession:
    """One data owner / model owner pair on one GPU: the BFV context, the DO's
    secret key, plans per (layer, role), one growing workspace, and the seeds
    of every encryption and mask.  Counts the ciphertext bytes each party sends."""

    def __init__(self, log_n: int = 13, num_primes: int = 3, prime_bits: int = 60, t_bits: int = 41,
                 frac_bits: int = 12, seed: int = 0, device: int = 0,
                 partitions: Optional[Dict[Tuple, Tuple]] = None):
        self.ctx = he.Context(log_n, num_primes, prime_bits, t_bits, device)
        self.sk = self.ctx.keygen(seed * 7919 + 1)
        self.t_bits, self.f = t_bits, frac_bits
        self.mask = (1 << t_bits) - 1
        self.device = torch.device(f"cuda:{device}")
        self.gen = torch.Generator(device=self.device)
        self.gen.manual_seed(seed)
        self._seed = (seed + 1) << 24
        self.plans: Dict[Tuple, he.Plan] = {}
        self.partitions = partitions or {}
        self._ws: Optional[torch.Tensor] = None
        self.record = False
        self.trace: list = []
        self.bytes_do_to_mo = 0
        self.bytes_mo_to_do = 0

    # ------------------------------------------------------------ plumbing
    def next_seed(self) -> int:
        self._seed += 1
        return self._seed

    def plan(self, layer: he.Layer, role: int) -> he.Plan:
        key = (layer.kind, layer.batch, layer.c_in, layer.c_out, layer.height, layer.width, layer.kernel,
               layer.pad, role)
        if key not in self.plans:
            self.plans[key] = he.Plan(self.ctx, layer, role, self.partitions.get(key))
        return self.plans[key]

    def ws(self, nbytes: int) -> torch.Tensor:
        if self._ws is None or self._ws.numel() * 8 < nbytes:
            self._ws = torch.empty(max(2, (int(nbytes) + 7) // 8), dtype=torch.int64, device=self.device)
        return self._ws

    # ------------------------------------------------------------ fixed point and sharing (simulated 2PC glue)
    def encode(self, x: torch.Tensor, frac: int) -> torch.Tensor:
        return torch.floor(x.double() * (1 << frac)).to(torch.int64) & self.mask

    def encode_grad(self, g: torch.Tensor, frac: int) -> torch.Tensor:
        return torch.floor(g.double() * (1 << frac) + 0.5).to(torch.int64) & self.mask

    def decode(self, r: torch.Tensor, frac: int) -> torch.Tensor:
        s = torch.where(r >= (1 << (self.t_bits - 1)), r - (1 << self.t_bits), r)
        return s.double() / (1 << frac)

    def share(self, r: torch.Tensor):
        r1 = torch.randint(0, 1 << self.t_bits, r.shape, generator=self.gen, device=self.device,
                           dtype=torch.int64)
        return (r - r1) & self.mask, r1

    def reconstruct(self, a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
        return (a + b) & self.mask

    # ------------------------------------------------------------ protocol steps (all on the GPU through the C ABI)
    def forward(self, layer: he.Layer, w_r: torch.Tensor, b_r: Optional[torch.Tensor], x0: torch.Tensor,
                x1: torch.Tensor):
        """Algorithm 1: returns the MO share y0 = s + b and the DO share y1 = W o X - s."""
        ctx, sk = self.ctx, self.sk
        plan = self.plan(layer, he.ROLE_FWD)
        S = plan.sizes
        ws = self.ws(max(S.ws_encrypt, S.ws_forward, S.ws_decrypt))
        pt = plan.new_pt(S.pt)
        he.encode_weights(ctx, plan, he.OPERAND_KERNEL, w_r.contiguous(), pt)                        # MO
        ct_in = plan.new_ct(S.ct_in)
        he.encrypt_share(ctx, sk, plan, he.OPERAND_INPUT, x1.contiguous(), self.next_seed(), ct_in, ws)  # DO
        ct_out = plan.new_ct(S.ct_out)
        y0 = torch.empty(S.out_elems, dtype=torch.int64, device=self.device)
        he.he_linear_forward(ctx, plan, ct_in, pt, x0.contiguous(), None if b_r is None else b_r.contiguous(),
                             self.next_seed(), ct_out, y0, ws)                                        # MO
        y1 = torch.empty_like(y0)
        he.decrypt_to_share(ctx, sk, plan, ct_out, y1, True, ws)                                      # DO
        self.bytes_do_to_mo += ct_in.numel() * 8
        self.bytes_mo_to_do += ct_out.numel() * 8
        return y0, y1

    def backward(self, layer: he.Layer, w_r: torch.Tensor, x0: torch.Tensor, x1: torch.Tensor,
                 g0: torch.Tensor, g1: torch.Tensor, need_dx: bool):
        """grad_X by the Alg.-1-like protocol (shares) and grad_W by Alg. 2 (revealed to the MO)."""
        ctx, sk = self.ctx, self.sk
        pd = self.plan(layer, he.ROLE_DGRAD) if need_dx else None
        pw = self.plan(layer, he.ROLE_WGRAD)
        sizes = [p.sizes for p in (pd, pw) if p is not None]
        need = max(max(S.ws_encrypt, S.ws_decrypt) for S in sizes)
        need = max(need, sum(S.ws_backward for S in sizes))
        ws = self.ws(need)
        g0, g1, x0, x1 = g0.contiguous(), g1.contiguous(), x0.contiguous(), x1.contiguous()
        ct_gy1_d = pt_wt = ct_gx = gx0 = None
        if pd is not None:
            ct_gy1_d = pd.new_ct(pd.sizes.ct_in)
            he.encrypt_share(ctx, sk, pd, he.OPERAND_INPUT, g1, self.next_seed(), ct_gy1_d, ws)         # DO
            pt_wt = pd.new_pt(pd.sizes.pt)
            he.encode_weights(ctx, pd, he.OPERAND_KERNEL, w_r.contiguous(), pt_wt)                      # MO
            ct_gx = pd.new_ct(pd.sizes.ct_out)
            gx0 = torch.empty(pd.sizes.out_elems, dtype=torch.int64, device=self.device)
            self.bytes_do_to_mo += ct_gy1_d.numel() * 8
            self.bytes_mo_to_do += ct_gx.numel() * 8
        Sw = pw.sizes
        ct_x1 = pw.new_ct(Sw.ct_in)
        he.encrypt_share(ctx, sk, pw, he.OPERAND_INPUT, x1, self.next_seed(), ct_x1, ws)                # DO
        ct_g1 = pw.new_ct(Sw.pt)
        he.encrypt_share(ctx, sk, pw, he.OPERAND_KERNEL, g1, self.next_seed(), ct_g1, ws)               # DO
        ct_gw = pw.new_ct(Sw.ct_out)
        gw_mask = torch.empty(Sw.out_elems, dtype=torch.int64, device=self.device)
        he.he_linear_backward(ctx, pd, pw, ct_gy1_d, pt_wt, ct_x1, ct_g1, g0, x0, self.next_seed(),
                              self.next_seed(), ct_gx, gx0, ct_gw, gw_mask, ws)                         # MO
        self.bytes_do_to_mo += (ct_x1.numel() + ct_g1.numel()) * 8
        self.bytes_mo_to_do += ct_gw.numel() * 8
        gx1 = None
        if pd is not None:
            gx1 = torch.empty_like(gx0)
            he.decrypt_to_share(ctx, sk, pd, ct_gx, gx1, True, ws)                                      # DO
        tilde = torch.empty(Sw.out_elems, dtype=torch.int64, device=self.device)
        he.decrypt_to_share(ctx, sk, pw, ct_gw, tilde, True, ws)                                        # DO
        he.pencil_ring_linear(ctx, pw, g1, x1, tilde, tilde)                # DO adds <gY>_1 (.) <X>_1 (Alg. 2 step 4)
        gw = torch.empty_like(tilde)
        he.pencil_ring_linear(ctx, pw, g0, x0, tilde, gw, addend2=gw_mask)  # MO adds s and its local term (step 6)
        fwd = self.plan(layer, he.ROLE_FWD)
        gb0 = torch.empty(layer.c_out, dtype=torch.int64, device=self.device)
        gb1 = torch.empty_like(gb0)
        he.pencil_bias_grad(ctx, fwd, g0, gb0)                              # each party sums its share
        he.pencil_bias_grad(ctx, fwd, g1, gb1)
        self.bytes_do_to_mo += gb1.numel() * 8 + tilde.numel() * 8
        return gx0, gx1, gw, self.reconstruct(gb0, gb1)


class HeLinearFn(torch.autograd.Function):
    """y = W o x + b over secret shares: forward = Algorithm 1, backward = Sec. 3.2.2
    (grad_X by an Alg.-1-like protocol, grad_W by Algorithm 2, grad_b by local sums)."""

    @staticmethod
    def forward(fctx, x, weight, bias, sess: HeSession, layer: he.Layer, name: str = ""):
        f = sess.f
        X = sess.encode(x, f)
        W = sess.encode(weight, f)
        B = sess.encode(bias, 2 * f) if bias is not None else None
        x0, x1 = sess.share(X)
        y0, y1 = sess.forward(layer, W, B, x0, x1)
        Y = sess.reconstruct(y0, y1)
        out_shape = (layer.batch, layer.c_out) if layer.kind == he.FC else (
            layer.batch, layer.c_out, layer.height + 2 * layer.pad - layer.kernel + 1,
            layer.width + 2 * layer.pad - layer.kernel + 1)
        fctx.save_for_backward(x0, x1, W)
        fctx.sess, fctx.layer, fctx.name = sess, layer, name
        fctx.has_bias = bias is not None
        if sess.record:
            sess.trace.append({"name": name, "pass": "fwd", "X": X, "W": W, "Y": Y.view(out_shape)})
        return sess.decode(Y, 2 * f).view(out_shape)

    @staticmethod
    def backward(fctx, gy):
        sess, layer = fctx.sess, fctx.layer
        x0, x1, W = fctx.saved_tensors
        f = sess.f
        G = sess.encode_grad(gy.contiguous(), f)
        g0, g1 = sess.share(G)
        need_dx = bool(fctx.needs_input_grad[0])
        gx0, gx1, gw, gb = sess.backward(layer, W, x0, x1, g0, g1, need_dx)
        gx = None
        GX = None
        if need_dx:
            GX = sess.reconstruct(gx0, gx1)
            gx = sess.decode(GX, 2 * f).view(x0.shape)
        gw_f = sess.decode(gw, 2 * f).view(W.shape)
        gb_f = sess.decode(gb, f) if fctx.has_bias else None
        if sess.record:
            sess.trace.append({"name": fctx.name, "pass": "bwd", "G": G, "GX": None if GX is None else GX.view(x0.shape),
                               "GW": gw.view(W.shape), "GB": gb})
        return gx, gw_f, gb_f, None, None, None


def he_linear(x, weight, bias, sess: HeSession, layer: he.Layer, name: str = ""):
    return HeLinearFn.apply(x, weight, bias, sess, layer, name)


def relu_ge(x: torch.Tensor) -> torch.Tensor:
    """ReLU with DReLU = 1{x >= 0} (the most-significant-bit rule of Appendix B),
    including its backward pass: grad * 1{x >= 0}."""
    return _ReluGe.apply(x)


class _ReluGe(torch.autograd.Function):
    @staticmethod
    def forward(fctx, x):
        m = x >= 0
        fctx.save_for_backward(m)
        return torch.where(m, x, torch.zeros_like(x))

    @staticmethod
    def backward(fctx, g):
        (m,) = fctx.saved_tensors
        return torch.where(m, g, torch.zeros_like(g))


class SecureCNN(torch.nn.Module):
    """conv3x3 3->16, ReLU, conv3x3 16->32, avgpool 2, FC (32 (H/2) (W/2)) -> classes,
    every linear layer through HeLinearFn; ReLU / AvgPool on reconstructed
    plaintext (the OT protocols of Appendix B are simulated exactly)."""

    def __init__(self, sess: HeSession, batch: int, params: dict, height: int = 32, width: int = 32):
        """params: float64 arrays w1 (c1, c0, 3, 3), b1, w2 (c2, c1, 3, 3), b2, w3 (classes, c2 H W / 4), b3."""
        super().__init__()
        self.sess = sess

        def p(name):
            return torch.nn.Parameter(torch.as_tensor(params[name], dtype=torch.float64).to(sess.device))
        self.w1, self.b1, self.w2, self.b2, self.w3, self.b3 = (p(k) for k in ("w1", "b1", "w2", "b2", "w3", "b3"))
        c1, c0 = self.w1.shape[:2]
        c2 = self.w2.shape[0]
        classes, fc_in = self.w3.shape
        self.l1 = he.Layer(he.CONV, batch, c0, c1, height, width, 3, 1)
        self.l2 = he.Layer(he.CONV, batch, c1, c2, height, width, 3, 1)
        self.l3 = he.Layer(he.FC, batch, fc_in, classes)

    def forward(self, x):
        s = self.sess
        h = relu_ge(he_linear(x, self.w1, self.b1, s, self.l1, "conv1"))
        h = he_linear(h, self.w2, self.b2, s, self.l2, "conv2")
        h = torch.nn.functional.avg_pool2d(h, 2)
        h = h.reshape(h.shape[0], -1)
        return he_linear(h, self.w3, self.b3, s, self.l3, "fc")
