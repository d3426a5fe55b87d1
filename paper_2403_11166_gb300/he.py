"""Thin ctypes binding of libpencil_he.so (include/pencil_he.h).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels behind the C ABI.  PyTorch supplies device memory and streams.
Shares, ciphertexts and plaintexts travel as torch.int64 tensors holding the
uint64 bit patterns.  Importing this module raises if the library has not been
built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpencil_he.so")

PENCIL_OK = 0
ERRORS = {-1: "PENCIL_E_ARG", -2: "PENCIL_E_SHAPE", -3: "PENCIL_E_PARAMS", -4: "PENCIL_E_CAPACITY",
          -5: "PENCIL_E_NOISE", -6: "PENCIL_E_TIMEOUT", -7: "PENCIL_E_CUDA", -8: "PENCIL_E_UNIMPL"}
FC, CONV = 0, 1
ROLE_FWD, ROLE_DGRAD, ROLE_WGRAD = 0, 1, 2
OPERAND_INPUT, OPERAND_KERNEL = 0, 1

# Every entry point declared in include/pencil_he.h.
EXPORTS = ("pencil_ctx_create", "pencil_ctx_destroy", "pencil_ctx_primes", "pencil_sync_status",
           "pencil_keygen", "pencil_sk_destroy", "pencil_plan_linear", "pencil_plan_destroy",
           "pencil_plan_sizes", "encode_weights", "encrypt_share", "he_linear_forward",
           "he_linear_backward", "decrypt_to_share", "pencil_ntt_batch", "pencil_profile",
           "pencil_profile_read", "pencil_mul_probe", "pencil_ring_linear", "pencil_bias_grad",
           "encrypt_share_noalloc", "pencil_ctx_tune", "pencil_ctx_get_tune", "pencil_batch_create",
           "pencil_batch_destroy", "pencil_batch_workspace", "pencil_batch_bind", "pencil_batch_commit",
           "pencil_batch_forward", "pencil_batch_set_step", "pencil_batch_read", "pencil_batch_withhold",
           "pencil_plan_candidates", "he_linear_forward_prepare", "he_linear_forward_apply", "pencil_plan_slice",
           "pencil_lincomb", "pencil_ctx_flooding", "pencil_pk_keygen", "pencil_pk_destroy",
           "encrypt_share_pk", "compact_returned", "decrypt_compact_to_share",
           "pencil_batch_bind_wgrad", "pencil_lincomb2")
BATCH_PT, BATCH_CT_IN, BATCH_CT_OUT, BATCH_CT_KERNEL = 0, 1, 2, 3
TUNE_NTT_LOG_RADIX = 0
TUNE_MAC_COLUMNS = 1
TUNE_MAC_STAGING = 2
TUNE_NTT_ARITH = 3
KERNEL_NAMES = ("ntt_raw", "intt_raw", "ntt_encrypt", "ntt_addplain", "ntt_encode", "ntt_mask", "intt_decrypt",
                "ntt_keygen", "mac", "mac_dual", "sample_err", "mask_poly", "mo_share", "decrypt_combine",
                "ring", "bias_grad", "ntt_mo_prep", "lincomb", "sample_pk", "ntt_pk_u", "ntt_encrypt_pk",
                "intt_compact")


class PencilError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where} failed: {ERRORS.get(code, code)}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_int32), ("num_primes", ctypes.c_int32),
                ("prime_bits", ctypes.c_int32), ("t_bits", ctypes.c_int32)]


class LayerDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("batch", ctypes.c_int32), ("c_in", ctypes.c_int32),
                ("c_out", ctypes.c_int32), ("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("pad", ctypes.c_int32)]


class Partition(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("bb", "cib", "cob", "th", "tw", "kth", "ktw")]

    def astuple(self):
        return tuple(getattr(self, k) for k, _ in self._fields_)


class PlanSizes(ctypes.Structure):
    _fields_ = [("part", Partition)] + [(k, ctypes.c_int64) for k in (
        "ct_in", "pt", "ct_out", "products", "ct_words", "pt_words", "out_elems",
        "ws_encrypt", "ws_forward", "ws_backward", "ws_decrypt", "ws_encrypt_pk")]


class ProfEntry(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("launches", ctypes.c_int32), ("ms", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2403_11166_gb300.build` "
                          "(the HE hot path has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, U64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
    sig = {
        "pencil_ctx_create": [ctypes.POINTER(Params), ctypes.c_int, ctypes.POINTER(P)],
        "pencil_ctx_destroy": [P],
        "pencil_ctx_primes": [P, P, P],
        "pencil_sync_status": [P, ctypes.POINTER(I32)],
        "pencil_keygen": [P, U64, ctypes.POINTER(P), P],
        "pencil_sk_destroy": [P],
        "pencil_plan_linear": [P, ctypes.POINTER(LayerDesc), I32, ctypes.POINTER(Partition), ctypes.POINTER(P)],
        "pencil_plan_destroy": [P],
        "pencil_plan_slice": [P, I32, I32, ctypes.POINTER(P)],
        "pencil_lincomb": [P, P, I64, I64, I64, I64, P, I32, P, I32, P, I64, P],
        "pencil_lincomb2": [P, P, I64, I64, I64, I64, I32, I64, I32, P, P, I32, P, I64, P],
        "pencil_ctx_flooding": [P, I32],
        "pencil_pk_keygen": [P, P, U64, ctypes.POINTER(P), P],
        "pencil_pk_destroy": [P],
        "encrypt_share_pk": [P, P, P, I32, P, U64, P, P, SZ, P],
        "compact_returned": [P, P, P, P, P],
        "decrypt_compact_to_share": [P, P, P, P, P, P, I32, P, SZ, P],
        "pencil_plan_sizes": [P, ctypes.POINTER(PlanSizes)],
        "encode_weights": [P, P, I32, P, P, P],
        "encrypt_share": [P, P, P, I32, P, U64, P, P, SZ, P],
        "he_linear_forward": [P, P, P, P, P, P, U64, P, P, P, SZ, P],
        "he_linear_forward_prepare": [P, P, P, P, U64, P, P, SZ, P],
        "he_linear_forward_apply": [P, P, P, P, P, P, SZ, P],
        "he_linear_backward": [P, P, P, P, P, P, P, P, P, U64, U64, P, P, P, P, P, SZ, P],
        "decrypt_to_share": [P, P, P, P, P, I32, P, SZ, P],
        "pencil_ntt_batch": [P, P, I64, I32, P],
        "pencil_profile": [P, I32],
        "pencil_profile_read": [P, ctypes.POINTER(ProfEntry), I32, ctypes.POINTER(I32)],
        "pencil_mul_probe": [P, I32, I64, I32, I32, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double), P],
        "pencil_ring_linear": [P, P, P, P, P, P, P, P],
        "pencil_bias_grad": [P, P, P, P, P],
        "encrypt_share_noalloc": [P, P, P, I32, P, U64, P, P],
        "pencil_ctx_tune": [P, I32, I32],
        "pencil_batch_create": [P, ctypes.POINTER(P), I32, ctypes.POINTER(P)],
        "pencil_batch_destroy": [P],
        "pencil_batch_workspace": [P, ctypes.POINTER(I64)],
        "pencil_batch_bind": [P, I32, P, P, P, P, P, P],
        "pencil_batch_bind_wgrad": [P, I32, P, P, P, P, P, P],
        "pencil_batch_commit": [P, P, P, SZ, U64, U64],
        "pencil_batch_forward": [P, P, P],
        "pencil_batch_set_step": [P, U64],
        "pencil_batch_read": [P, I32, I32, P, P],
        "pencil_batch_withhold": [P, I32],
        "pencil_plan_candidates": [P, ctypes.POINTER(LayerDesc), I32, I32, ctypes.POINTER(Partition),
                                   ctypes.POINTER(I32)],
        "pencil_ctx_get_tune": [P, I32, ctypes.POINTER(I32)],
    }
    for name in EXPORTS:
        fn = getattr(lib, name)
        fn.argtypes = sig[name]
        fn.restype = ctypes.c_int
    return lib


lib = _load()


def _check(code: int, where: str):
    if code != PENCIL_OK:
        raise PencilError(code, where)


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_cuda or not t.is_contiguous() or t.dtype not in (torch.int64, torch.uint64):
        raise ValueError("tensors must be contiguous CUDA int64/uint64")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """BFV context (pencil_ctx_create)."""

    def __init__(self, log_n: int, num_primes: int, prime_bits: int, t_bits: int = 41, device: int = 0):
        self.params = Params(log_n, num_primes, prime_bits, t_bits)
        self.device = device
        self.n = 1 << log_n
        self.L = num_primes
        self.t_bits = t_bits
        h = ctypes.c_void_p()
        _check(lib.pencil_ctx_create(ctypes.byref(self.params), device, ctypes.byref(h)), "pencil_ctx_create")
        self.h = h

    def primes(self):
        q = (ctypes.c_uint64 * self.L)()
        r = (ctypes.c_uint64 * self.L)()
        _check(lib.pencil_ctx_primes(self.h, q, r), "pencil_ctx_primes")
        return list(q), list(r)

    def tune(self, knob: int, value: int):
        _check(lib.pencil_ctx_tune(self.h, knob, value), "pencil_ctx_tune")

    def get_tune(self, knob: int) -> int:
        v = ctypes.c_int32()
        _check(lib.pencil_ctx_get_tune(self.h, knob, ctypes.byref(v)), "pencil_ctx_get_tune")
        return v.value

    def sync_status(self) -> int:
        s = ctypes.c_int32()
        _check(lib.pencil_sync_status(self.h, ctypes.byref(s)), "pencil_sync_status")
        return s.value

    def profile(self, enable: bool):
        _check(lib.pencil_profile(self.h, int(enable)), "pencil_profile")

    def profile_read(self) -> dict:
        """{kernel name: (launches, total ms)} for the launches recorded since profile(True)."""
        buf = (ProfEntry * 32)()
        n = ctypes.c_int32()
        _check(lib.pencil_profile_read(self.h, buf, 32, ctypes.byref(n)), "pencil_profile_read")
        return {KERNEL_NAMES[buf[i].kernel]: (buf[i].launches, buf[i].ms) for i in range(n.value)}

    def mul_probe(self, which: int, iters: int, blocks: int, threads: int = 256, stream=None):
        """(ms, chain steps) of the register-only multiply probe (0: mad.lo.u32, 1: Shoup mod-mul)."""
        ms, steps = ctypes.c_double(), ctypes.c_double()
        _check(lib.pencil_mul_probe(self.h, which, iters, blocks, threads, ctypes.byref(ms), ctypes.byref(steps),
                                    _stream(stream)), "pencil_mul_probe")
        return ms.value, steps.value

    def keygen(self, seed: int, stream=None) -> "SecretKey":
        return SecretKey(self, seed, stream)

    def pk_keygen(self, sk: "SecretKey", seed: int, stream=None) -> "PublicKey":
        return PublicKey(self, sk, seed, stream)

    def flooding(self, bits: int):
        """pencil_ctx_flooding: flood the noise of returned ciphertexts (0 = off)."""
        _check(lib.pencil_ctx_flooding(self.h, bits), "pencil_ctx_flooding")

    def close(self):
        if self.h:
            lib.pencil_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SecretKey:
    def __init__(self, ctx: Context, seed: int, stream=None):
        self.ctx = ctx
        h = ctypes.c_void_p()
        _check(lib.pencil_keygen(ctx.h, seed, ctypes.byref(h), _stream(stream)), "pencil_keygen")
        self.h = h

    def __del__(self):
        try:
            if self.h and self.ctx.h:
                lib.pencil_sk_destroy(self.h)
        except Exception:
            pass


class PublicKey:
    def __init__(self, ctx: Context, sk: SecretKey, seed: int, stream=None):
        self.ctx = ctx
        h = ctypes.c_void_p()
        _check(lib.pencil_pk_keygen(ctx.h, sk.h, seed, ctypes.byref(h), _stream(stream)), "pencil_pk_keygen")
        self.h = h

    def __del__(self):
        try:
            if self.h and self.ctx.h:
                lib.pencil_pk_destroy(self.h)
        except Exception:
            pass


@dataclass
class Layer:
    kind: int
    batch: int
    c_in: int
    c_out: int
    height: int = 1
    width: int = 1
    kernel: int = 1
    pad: int = 0

    def desc(self) -> LayerDesc:
        return LayerDesc(self.kind, self.batch, self.c_in, self.c_out, self.height, self.width,
                         self.kernel, self.pad)


class Plan:
    """pencil_plan_linear for one role; `part` = None lets the planner choose."""

    def __init__(self, ctx: Context, layer: Layer, role: int, part=None):
        self.ctx = ctx
        self.layer = layer
        self.role = role
        d = layer.desc()
        pp = ctypes.byref(Partition(*part)) if part is not None else None
        h = ctypes.c_void_p()
        _check(lib.pencil_plan_linear(ctx.h, ctypes.byref(d), role, pp, ctypes.byref(h)), "pencil_plan_linear")
        self.h = h
        s = PlanSizes()
        _check(lib.pencil_plan_sizes(h, ctypes.byref(s)), "pencil_plan_sizes")
        self.sizes = s
        self.part = s.part.astuple()
        self.parent = None
        self.row_range = None

    @property
    def rows(self) -> int:
        """M, the output rows of the partition (ct_in = M K, pt = K NC, ct_out = M NC)."""
        S = self.sizes
        return math.isqrt(S.ct_in * S.ct_out // S.pt)

    def slice(self, m_first: int, m_count: int) -> "Plan":
        """pencil_plan_slice: the output rows [m_first, m_first + m_count) of this plan (same
        buffers and workspaces; keeps this plan alive)."""
        h = ctypes.c_void_p()
        _check(lib.pencil_plan_slice(self.h, m_first, m_count, ctypes.byref(h)), "pencil_plan_slice")
        sl = Plan.__new__(Plan)
        sl.ctx, sl.layer, sl.role, sl.h = self.ctx, self.layer, self.role, h
        sl.sizes, sl.part, sl.parent, sl.row_range = self.sizes, self.part, self, (m_first, m_count)
        return sl

    def new_ct(self, count: int) -> torch.Tensor:
        return torch.empty((count, 2, self.ctx.L, self.ctx.n), dtype=torch.int64, device=f"cuda:{self.ctx.device}")

    def new_pt(self, count: int) -> torch.Tensor:
        return torch.empty((count, self.ctx.L, self.ctx.n), dtype=torch.int64, device=f"cuda:{self.ctx.device}")

    def new_ws(self, nbytes: int) -> torch.Tensor:
        words = max(2, (int(nbytes) + 7) // 8)
        return torch.empty(words, dtype=torch.int64, device=f"cuda:{self.ctx.device}")

    def __del__(self):
        try:
            if self.h and self.ctx.h:
                lib.pencil_plan_destroy(self.h)
        except Exception:
            pass


def _ws(ws):
    return _ptr(ws), ctypes.c_size_t(ws.numel() * 8)


def encode_weights(ctx: Context, plan: Plan, operand: int, values: torch.Tensor, pt: torch.Tensor, stream=None):
    _check(lib.encode_weights(ctx.h, plan.h, operand, _ptr(values), _ptr(pt), _stream(stream)), "encode_weights")


def encrypt_share(ctx: Context, sk: SecretKey, plan: Plan, operand: int, share: torch.Tensor, seed: int,
                  ct: torch.Tensor, ws: torch.Tensor, stream=None):
    w, nb = _ws(ws)
    _check(lib.encrypt_share(ctx.h, sk.h, plan.h, operand, _ptr(share), seed, _ptr(ct), w, nb, _stream(stream)),
           "encrypt_share")


def encrypt_share_pk(ctx: Context, pk: PublicKey, plan: Plan, operand: int, share: torch.Tensor, seed: int,
                     ct: torch.Tensor, ws: torch.Tensor, stream=None):
    w, nb = _ws(ws)
    _check(lib.encrypt_share_pk(ctx.h, pk.h, plan.h, operand, _ptr(share), seed, _ptr(ct), w, nb, _stream(stream)),
           "encrypt_share_pk")


def he_linear_forward(ctx: Context, plan: Plan, ct_in, pt, x0, bias, mask_seed: int, ct_out, y0, ws, stream=None):
    w, nb = _ws(ws)
    _check(lib.he_linear_forward(ctx.h, plan.h, _ptr(ct_in), _ptr(pt), _ptr(x0), _ptr(bias), mask_seed,
                                 _ptr(ct_out), _ptr(y0), w, nb, _stream(stream)), "he_linear_forward")


def he_linear_forward_prepare(ctx: Context, plan: Plan, x0, bias, mask_seed: int, y0, ws, stream=None):
    w, nb = _ws(ws)
    _check(lib.he_linear_forward_prepare(ctx.h, plan.h, _ptr(x0), _ptr(bias), mask_seed, _ptr(y0), w, nb,
                                         _stream(stream)), "he_linear_forward_prepare")


def he_linear_forward_apply(ctx: Context, plan: Plan, ct_in, pt, ct_out, ws, stream=None):
    w, nb = _ws(ws)
    _check(lib.he_linear_forward_apply(ctx.h, plan.h, _ptr(ct_in), _ptr(pt), _ptr(ct_out), w, nb, _stream(stream)),
           "he_linear_forward_apply")


def pencil_lincomb(ctx: Context, src, scalars, count: int, out, addend=None, negate: bool = False,
                   src_offset: int = 0, inner: int = None, outer_stride: int = 0, term_stride: int = 0, stream=None):
    """out[e] = addend[e] +/- sum_i scalars[i] src[src_offset + (e // inner) outer_stride + e % inner
    + i term_stride] mod t (see pencil_lincomb in the header)."""
    ks = (ctypes.c_uint64 * max(1, len(scalars)))(*[int(v) for v in scalars])
    _check(lib.pencil_lincomb(ctx.h, _ptr(src), src_offset, count if inner is None else inner, outer_stride,
                              term_stride, ks, len(scalars), _ptr(addend), int(negate), _ptr(out), count,
                              _stream(stream)), "pencil_lincomb")


def pencil_lincomb2(ctx: Context, src, scalars, terms: int, terms2: int, count: int, out, addend=None,
                    negate: bool = False, src_offset: int = 0, inner: int = None, outer_stride: int = 0,
                    term_stride: int = 0, term_stride2: int = 0, stream=None):
    """out[e] = addend[e] +/- sum_{i2, i} scalars[i2 * terms + i] src[src_offset + (e // inner) outer_stride
    + e % inner + i term_stride + i2 term_stride2] mod t (see pencil_lincomb2 in the header)."""
    ks = (ctypes.c_uint64 * max(1, len(scalars)))(*[int(v) for v in scalars])
    _check(lib.pencil_lincomb2(ctx.h, _ptr(src), src_offset, count if inner is None else inner, outer_stride,
                               term_stride, terms, term_stride2, terms2, ks, _ptr(addend), int(negate), _ptr(out),
                               count, _stream(stream)), "pencil_lincomb2")


def he_linear_backward(ctx: Context, plan_dgrad, plan_wgrad, ct_gy1_d, pt_wt, ct_x1_w, ct_gy1_w, gy0, x0,
                       mask_seed_x: int, mask_seed_w: int, ct_gx, gx0, ct_gw, gw_mask, ws, stream=None):
    w, nb = _ws(ws)
    _check(lib.he_linear_backward(
        ctx.h, plan_dgrad.h if plan_dgrad is not None else None, plan_wgrad.h if plan_wgrad is not None else None,
        _ptr(ct_gy1_d), _ptr(pt_wt), _ptr(ct_x1_w), _ptr(ct_gy1_w), _ptr(gy0), _ptr(x0), mask_seed_x, mask_seed_w,
        _ptr(ct_gx), _ptr(gx0), _ptr(ct_gw), _ptr(gw_mask), w, nb, _stream(stream)), "he_linear_backward")


def decrypt_to_share(ctx: Context, sk: SecretKey, plan: Plan, ct_out, y1, check_noise: bool, ws, stream=None):
    w, nb = _ws(ws)
    _check(lib.decrypt_to_share(ctx.h, sk.h, plan.h, _ptr(ct_out), _ptr(y1), int(check_noise), w, nb,
                                _stream(stream)), "decrypt_to_share")


def compact_returned(ctx: Context, plan: Plan, ct_out, c0c, stream=None):
    """MO: c0 of the returned ciphertexts at their output coefficients only,
    c0c[limb][flat] (int64 tensor of L x out_elems)."""
    _check(lib.compact_returned(ctx.h, plan.h, _ptr(ct_out), _ptr(c0c), _stream(stream)), "compact_returned")


def decrypt_compact_to_share(ctx: Context, sk: SecretKey, plan: Plan, ct_out, c0c, y1, check: bool, ws,
                             stream=None):
    w, nb = _ws(ws)
    _check(lib.decrypt_compact_to_share(ctx.h, sk.h, plan.h, _ptr(ct_out), _ptr(c0c), _ptr(y1), 1 if check else 0,
                                        w, nb, _stream(stream)), "decrypt_compact_to_share")


def pencil_ntt_batch(ctx: Context, polys: torch.Tensor, inverse: bool, stream=None):
    count = polys.numel() // (ctx.L * ctx.n)
    _check(lib.pencil_ntt_batch(ctx.h, _ptr(polys), count, int(inverse), _stream(stream)), "pencil_ntt_batch")


def pencil_ring_linear(ctx: Context, plan: Plan, kernel_operand, input_operand, addend, out, addend2=None,
                       stream=None):
    _check(lib.pencil_ring_linear(ctx.h, plan.h, _ptr(kernel_operand), _ptr(input_operand), _ptr(addend),
                                  _ptr(addend2), _ptr(out), _stream(stream)), "pencil_ring_linear")


def pencil_bias_grad(ctx: Context, plan: Plan, g, out, stream=None):
    _check(lib.pencil_bias_grad(ctx.h, plan.h, _ptr(g), _ptr(out), _stream(stream)), "pencil_bias_grad")


def encrypt_share_noalloc(ctx: Context, sk: SecretKey, plan: Plan, operand: int, share: torch.Tensor, seed: int,
                          ct: torch.Tensor, stream=None):
    """encrypt_share without a workspace: for callers that may not allocate device
    memory while encrypting.  Its scratch is a static 8 MiB device array in the
    library (count x N bytes at most), shared by every call on a device: calls must
    not overlap on the GPU.  The first call on a device should precede any stream
    capture."""
    _check(lib.encrypt_share_noalloc(ctx.h, sk.h, plan.h, operand, _ptr(share), seed, _ptr(ct), _stream(stream)),
           "encrypt_share_noalloc")


class Batch:
    """Many plans of one context (forward, input-gradient and weight-gradient
    products) as one fixed launch sequence (pencil_batch_*)."""

    def __init__(self, ctx: Context, plans):
        self.ctx = ctx
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.h.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(lib.pencil_batch_create(ctx.h, arr, len(self.plans), ctypes.byref(h)), "pencil_batch_create")
        self.h = h
        b = ctypes.c_int64()
        _check(lib.pencil_batch_workspace(h, ctypes.byref(b)), "pencil_batch_workspace")
        self.workspace_bytes = b.value
        self._keep = []

    def bind(self, layer: int, W, x1, x0, bias, y0, y1):
        self._keep.append((W, x1, x0, bias, y0, y1))
        _check(lib.pencil_batch_bind(self.h, layer, _ptr(W), _ptr(x1), _ptr(x0), _ptr(bias), _ptr(y0), _ptr(y1)),
               "pencil_batch_bind")

    def bind_wgrad(self, layer: int, gy0, gy1, x0, x1, gw_mask, tilde):
        self._keep.append((gy0, gy1, x0, x1, gw_mask, tilde))
        _check(lib.pencil_batch_bind_wgrad(self.h, layer, _ptr(gy0), _ptr(gy1), _ptr(x0), _ptr(x1), _ptr(gw_mask),
                                           _ptr(tilde)), "pencil_batch_bind_wgrad")

    def commit(self, sk: SecretKey, ws: torch.Tensor, enc_seed: int, mask_seed: int):
        self._ws = ws
        _check(lib.pencil_batch_commit(self.h, sk.h, _ptr(ws), ctypes.c_size_t(ws.numel() * 8), enc_seed, mask_seed),
               "pencil_batch_commit")

    def forward(self, stream=None):
        _check(lib.pencil_batch_forward(self.ctx.h, self.h, _stream(stream)), "pencil_batch_forward")

    def set_step(self, step: int):
        _check(lib.pencil_batch_set_step(self.h, step), "pencil_batch_set_step")

    def read(self, layer: int, which: int, dst: torch.Tensor, stream=None):
        _check(lib.pencil_batch_read(self.h, layer, which, _ptr(dst), _stream(stream)), "pencil_batch_read")

    def withhold(self, layer: int):
        _check(lib.pencil_batch_withhold(self.h, layer), "pencil_batch_withhold")

    def __del__(self):
        try:
            if self.h and self.ctx.h:
                lib.pencil_batch_destroy(self.h)
        except Exception:
            pass


def plan_candidates(ctx: Context, layer: Layer, role: int, max_count: int = 8):
    """Cheapest-first partitions of the planner's cost model (tuples)."""
    out = (Partition * max_count)()
    n = ctypes.c_int32()
    d = layer.desc()
    _check(lib.pencil_plan_candidates(ctx.h, ctypes.byref(d), role, max_count, out, ctypes.byref(n)),
           "pencil_plan_candidates")
    return [out[i].astuple() for i in range(n.value)]
