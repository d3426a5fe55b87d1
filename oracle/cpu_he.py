"""ctypes wrapper of oracle/cpu_he.c, the plain CPU build of the HE linear-layer
pipeline (oracle directory: tests and the timed CPU baseline of bench.py only).

The constants that need exact big integers (Delta mod q_j, q mod t, the CRT
factors (q / q_j)^{-1} mod q_j and t / q_j in 0.128 fixed point) are computed
here from the oracle's parameters; the role arrays (padded input, rotated or
transposed kernel of a layer role) come from oracle.protocol.role_input /
role_kernel; everything per coefficient runs in C.  `layer_alg1` and
`layer_alg2` mirror protocol.he_linear and protocol.he_wgrad.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import protocol
from .packing import Partition, counts
from .params import BfvParams
from .sampling import cdt_table

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "cpu_he.c"), os.path.join(HERE, "cpu_ntt.c")]
LIB = os.path.join(HERE, "_build", "libcpu_he.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in SRCS):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    cmd = ["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", *SRCS, "-o", LIB + ".tmp"]
    subprocess.run(cmd, check=True, capture_output=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


class _Geom(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in ("B", "Ci", "Co", "H", "W", "KH", "KW")]


class _Part(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in ("bb", "cib", "cob", "th", "tw", "kth", "ktw")]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P, I, U = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64
        G, Pt = ctypes.POINTER(_Geom), ctypes.POINTER(_Part)
        _lib.cpu_he_create.restype = P
        _lib.cpu_he_create.argtypes = [I, I, P, P, I, U, P, P, P, P, P]
        _lib.cpu_he_destroy.argtypes = [P]
        _lib.cpu_he_keygen.argtypes = [P, U]
        _lib.cpu_he_encode.argtypes = [P, G, Pt, I, P, P, I]
        _lib.cpu_he_encrypt.argtypes = [P, G, Pt, I, P, U, P, I]
        _lib.cpu_he_alg1.argtypes = [P, G, Pt, P, P, P, P, U, I, P, P, I]
        _lib.cpu_he_alg2.argtypes = [P, G, Pt, P, P, P, P, U, P, P, I]
        _lib.cpu_he_decrypt.argtypes = [P, G, Pt, I, P, P, I]
    return _lib


def _u64(a) -> np.ndarray:
    a = np.ascontiguousarray(a)
    return a if a.dtype == np.uint64 else np.ascontiguousarray(a.astype(np.int64).view(np.uint64))


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class CpuHe:
    """One BFV context and secret key of the C pipeline."""

    def __init__(self, p: BfvParams, sk_seed: int):
        self.p = p
        Q, t = p.q, p.t
        qs = p.primes
        arr = lambda v: np.array(v, dtype=np.uint64)
        th = [(1 << (128 + p.t_bits)) // q for q in qs]
        self._keep = [arr(qs), arr(p.psis), arr([(Q // t) % q for q in qs]),
                      arr([pow(Q // q, -1, q) for q in qs]), arr([v >> 64 for v in th]),
                      arr([v & ((1 << 64) - 1) for v in th]), arr(cdt_table(p.sigma))]
        k = self._keep
        self.h = lib().cpu_he_create(p.log_n, len(qs), _ptr(k[0]), _ptr(k[1]), p.t_bits, Q % t, _ptr(k[2]),
                                     _ptr(k[3]), _ptr(k[4]), _ptr(k[5]), _ptr(k[6]))
        if not self.h:
            raise ValueError("unsupported parameters")
        lib().cpu_he_keygen(self.h, sk_seed)

    def __del__(self):
        if getattr(self, "h", None):
            lib().cpu_he_destroy(self.h)
            self.h = None

    # ---------------------------------------------------------------- stages
    def _gp(self, g, part):
        return (ctypes.byref(_Geom(g.B, g.Ci, g.Co, g.H, g.W, g.KH, g.KW)),
                ctypes.byref(_Part(part.bb, part.cib, part.cob, part.th, part.tw, part.kth, part.ktw)))

    def _ln(self):
        return len(self.p.primes), self.p.n

    def encode(self, g, part: Partition, kind: int, src, threads: int = 0) -> np.ndarray:
        """Plaintext multipliers at input (kind 0) or kernel (kind 1) positions: [count][L][N]."""
        c = counts(g, part)
        count = c.ct_in if kind == 0 else c.pt
        out = np.empty((count,) + self._ln(), dtype=np.uint64)
        src = _u64(src)
        lib().cpu_he_encode(self.h, *self._gp(g, part), kind, _ptr(src), _ptr(out), threads)
        return out

    def encrypt(self, g, part: Partition, kind: int, src, seed: int, threads: int = 0) -> np.ndarray:
        """Symmetric encryptions at input (kind 0) or kernel (kind 1) positions: [count][2][L][N]."""
        c = counts(g, part)
        count = c.ct_in if kind == 0 else c.pt
        out = np.empty((count, 2) + self._ln(), dtype=np.uint64)
        src = _u64(src)
        lib().cpu_he_encrypt(self.h, *self._gp(g, part), kind, _ptr(src), seed, _ptr(out), threads)
        return out

    def alg1(self, g, part: Partition, ct_in, pt, V0, bias, mask_seed: int, order: int, out_elems: int,
             threads: int = 0):
        c = counts(g, part)
        ct_out = np.empty((c.ct_out, 2) + self._ln(), dtype=np.uint64)
        y0 = np.empty(out_elems, dtype=np.uint64)
        V0 = None if V0 is None else _u64(V0)
        bias = None if bias is None else _u64(bias)
        lib().cpu_he_alg1(self.h, *self._gp(g, part), _ptr(ct_in), _ptr(pt), None if V0 is None else _ptr(V0),
                          None if bias is None else _ptr(bias), mask_seed, order, _ptr(ct_out), _ptr(y0), threads)
        return ct_out, y0

    def alg2(self, g, part: Partition, ct_x1, pt_gy0, ct_gy1, pt_x0, mask_seed: int, out_elems: int,
             threads: int = 0):
        c = counts(g, part)
        ct_out = np.empty((c.ct_out, 2) + self._ln(), dtype=np.uint64)
        y0 = np.empty(out_elems, dtype=np.uint64)
        lib().cpu_he_alg2(self.h, *self._gp(g, part), _ptr(ct_x1), _ptr(pt_gy0), _ptr(ct_gy1), _ptr(pt_x0),
                          mask_seed, _ptr(ct_out), _ptr(y0), threads)
        return ct_out, y0

    def decrypt(self, g, part: Partition, order: int, ct_out, out_elems: int, threads: int = 0) -> np.ndarray:
        y1 = np.zeros(out_elems, dtype=np.uint64)
        lib().cpu_he_decrypt(self.h, *self._gp(g, part), order, _ptr(ct_out), _ptr(y1), threads)
        return y1

    # ---------------------------------------------------------------- whole protocol steps
    def layer_alg1(self, layer, role: str, part: Partition, kernel, x1, x0, enc_seed: int, mask_seed: int,
                   bias=None, threads: int = 0, with_encode: bool = True, pt=None):
        """Alg. 1 for the forward or input-gradient role: the DO encrypts x1, the MO
        encodes the kernel and evaluates, the DO decrypts.  Returns (y0, y1, ct_in, pt, ct_out)."""
        g = protocol.geometry(layer, role)
        out_elems = int(np.prod(protocol.output_shape(layer, role)))
        if with_encode or pt is None:
            pt = self.encode(g, part, 1, protocol.role_kernel(layer, role, kernel), threads)
        ct_in = self.encrypt(g, part, 0, protocol.role_input(layer, role, _u64(x1)), enc_seed, threads)
        ct_out, y0 = self.alg1(g, part, ct_in, pt, protocol.role_input(layer, role, _u64(x0)),
                               bias if role == protocol.FWD else None, mask_seed, 0, out_elems, threads)
        y1 = self.decrypt(g, part, 0, ct_out, out_elems, threads)
        return y0, y1, ct_in, pt, ct_out

    def layer_alg2(self, layer, part: Partition, gy0, gy1, x0, x1, seed_x: int, seed_g: int, mask_seed: int,
                   threads: int = 0):
        """Alg. 2 cross terms: returns (decrypted tilde, MO mask s, ct_x1, ct_gy1, ct_out)."""
        W = protocol.WGRAD
        g = protocol.geometry(layer, W)
        out_elems = int(np.prod(protocol.output_shape(layer, W)))
        ct_x1 = self.encrypt(g, part, 0, protocol.role_input(layer, W, _u64(x1)), seed_x, threads)
        ct_gy1 = self.encrypt(g, part, 1, protocol.role_kernel(layer, W, _u64(gy1)), seed_g, threads)
        pt_gy0 = self.encode(g, part, 1, protocol.role_kernel(layer, W, _u64(gy0)), threads)
        pt_x0 = self.encode(g, part, 0, protocol.role_input(layer, W, _u64(x0)), threads)
        ct_out, s = self.alg2(g, part, ct_x1, pt_gy0, ct_gy1, pt_x0, mask_seed, out_elems, threads)
        tilde = self.decrypt(g, part, 1, ct_out, out_elems, threads)
        return tilde, s, ct_x1, ct_gy1, ct_out


def max_threads() -> int:
    from .cpu_ntt import max_threads as mt
    return mt()
