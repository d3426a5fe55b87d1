"""ctypes wrapper of oracle/cpu_ntt.c, the plain CPU NTT baseline (oracle
directory: tests and the timed CPU baseline of bench.py only)."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_ntt.c")
LIB = os.path.join(HERE, "_build", "libcpu_ntt.so")


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    cmd = ["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", SRC, "-o", LIB + ".tmp"]
    subprocess.run(cmd, check=True, capture_output=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P, I, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_long
        U = ctypes.c_uint64
        _lib.cpu_ntt_tables.argtypes = [U, U, I, P, P, P, P]
        _lib.cpu_ntt_batch.argtypes = [P, L, I, U, P, P, P, P, I, I]
        _lib.cpu_ntt_max_threads.restype = I
    return _lib


class CpuNtt:
    def __init__(self, q: int, psi: int, log_n: int):
        self.q, self.log_n, self.n = q, log_n, 1 << log_n
        self.tabs = [np.zeros(self.n, dtype=np.uint64) for _ in range(4)]
        lib().cpu_ntt_tables(q, psi, log_n, *[t.ctypes.data for t in self.tabs])

    def run(self, a: np.ndarray, inverse: bool = False, threads: int = 0) -> None:
        """In place on a C-contiguous uint64 array [count][N]."""
        assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"] and a.shape[-1] == self.n
        lib().cpu_ntt_batch(a.ctypes.data, a.size // self.n, self.log_n, self.q, *[t.ctypes.data for t in self.tabs],
                            int(inverse), threads)


def max_threads() -> int:
    return lib().cpu_ntt_max_threads()
