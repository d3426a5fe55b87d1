"""Seeded synthetic inputs (no arithmetic of the method lives here).

Workload recipe: activations and weights are N(0, 1) samples clipped to +-8
and put in fixed point with f = 12 fractional bits (floor(x * 2^f), Sec. 2.3);
secret shares and masks are uniform in Z_t with t = 2^41.  Everything comes
from numpy's PCG64 `default_rng(seed)`.  Used by the tests and by bench.py.
"""
from __future__ import annotations

import numpy as np

T_BITS = 41
FRAC_BITS = 12


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def gaussian_fixed(g: np.random.Generator, shape, frac_bits: int = FRAC_BITS,
                   clip: float = 8.0, scale: float = 1.0) -> np.ndarray:
    """floor(clip(N(0, scale^2), -clip, clip) * 2^frac_bits) as int64."""
    x = np.clip(g.standard_normal(shape) * scale, -clip, clip)
    return np.floor(x * (1 << frac_bits)).astype(np.int64)


def uniform_zt(g: np.random.Generator, shape, t_bits: int = T_BITS) -> np.ndarray:
    """Uniform values in [0, 2^t_bits) as uint64."""
    return g.integers(0, 1 << t_bits, size=shape, dtype=np.uint64)


def split_shares(g: np.random.Generator, x: np.ndarray, t_bits: int = T_BITS):
    """Additive sharing over Z_t: returns (x0, x1) with x1 uniform and
    x0 = x - x1 mod 2^t_bits (both uint64)."""
    x1 = uniform_zt(g, np.shape(x), t_bits)
    xu = np.asarray(x).astype(np.int64).view(np.uint64)
    with np.errstate(over="ignore"):
        x0 = (xu - x1) & np.uint64((1 << t_bits) - 1)
    return x0, x1
