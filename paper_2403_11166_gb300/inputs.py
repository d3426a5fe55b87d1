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


def cnn_params(seed: int, channels=(3, 16, 32), height: int = 32, width: int = 32, classes: int = 10,
               frac_bits: int = FRAC_BITS) -> dict:
    """Weights of the 3-layer CNN workload: N(0, 1/fan_in) rounded down to the
    fixed-point grid, zero biases (float64 numpy arrays)."""
    g = rng(seed)
    c0, c1, c2 = channels
    fc_in = c2 * (height // 2) * (width // 2)

    def w(shape, fan):
        return np.floor(g.standard_normal(shape) / np.sqrt(fan) * (1 << frac_bits)) / (1 << frac_bits)
    return {"w1": w((c1, c0, 3, 3), c0 * 9), "b1": np.zeros(c1), "w2": w((c2, c1, 3, 3), c1 * 9),
            "b2": np.zeros(c2), "w3": w((classes, fc_in), fc_in), "b3": np.zeros(classes)}
