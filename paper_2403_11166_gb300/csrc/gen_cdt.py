"""Writes cdt_table.h: the cumulative table used by the CUDA sampler for the
encryption error (discrete Gaussian, sigma = 3.2, support [-19, 19]).

T[j] = floor(2^63 * P(|E| <= j)), j = 0..18, with P(E = x) proportional to
exp(-x^2 / (2 sigma^2)).  Evaluated with Python's decimal module at 80
significant digits (correctly rounded exp), so every entry is exact.

Run:  python paper_2403_11166_gb300/csrc/gen_cdt.py
"""
import os
from decimal import Decimal, getcontext

SIGMA = Decimal("3.2")
TAIL = 19


def table():
    getcontext().prec = 80
    rho = [(-(Decimal(x) ** 2) / (2 * SIGMA * SIGMA)).exp() for x in range(TAIL + 1)]
    z = rho[0] + 2 * sum(rho[1:])
    out, acc = [], Decimal(0)
    for j in range(TAIL):
        acc += rho[0] if j == 0 else 2 * rho[j]
        out.append(int((acc / z * (Decimal(2) ** 63)).to_integral_value(rounding="ROUND_FLOOR")))
    return out


def main():
    vals = table()
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "cdt_table.h"), "w") as f:
        f.write("// Generated by gen_cdt.py: floor(2^63 * P(|E| <= j)) for the discrete Gaussian\n")
        f.write("// with sigma = 3.2 on [-19, 19].  Do not edit.\n#pragma once\n#include <stdint.h>\n")
        f.write(f"#define PENCIL_CDT_LEN {len(vals)}\n")
        f.write("static const uint64_t kPencilCdt[PENCIL_CDT_LEN] = {\n")
        for v in vals:
            f.write(f"    0x{v:016x}ull,\n")
        f.write("};\n")


if __name__ == "__main__":
    main()
