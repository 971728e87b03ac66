"""Writes exp2_table.h: 2^(j/256), j = 0..255, as double-float pairs.

Each value is computed to 60 decimal digits with mpmath and split into
hi = float32(v) and lo = float32(v - hi) (both round to nearest), so
hi + lo is v to about 2^-48 relative.  The table is the 256-entry table of
the table-driven exponential (Tang's method) used by the kernel builds and
the fused prediction.  Run from this directory: python gen_exp2_table.py
"""
import struct

import mpmath


def f32(x):
    """x rounded once to a 24-bit significand (round to nearest even); the
    results here are far from the float32 overflow and subnormal ranges."""
    with mpmath.workprec(24):
        r = +x
    y = float(r)
    assert struct.unpack("<f", struct.pack("<f", y))[0] == y
    return y


def hexf(x):
    return float(x).hex() + "f"


def main():
    mpmath.mp.dps = 60
    lines = ["// Generated by gen_exp2_table.py: 2^(j/256) = hi + lo, j = 0..255, hi and lo",
             "// float32 (round to nearest), computed to 60 digits.  Do not edit.",
             "#pragma once",
             "static __device__ const float2 krr_exp2_tab[256] = {"]
    for j in range(256):
        v = mpmath.power(2, mpmath.mpf(j) / 256)
        hi = f32(v)
        lo = f32(v - mpmath.mpf(hi))
        lines.append("    {%s, %s}," % (hexf(hi), hexf(lo)))
    lines.append("};")
    with open("exp2_table.h", "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
