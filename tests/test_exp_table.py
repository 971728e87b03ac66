"""The double-float table of 2^(j/256) that the kernels' exponential reads
(csrc/exp2_table.h) is correct: hi is 2^(j/256) rounded to float32, lo is the
remainder rounded to float32, and hi + lo is within 2^-47 relative of the
value computed independently here with 50-digit decimal arithmetic."""
import math
import os
import re
import struct
from decimal import ROUND_HALF_EVEN, Decimal, getcontext

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1805_00569_gb300", "csrc", "exp2_table.h")


def f32(x: float) -> float:
    return struct.unpack("<f", struct.pack("<f", x))[0]


def round_f32(d: Decimal) -> float:
    """d rounded to a 24-bit significand, ties to even (normal range only)."""
    if d == 0:
        return 0.0
    a = abs(d)
    e = math.frexp(float(a))[1] - 1
    while Decimal(2) ** e > a:
        e -= 1
    while Decimal(2) ** (e + 1) <= a:
        e += 1
    m = int((a / Decimal(2) ** (e - 23)).to_integral_value(rounding=ROUND_HALF_EVEN))
    return math.copysign(math.ldexp(m, e - 23), float(d))


def test_exp2_table_values():
    getcontext().prec = 50
    pairs = re.findall(r"\{(\S+)f, (\S+)f\}", open(HDR).read())
    assert len(pairs) == 256
    for j, (h, l) in enumerate(pairs):
        hi, lo = float.fromhex(h), float.fromhex(l)
        assert f32(hi) == hi and f32(lo) == lo
        v = Decimal(2) ** (Decimal(j) / Decimal(256))
        assert hi == round_f32(v)
        assert lo == round_f32(v - Decimal(hi))
        err = abs(Decimal(hi) + Decimal(lo) - v) / v
        assert err < Decimal(2) ** -47, (j, err)
