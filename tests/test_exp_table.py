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


def _bits(x: float) -> int:
    """Significant bits of a binary float."""
    m, _ = math.frexp(abs(x))
    n = 0
    while m:
        m = m * 2 - int(m * 2)
        n += 1
    return n


def test_range_reduction_constants():
    """The exponential splits ln2/256 = C1 + C2 + C3 with C1 short enough that
    n C1 is exact for |n| < 2^15 (arguments down to -87), C2 and C3 float32,
    and the three together within 2^-56 relative of ln2/256: for |x| <= 87
    the reduced argument is then off by at most 87 * 2^-56 ~ 1.2e-15, far
    below the exponential's ~7e-13 relative error."""
    getcontext().prec = 50
    src = open(os.path.join(ROOT, "paper_1805_00569_gb300", "csrc", "common.cuh")).read()
    m = re.search(r"C1 = (\S+)f, C2 = (\S+)f, C3 = (\S+)f;", src)
    c1, c2, c3 = (float.fromhex(v) for v in m.groups())
    assert all(f32(c) == c for c in (c1, c2, c3))
    assert _bits(c1) + 15 <= 24  # n C1 exact in float32
    ln2_256 = Decimal(2).ln() / 256
    assert abs(Decimal(c1) + Decimal(c2) + Decimal(c3) - ln2_256) / ln2_256 < Decimal(2) ** -56
    m = re.search(r"__fmaf_rn\(x\.hi, (\S+)f, (\S+)f\);", src)
    inv, big = float(m.group(1)), float.fromhex(m.group(2))
    assert abs(Decimal(f32(inv)) - 256 / Decimal(2).ln()) / (256 / Decimal(2).ln()) < Decimal(2) ** -24
    # n is rounded by adding 1.5 2^23 (float32 integers there are spaced 1) and
    # read back from the bits: exact for |n| < 2^22 (here |n| <= 87 * 256 / ln2)
    assert big == 1.5 * 2.0 ** 23 and f32(big) == big
    assert re.search(r"__float_as_int\(rnd\) - 0x4B400000", src)
    assert struct.unpack("<I", struct.pack("<f", big))[0] == 0x4B400000
    assert 87 * 256 / math.log(2) < 2 ** 22
    for n in (0, -1, -255, -256, -32130):  # the bit trick recovers n
        rnd = f32(big + n)
        assert struct.unpack("<i", struct.pack("<f", rnd))[0] - 0x4B400000 == n
