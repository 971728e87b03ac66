"""CPU model of the BF16 slicing of the exact slice-Gram distances: the
slices of a feature x are the base-256 digits of v = x 2^(7 - e) (e: frexp's
exponent of the row's largest magnitude), each the nearest integer (ties to
even) to what the digits before it leave, c_0 = rint(v), c_1 =
rint((v - c_0) 256), ...  The slicing kernel takes them from the double's
bits in 64-bit integers (F = v 2^56 truncated, a sticky flag for the bits
shifted out, the scaling's underflow to a signed zero reproduced).  This test
restates both forms and checks that they give the same digits, signed zeros
included, on random rows, tie-heavy rows, subnormals and rows whose smaller
features underflow when scaled by the largest."""
import math
import struct

import numpy as np

SLICES = 5


def fp64_digits(x, e):
    v = math.ldexp(x, 7 - e)
    out = []
    for _ in range(SLICES):
        c = float(np.rint(v))
        out.append(c)
        v = (v - c) * 256.0
    return out


def integer_digits(x, e):
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    neg = b >> 63
    E = (b >> 52) & 0x7FF
    m = b & ((1 << 52) - 1)
    if E:
        m |= 1 << 52
    sh = max(E, 1) - 1012 - e
    t = max(E, 1) + 7 - e
    vzero = m == 0 or (t <= 0 and (-t >= 53 or m <= (1 << -t)))
    F, sticky = 0, False
    if not vzero:
        if sh >= 0:
            F = m << sh
        elif sh > -64:
            F, sticky = m >> -sh, (m & ((1 << -sh) - 1)) != 0
        else:
            sticky = True
    assert F < 2 ** 63
    dsign = (-1 if neg else 1) if sticky else 0
    R = -F if neg else F
    out = []
    for s in range(SLICES):
        k = 56 - 8 * s
        q = R >> k
        rem = R - (q << k)
        half = 1 << (k - 1)
        c = q + 1 if (rem > half or (rem == half and (dsign > 0 or (dsign == 0 and q & 1)))) else q
        assert abs(c) <= 128
        negz = c == 0 and (R < 0 or (R == 0 and dsign < 0) or (s == 0 and neg and vzero))
        out.append(-0.0 if negz else float(c))
        R -= c << k
    return out


def _rows(rng, count):
    special = [0.0, -0.0, 5e-324, -5e-324, 2.5, -2.5, 0.5, -1e-300, 1e-310, 1e300, -3e-320, 1e-200]
    for i in range(count):
        kind = i % 5
        if kind == 0:
            yield rng.standard_normal(8) * 10.0 ** rng.integers(-30, 30)
        elif kind == 1:
            yield rng.standard_normal(8) * np.exp2(rng.integers(-60, 0, 8).astype(float))
        elif kind == 2:  # few significant bits: exact half-way remainders
            yield np.round(rng.standard_normal(8) * 2 ** 12) / 2.0 ** rng.integers(0, 40)
        elif kind == 3:
            yield np.array([special[j] for j in rng.integers(0, len(special), 8)])
        else:
            yield rng.integers(-300, 300, 8) / 2.0 ** rng.integers(0, 60)


def test_integer_digits_equal_the_fp64_steps():
    rng = np.random.default_rng(2024)
    for row in _rows(rng, 4000):
        mx = max(abs(float(v)) for v in row)
        e = math.frexp(mx)[1] if mx > 0 else 0
        for x in row:
            a, b = fp64_digits(float(x), e), integer_digits(float(x), e)
            assert [struct.pack("<d", v) for v in a] == [struct.pack("<d", v) for v in b], (x, e, a, b)


def test_digits_reconstruct_the_feature():
    """Five digits carry x to within half a unit of the fifth digit (2^-33 of
    2^e), and an exact half-way value keeps the even digit."""
    rng = np.random.default_rng(7)
    for row in _rows(rng, 500):
        mx = max(abs(float(v)) for v in row)
        if mx == 0 or not math.isfinite(mx):
            continue
        e = math.frexp(mx)[1]
        for x in row:
            c = integer_digits(float(x), e)
            back = sum(ci * 256.0 ** -s for s, ci in enumerate(c))
            assert abs(back - math.ldexp(float(x), 7 - e)) <= 0.5 * 256.0 ** -4 * (1 + 1e-12)
    assert integer_digits(2.5, 2)[0] == 80.0  # v = 2.5 * 2^5 = 80 exactly
    assert integer_digits(1.5 * 2 ** -8, 1)[:2] == [0.0, 96.0]
    assert fp64_digits(0.5 * 2 ** -6, 1)[0] == 0.0 == integer_digits(0.5 * 2 ** -6, 1)[0]  # rint(0.5) = 0
