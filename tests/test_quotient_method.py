"""The method behind the device's C(t) = sumc / card (exact_quotient in
csrc/kohler_common.cuh), restated step for step in Python and checked against
Python's correctly rounded division on CPU.

The device computes the quotient of two counts below 2^53 without the FP64
pipe: both operands normalised to 53 bits, six radix-2^9 long-division digits
estimated in float32 from the top 23 bits of the remainder and of the divisor
and corrected against the exact remainder, then rounding to nearest even on
the top 53 bits.  The GPU parity tests compare every C(t)
with the oracle's double division bit for bit; this test shows that the method
itself is exact (the digit estimate is never off by more than the correction
allows), over structured and random operands, including the ranges the curve
produces (card below 2^33, C(t) below M).
"""
import random
import struct

import numpy as np

F = np.float32


def f23(v: int) -> np.float32:
    """float32 of v < 2^23, as the device makes it: 2^23 + v read as a float, less 2^23."""
    assert 0 <= v < (1 << 23)
    x = np.frombuffer(struct.pack("<I", 0x4B000000 | v), dtype=np.float32)[0]
    return F(x - F(8388608.0))


def quotient(a: int, b: int) -> float:
    if a == 0:
        return 0.0
    la, lb = a.bit_length() - 1, b.bit_length() - 1
    A, B = a << (52 - la), b << (52 - lb)
    rB = F(512.0) / f23(B >> 30)  # float32 division, round to nearest
    if A >= B:
        X, R, e = 1, A - B, la - lb
    else:
        X, R, e = 0, A, la - lb - 1
    worst = 0
    for _ in range(6):
        x = F(F(f23(R >> 30) * rB) + F(8388608.0))  # float32 product, then rounded to an integer
        d = struct.unpack("<I", struct.pack("<f", x))[0] & 0x7FFFFF
        r = (R << 9) - d * B
        fix = 0
        while r < 0:
            d, r, fix = d - 1, r + B, fix + 1
        while r >= B:
            d, r, fix = d + 1, r - B, fix + 1
        worst = max(worst, fix)
        X, R = (X << 9) | d, r
    assert worst <= 3, "the device corrects a digit at most three times"
    if X >> 54:
        m, g, st = X >> 2, (X >> 1) & 1, (X & 1) or R != 0
    else:
        m, g, st = X >> 1, X & 1, R != 0
    if g and (st or (m & 1)):
        m += 1
        if m >> 53:
            m, e = m >> 1, e + 1
    bits = ((e + 1023) << 52) | (m & ((1 << 52) - 1))
    return struct.unpack("<d", struct.pack("<Q", bits))[0]


def same(a, b):
    want = a / b
    got = quotient(a, b)
    return struct.pack("<d", want) == struct.pack("<d", got)


def test_small_operands_exhaustive():
    assert all(same(a, b) for b in range(1, 130) for a in range(0, 700))


def test_structured_operands():
    bs = list(range(1, 64)) + [2 ** k + d for k in range(1, 53) for d in (-1, 0, 1) if 1 <= 2 ** k + d < 2 ** 53]
    for b in bs:
        for a in (0, 1, 2, b - 1, b, b + 1, 2 * b - 1, 2 * b + 1, 255 * b + 1, 2 ** 52, 2 ** 53 - 1):
            if 0 <= a < 2 ** 53:
                assert same(a, b), (a, b)


def test_random_operands():
    rng = random.Random(7)
    for _ in range(40000):
        la, lb = rng.randrange(53), rng.randrange(53)
        a = rng.randrange(1 << la, 1 << (la + 1))
        b = rng.randrange(1 << lb, 1 << (lb + 1))
        assert same(min(a, 2 ** 53 - 1), min(b, 2 ** 53 - 1)), (a, b)
    for _ in range(40000):  # the curve's range: card < 2^33, C(t) < 256
        b = rng.randrange(1, 1 << 33)
        a = rng.randrange(0, 256 * b)
        assert same(a, b), (a, b)


def test_planted_mistakes_are_caught():
    # a method that truncates instead of rounding, or drops the remainder from
    # the sticky bit, differs from the correctly rounded quotient
    a, b = 2, 3  # 0.666...: its 54th bit is 1, remainder non-zero
    x = quotient(a, b)
    trunc = struct.unpack("<d", struct.pack("<Q", struct.unpack("<Q", struct.pack("<d", x))[0] - 1))[0]
    assert x == 2 / 3 and trunc != 2 / 3
