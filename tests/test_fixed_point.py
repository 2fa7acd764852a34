"""The exact fixed-point accumulation that makes the FP32 spreading
order-independent, checked in exact rational arithmetic on the CPU.

Each contribution C (a float32 product w * wx in units of 2^-k) is split by
three fused multiply-adds around the magic number M = 1.5 * 2^23:
    t1 = fma(w, wx, M)            bits(t1) = Mb + h,  h = round(C)
    z  = fma(t1, -2048, 2049 M)   exact
    t2 = fma(2048 w, wx, z)       bits(t2) = Mb + l,  l = round(2048 (C - h))
and the bit patterns are added as 32-bit integers.  After n <= 1024 terms
the words are hi = n Mb + H, lo = n Mb + L (mod 2^32); L is the
sign-extended low 22 bits of lo, H = (hi - lo) + L, and the face value is
S = 2048 H + L, rounded once to float32 (units of 2^-(k+11)).  These tests
restate that arithmetic with exact rationals and check every claim: the
split, the exactness of z, the decoding under wrap-around, and that S is the
exact sum of the per-term integers.
"""
from fractions import Fraction as Fr
import random
import struct

M = 12582912.0           # 1.5 * 2^23
MB = 0x4B400000          # bit pattern of M


def f32_rne(q: Fr) -> Fr:
    """Exact rational q rounded to the nearest float32 (ties to even)."""
    if q == 0:
        return Fr(0)
    s = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fr(2) ** e > a:
        e -= 1
    while Fr(2) ** (e + 1) <= a:
        e += 1
    scale = Fr(2) ** (23 - e)          # 2^23 <= a * scale < 2^24
    m = a * scale
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fr(1, 2) or (rem == Fr(1, 2) and fl % 2 == 1):
        fl += 1
    return s * Fr(fl) / scale


def fma32(a: Fr, b: Fr, c: Fr) -> Fr:
    return f32_rne(a * b + c)


def bits(x: Fr) -> int:
    return struct.unpack("<I", struct.pack("<f", float(x)))[0]


def rne_int(q: Fr) -> int:
    fl = q.numerator // q.denominator
    rem = q - fl
    if rem > Fr(1, 2) or (rem == Fr(1, 2) and fl % 2 == 1):
        fl += 1
    return fl


def rand_f32(rng, lo, hi):
    return f32_rne(Fr(rng.uniform(lo, hi)))


def split(w: Fr, wx: Fr):
    t1 = fma32(w, wx, Fr(M))
    z = fma32(t1, Fr(-2048), Fr(M) * 2049)
    assert z == Fr(M) * 2049 - 2048 * t1                    # z is exact
    t2 = fma32(f32_rne(2048 * w), wx, z)
    return bits(t1), bits(t2)


def test_split_is_round_and_residual():
    rng = random.Random(1)
    for _ in range(2000):
        # |C| < 2^19: |w| < 2^19 (weight products <= 1/8 folded in), wx in [0, 1)
        w = rand_f32(rng, -2.0 ** 19, 2.0 ** 19)
        wx = rand_f32(rng, 0.0, 1.0)
        C = w * wx
        b1, b2 = split(w, wx)
        h = rne_int(C)
        assert (b1 - MB) == h
        assert (b2 - MB) == rne_int(2048 * (C - h))
        assert abs(b2 - MB) <= 1024


def test_words_decode_to_the_exact_sum_under_wraparound():
    rng = random.Random(2)
    for trial in range(40):
        n = rng.choice([1, 7, 300, 1024])
        hi = lo = 0
        exact = 0
        true_sum = Fr(0)
        for _ in range(n):
            w = rand_f32(rng, -2.0 ** 19, 2.0 ** 19)
            wx = rand_f32(rng, 0.0, 1.0)
            b1, b2 = split(w, wx)
            hi = (hi + b1) & 0xFFFFFFFF
            lo = (lo + b2) & 0xFFFFFFFF
            exact += 2048 * (b1 - MB) + (b2 - MB)
            true_sum += w * wx
        L = lo & 0x3FFFFF
        L = L - (1 << 22) if L & (1 << 21) else L              # sign-extend 22 bits
        H = ((hi - lo) & 0xFFFFFFFF)
        H = H - (1 << 32) if H & (1 << 31) else H
        H += L
        S = 2048 * H + L
        assert S == exact
        # the value is rounded once: fma(float(S >> 24), 2^24, float(S & 0xFFFFFF))
        top, low = S >> 24, S & 0xFFFFFF
        assert abs(top) < 2 ** 23
        assert fma32(Fr(top), Fr(2 ** 24), Fr(low)) == f32_rne(Fr(S))
        # each term is carried to within half a unit of 2^-11
        assert abs(Fr(S) - 2048 * true_sum) <= Fr(n, 2)
