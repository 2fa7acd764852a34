"""The exact fixed-point accumulation that makes the FP32 spreading
order-independent, checked in exact rational arithmetic on the CPU.

Each contribution C (a float32 product w * wx in units of 2^-k of its tile)
is split by three fused multiply-adds around the magic number M = 1.5 * 2^23:
    t1 = fma(w, wx, M)            bits(t1) = Mb + h,  h = round(C)
    z  = fma(t1, -2048, 2049 M)   exact
    t2 = fma(2048 w, wx, z)       bits(t2) = Mb + l,  l = round(2048 (C - h))
and the bit patterns are added as 32-bit integers.  After n <= 1024 terms
the words are hi = n Mb + H, lo = n Mb + L (mod 2^32); L is the
sign-extended low 22 bits of lo, H = (hi - lo) + L, and the item stores
S = 2048 H + L.  The exponent of a tile,
    k = min(21, 30 - ceil_log2(min(n_tile, 1024))) - e,   cm = max|V| |scale| / 8 < 2^e,
keeps every contribution below 2^21 and |H| below 2^31 (1024: the largest
work item any tuning may choose, so the exponent does not depend on the
tuning).  The merge sums a face's S per source tile in 64 bits, shifts the
source sums to one exponent (units of 2^-(k+11))
    k_ref = min(max_s k'_s, min_s (k'_s + 17 - ceil_log2(m_s))),  k'_s = k_s + 11,
(m_s = ceil(n_s / 512) bounds source s's work items under any tuning),
and converts the total with two exactly rounded 32-bit halves and one fma.
These tests restate that arithmetic with exact rationals and check each
claim: the split, the exactness of z, the decoding under wrap-around, the
absence of overflow for the worst placements the bound allows, the alignment
headroom, and the final conversion.
"""
from fractions import Fraction as Fr
import math
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


def ceil_log2(n):
    return (n - 1).bit_length() if n > 1 else 0


def frexp_e(x: float) -> int:
    return math.frexp(x)[1]


def tile_exp(vmax: float, npts: int, chunk: int, scale: float) -> int:
    """The kernel's per-tile exponent (float32 arithmetic for cm)."""
    cm = float(f32_rne(f32_rne(Fr(0.125) * Fr(vmax)) * Fr(abs(scale))))
    if not cm > 0:
        return 0
    k = min(21, 30 - ceil_log2(min(npts, chunk))) - frexp_e(cm)
    return max(-100, min(k, 100))


def test_split_is_round_and_residual():
    rng = random.Random(1)
    for _ in range(2000):
        w = rand_f32(rng, -2.0 ** 21, 2.0 ** 21)
        wx = rand_f32(rng, 0.0, 1.0)
        C = w * wx
        b1, b2 = split(w, wx)
        h = rne_int(C)
        assert (b1 - MB) == h
        assert (b2 - MB) == rne_int(2048 * (C - h))
        assert abs(b2 - MB) <= 1024


def decode(hi: int, lo: int) -> int:
    L = lo & 0x3FFFFF
    L = L - (1 << 22) if L & (1 << 21) else L              # sign-extend 22 bits
    H = ((hi - lo) & 0xFFFFFFFF)
    H = H - (1 << 32) if H & (1 << 31) else H
    H += L
    return 2048 * H + L


def test_words_decode_to_the_exact_sum_under_wraparound():
    rng = random.Random(2)
    for trial in range(40):
        n = rng.choice([1, 7, 300, 1024])
        hi = lo = 0
        exact = 0
        true_sum = Fr(0)
        for _ in range(n):
            w = rand_f32(rng, -2.0 ** 20, 2.0 ** 20)
            wx = rand_f32(rng, 0.0, 1.0)
            b1, b2 = split(w, wx)
            hi = (hi + b1) & 0xFFFFFFFF
            lo = (lo + b2) & 0xFFFFFFFF
            exact += 2048 * (b1 - MB) + (b2 - MB)
            true_sum += w * wx
        if abs(exact) >= 2048 * 2 ** 31:
            continue
        S = decode(hi, lo)
        assert S == exact
        # each term is carried to within half a unit of 2^-11
        assert abs(Fr(S) - 2048 * true_sum) <= Fr(n, 2)


def _contribution(v: Fr, vscale: Fr, wz: Fr, wy: Fr, wx: Fr) -> int:
    # staging: v' = v vscale, a = v' wz, row = a wy (float32 products); the
    # lane then adds fma(row, wx, M)
    vv = f32_rne(v * vscale)
    a = f32_rne(vv * wz)
    r = f32_rne(a * wy)
    b1, _ = split(r, wx)
    return b1 - MB


def test_tile_exponent_bounds_every_item_sum():
    # Worst placement the bound allows: n_eff points all at the tile's
    # largest |V|, all on the face where each 1-D weight is at its maximum
    # 1/2 (the kernel's weights never exceed 1/2 by more than float rounding).
    rng = random.Random(3)
    half = f32_rne(Fr(1, 2) * (1 + Fr(1, 2 ** 23)))   # 1/2 rounded up by an ulp
    for _ in range(200):
        vmax = float(rand_f32(rng, 1e-20, 1e20)) * rng.choice([1, 1e-10, 1e10])
        scale = float(f32_rne(Fr(rng.choice([1.0, 256.0 ** 3, 1.0 / 7.0, 3.3e4]))))
        npts = rng.choice([1, 2, 37, 300, 511, 512, 1000, 1024, 5000])
        k = tile_exp(vmax, npts, 1024, scale)
        vscale = f32_rne(Fr(scale) * Fr(2) ** k)
        c = _contribution(Fr(vmax), vscale, half, half, half)
        assert abs(c) < 2 ** 21
        neff = min(npts, 1024)                    # the most points an item can hold
        assert neff * abs(c) < 2 ** 31            # |H| < 2^31: no word can wrap
        # the resolution is not wasted: the largest contribution uses at least
        # 2^19 / n_eff-scaled units (within a factor 4 of the bound)
        assert abs(c) * 2 ** ceil_log2(neff) >= 2 ** 27 or abs(c) >= 2 ** 19


def align(v: int, sh: int) -> int:
    return v << sh if sh >= 0 else v >> -sh        # Python >> is floor, like the kernel's


def to_float(S: int, k_ref: int) -> Fr:
    """Two exactly rounded 32-bit halves of |S| joined by one fma, scaled."""
    m = abs(S)
    assert m < 2 ** 64
    f = fma32(f32_rne(Fr(m >> 32)), Fr(2 ** 32), f32_rne(Fr(m & 0xFFFFFFFF)))
    f = -f if S < 0 else f
    return f * Fr(2) ** (-k_ref)


def test_merge_alignment_headroom_and_conversion():
    rng = random.Random(4)
    for _ in range(400):
        nsrc = rng.randint(1, 8)
        ks = [rng.randint(-40, 60) + 11 for _ in range(nsrc)]
        # a source tile of npts points, cut into work items of 512..1024
        # points by the tuning; the cap uses the tuning-free bound m
        npts = [rng.choice([1, 300, 1024, 1500, 9000, 102400]) for _ in range(nsrc)]
        items = [-(-n // rng.choice([512, 700, 1024])) for n in npts]
        m = [-(-n // 512) for n in npts]
        assert all(i <= b for i, b in zip(items, m))
        kmax = max(ks)
        kcap = min(k + 17 - ceil_log2(b) for k, b in zip(ks, m))
        k_ref = min(kmax, kcap)
        total = 0
        exact = Fr(0)
        for k, n in zip(ks, items):
            # a source sum: n item values S = 2048 H + L, each below 2^42
            S = sum(rng.randint(-(2 ** 42) + 1, 2 ** 42 - 1) for _ in range(n))
            a = align(S, k_ref - k)
            assert abs(a) < 2 ** 59
            total += a
            exact += Fr(S) * Fr(2) ** (-k)
            if k <= k_ref:
                assert Fr(a) * Fr(2) ** (-k_ref) == Fr(S) * Fr(2) ** (-k)   # exact
        assert abs(total) < 2 ** 62
        got = to_float(total, k_ref)
        # within one unit in the last place of the float32 result (the right
        # shifts of finer sources lose less than one unit of 2^-k_ref each)
        ref = f32_rne(Fr(total) * Fr(2) ** (-k_ref))
        if ref != 0:
            ulp = Fr(2) ** (frexp_e(float(abs(ref))) - 24)
            assert abs(got - ref) <= ulp
        assert abs(Fr(total) * Fr(2) ** (-k_ref) - exact) <= Fr(nsrc) * Fr(2) ** (-k_ref)


def test_conversion_is_exact_below_2_to_24():
    for S in (0, 1, -1, 12345, -(2 ** 24) + 1, 2 ** 24, -(2 ** 24)):
        assert to_float(S, 0) == Fr(S)
