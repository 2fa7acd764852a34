"""The compensated FP32 sums that replace FP64 for the cancellation-prone
scalars of the force (J - 1 and I4f - 1), checked in exact rational
arithmetic on the CPU.

The running sum (hi, lo) of terms a_i b_i is advanced as in the Dot2
algorithm of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005): the
exact product p + e = a b by one fused multiply-add (e = fma(a, b, -p)),
Knuth's TwoSum s + t = hi + p, and every rounding error collected in lo.
Their error bound for n terms is |res - x| <= u |x| + gamma_n^2 sum |a_i b_i|
with u = 2^-24 and gamma_n = n u / (1 - n u): the result is as accurate as
if the sum were formed in twice the working precision and then rounded.
This test restates the steps with float32 rounding emulated exactly and
checks that bound on sums that cancel to 1e-7 of their terms, the regime of
J - 1 for nearly isochoric deformations.
"""
from fractions import Fraction as Fr
import random

U = Fr(1, 2 ** 24)


def f32(q: Fr) -> Fr:
    if q == 0:
        return Fr(0)
    s = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fr(2) ** e > a:
        e -= 1
    while Fr(2) ** (e + 1) <= a:
        e += 1
    scale = Fr(2) ** (23 - e)
    m = a * scale
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fr(1, 2) or (rem == Fr(1, 2) and fl % 2 == 1):
        fl += 1
    return s * Fr(fl) / scale


def two_sum(a, b):
    s = f32(a + b)
    v = f32(s - a)
    e = f32(f32(a - f32(s - v)) + f32(b - v))
    return s, e


def dacc(acc, a, b):                       # acc + a b
    hi, lo = acc
    p = f32(a * b)
    pe = f32(a * b - p)                    # the fma residual: exact
    assert p + pe == a * b
    s, t = two_sum(hi, p)
    assert s + t == hi + p                 # TwoSum is exact
    return s, f32(lo + f32(t + pe))


def sacc(acc, a):                          # acc + a
    hi, lo = acc
    s, t = two_sum(hi, a)
    return s, f32(lo + t)


def test_dot2_meets_its_error_bound_on_cancelling_sums():
    rng = random.Random(3)
    plain_misses = 0
    for trial in range(300):
        n = rng.choice([3, 6, 9])
        a = [f32(Fr(rng.uniform(-1.5, 1.5))) for _ in range(n)]
        b = [f32(Fr(rng.uniform(-1.5, 1.5))) for _ in range(n)]
        x = sum(ai * bi for ai, bi in zip(a, b))
        # a constant that cancels the sum to ~1e-7 of its terms: c = -f32(x) + tiny
        c = -f32(x + Fr(rng.uniform(-1e-7, 1e-7)))
        acc = sacc((Fr(0), Fr(0)), c)
        for ai, bi in zip(a, b):
            acc = dacc(acc, ai, bi)
        res = f32(acc[0] + acc[1])
        exact = x + c
        g = n * U / (1 - n * U)
        bound = U * abs(exact) + g * g * (sum(abs(ai * bi) for ai, bi in zip(a, b)) + abs(c))
        assert abs(res - exact) <= bound
        # plain FP32 accumulation (one fma per term) misses the same bound
        plain = f32(c)
        for ai, bi in zip(a, b):
            plain = f32(ai * bi + plain)
        plain_misses += abs(plain - exact) > bound
    assert plain_misses > 150
