// Double-float values: the unevaluated sum hi + lo of two FP32 numbers, about
// 48 significant bits, built from the error-free transformations of Knuth
// (TwoSum: the rounding error of a sum, The Art of Computer Programming
// vol. 2, 4.2.2) and of Dekker (1971: the exact product, here through one
// fused multiply-add, e = fma(a, b, -ab)).  The intrinsics __fadd_rn /
// __fmul_rn keep the compiler from contracting or reassociating the steps
// whose rounding errors the transformations capture.
//
// On GB300 the FP64 pipe runs at 1/64 of the FP32 rate, so a double-float
// operation (5 to 20 FP32 operations) costs a fraction of one FP64 operation;
// it serves the force kernel's cancellation-prone scalars (J - 1 and
// I4f - 1, short sums of FP32 numbers and of products of two of them, which
// double-float holds exactly), through the compensated accumulation below.
#pragma once
#include <cuda_runtime.h>

namespace ibfe {

struct df {
  float hi, lo;
  __host__ __device__ constexpr df() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit df(float x) : hi(x), lo(0.f) {}
  __host__ __device__ constexpr explicit df(int x) : hi(float(x)), lo(0.f) {}
  __device__ explicit operator float() const { return __fadd_rn(hi, lo); }
  __device__ explicit operator double() const { return double(hi) + double(lo); }
};

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fadd_rn(s, -a);
  const float e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -v)), __fadd_rn(b, -v));
  return df(s, e);
}

// p + e = a b exactly (the fused multiply-add returns the rounding error)
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df(p, fmaf(a, b, -p));
}

// ordering by the rounded values (the pairs the accumulation below leaves
// need not be normalised, so hi alone may not carry the sign)
__device__ __forceinline__ bool operator>(df a, df b) {
  return __fadd_rn(a.hi, a.lo) > __fadd_rn(b.hi, b.lo);
}

// Compensated accumulation (the Dot2 / Sum2 algorithms of Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005): the
// running sum's hi part is advanced with TwoSum and every rounding error
// (of the sums and of the exact products) is collected in lo, so a short sum
// of FP32 numbers and products is as accurate as if computed in twice the
// working precision, at about ten FP32 operations per term.
__device__ __forceinline__ df dacc(df acc, float a, float b) {  // acc + a b
  const df p = two_prod(a, b);
  const df s = two_sum(acc.hi, p.hi);
  return df(s.hi, __fadd_rn(acc.lo, __fadd_rn(s.lo, p.lo)));
}
__device__ __forceinline__ df sacc(df acc, float a) {  // acc + a
  const df s = two_sum(acc.hi, a);
  return df(s.hi, __fadd_rn(acc.lo, s.lo));
}
// The same interface for the plain scalar types: one fused multiply-add in
// double (the product of two FP32 numbers is exact there) or in float.
__device__ __forceinline__ double dacc(double acc, double a, double b) { return fma(a, b, acc); }
__device__ __forceinline__ double sacc(double acc, double a) { return acc + a; }
__device__ __forceinline__ float dacc(float acc, float a, float b) { return fmaf(a, b, acc); }
__device__ __forceinline__ float sacc(float acc, float a) { return acc + a; }

// Double-float arithmetic on double-float operands (the kinematics of the
// exact volumetric invariant): sums of two pairs, products, products with a
// float, and the quotient, each within a few units of 2^-44 relative (the
// accumulations below leave the pair unnormalised; norm() restores
// |lo| <= ulp(hi) / 2).
__device__ __forceinline__ df norm(df a) { return two_sum(a.hi, a.lo); }
__device__ __forceinline__ df neg(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df dadd(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df dmul(df a, df b) {
  const df p = two_prod(a.hi, b.hi);
  return two_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}
// acc + a b with a double-float a and a float b
__device__ __forceinline__ df dfma(df acc, df a, float b) {
  const df p = two_prod(a.hi, b);
  const df s = two_sum(acc.hi, p.hi);
  return df(s.hi, __fadd_rn(__fadd_rn(acc.lo, s.lo), fmaf(a.lo, b, p.lo)));
}
// acc + a b, both double-float
__device__ __forceinline__ df dfma(df acc, df a, df b) {
  const df p = two_prod(a.hi, b.hi);
  const df s = two_sum(acc.hi, p.hi);
  return df(s.hi, __fadd_rn(__fadd_rn(acc.lo, s.lo), fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo))));
}
// a / b: the float quotient of the leading parts, corrected once by the
// double-float residual a - b q
__device__ __forceinline__ df ddiv(df a, df b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const df r = dadd(a, neg(dmul(b, df(q1))));
  return two_sum(q1, __fdiv_rn(r.hi, b.hi));
}

// ln(1 + x) of a double-float argument.  The stress consumes ln J rounded to
// FP32, so the FP32 logarithm of the correctly rounded argument is as good as
// an extended one: what must not lose digits is the argument J - 1 itself,
// which the compensated sums above deliver.
__device__ __forceinline__ df log1p_s(df x) { return df(log1pf(float(x))); }

}  // namespace ibfe
