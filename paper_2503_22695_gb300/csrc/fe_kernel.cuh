// Hyperelastic nodal force of the immersed structure (Section 4.4:
// F_i = -sum_q P(X_q) : grad_X phi_i(X_q) w_q) and its adjoints, on trilinear
// hexahedra with the 2x2x2 Gauss rule.  One thread per element; the eight
// Gauss points are unrolled so every shape-function value is a compile-time
// constant.
//
// Kinematics are carried as the displacement gradient H = F - I, formed from
// node differences relative to corner 0 (split positions subtract their
// integer cells exactly), so J - 1, I1 - 3 and I4 - 1 are evaluated without
// cancellation:
//   J - 1   = tr H + ((tr H)^2 - tr(H^2))/2 + det H
//   I1 - 3  = 2 tr H + |H|^2
//   I4 - 1  = (|e|^2 - 1) + 2 e.(H e) + |H e|^2
//   I8      = e_f.e_s + e_f.(H e_s) + e_s.(H e_f) + (H e_f).(H e_s)
// The scalars of the volumetric term and of the fibre term near I4f = 1 are
// accumulated in the type S: J - 1 and the fibre invariant I4f - 1 are short
// sums of FP32 numbers and of products of two of them, so with S = df
// (split-precision plans) they are compensated FP32 pairs, exact products and
// error-free sums (dfloat.cuh), as accurate as twice the working precision and
// free of FP64 instructions (GB300 executes FP64 at 1/64 of the FP32 rate);
// with S = double (FP64 plans) plain double, with S = float (the all-FP32
// option) plain float.  ln J is then log1p of the accurately rounded J - 1.
// Once I4f - 1 is known, the fibre coefficient
// 2 a_f (I4f - 1) exp(b_f (I4f - 1)^2) is a product of well-conditioned factors
// and is formed in Real: exp has relative error (argument error) x (argument),
// small here.  The sheet family e_s and the coupling I8 of Holzapfel-Ogden use
// the same cancellation-free formulas in Real.  Everything else is in Real
// (float for split-precision plans, double for FP64 plans).
//
// With Du = sum_a du_a (x) dN_a/dxi (3x3) and J0 = sum_a dX_a (x) dN_a/dxi:
//   H = Du J0^-1, and the corner forces are
//   G_a -= (P J0^-T w j0) dN_a/dxi  (w: the force rule's weight),
// so the X-gradients of the shape functions are never formed.
//
// This header holds the device code and the launcher template fe_run; the
// instantiations are spread over fe_force_f32.cu (split-precision plans) and
// fe_force_var.cu (FP32-scalar and FP64 plans) so that they compile in
// parallel, and fe_force.cu picks one per call.
#pragma once
#include <algorithm>
#include <cstdio>

#include "dfloat.cuh"
#include "ib_device.cuh"

namespace ibfe {
namespace {


template <typename Real>
struct FeArgs {
  int E;
  int64_t N;
  const int32_t* conn;
  const Real* X;
  const Real* fib;       // [6][E] or null
  const int32_t* mat_id; // [E] or null
  NodeLoader<Real> pos;
  Real h;
  float hlo;             // h - float(h) (split-precision plans: h as a double-float)
  const float2* jx;      // [QF][E] exact J - 1 (IB_FP32_SPLIT_DFVOL) or null
  const Real* v;         // [3][N] direction (adjoint) or null
  Real* out;             // [24][E] corner contributions
  double* epart;         // per-element partial sums or null: the energy [E] in
                         // double, the parameter gradients [kParamRow][E] in Real
  int* status;
  int* next;             // block counter, zero at launch
  const InstDev* inst;   // packed plans: instance table (each instance's h), else null
  const int32_t* elem_inst;  // packed plans: instance of each element
  const MatRow* mats;    // packed plans: material table in device memory, else null
};

template <typename T>
__device__ __forceinline__ T det3(const T A[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

// cof(A)_ij = d det A / d A_ij
template <typename T>
__device__ __forceinline__ void cofactor(const T A[3][3], T C[3][3]) {
  C[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
  C[0][1] = A[1][2] * A[2][0] - A[1][0] * A[2][2];
  C[0][2] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
  C[1][0] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
  C[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
  C[1][2] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
  C[2][0] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
  C[2][1] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
  C[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
}


// Quantities of one fibre family needed by the stress and its derivatives.
template <typename Real, typename S>
struct Fibre {
  Real Fe[3];  // F e
  S d;         // I4* - 1 = max(I4 - 1, 0), or I4 - 1 without the clamp
  S d4;        // I4 - 1
};

template <typename Real, typename S>
__device__ __forceinline__ void fibre_kin(const Real H[3][3], const Real e[3], S en1,
                                          Fibre<Real, S>& f, bool clamp = true) {
  Real He[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) He[i] = H[i][0] * e[0] + H[i][1] * e[1] + H[i][2] * e[2];
  // I4 - 1 = (|e|^2 - 1) + He.(2e + He): the products are exact in S, the
  // sum compensated; 2e + He carries a rounding of order ulp(1) |He|, far
  // below the result's
  S I4m1 = en1;
#pragma unroll
  for (int i = 0; i < 3; ++i) I4m1 = dacc(I4m1, He[i], Real(2) * e[i] + He[i]);
  f.d4 = I4m1;
  f.d = (!clamp || I4m1 > S(0)) ? I4m1 : S(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) f.Fe[i] = e[i] + He[i];
}

// ln(1 + x) in double.  For |x| <= 1/8 it is 2 atanh(s) with s = x / (2 + x)
// (|s| <= 1/17), summed as s (2 + 2z/3 + 2z^2/5 + ... + 2z^6/13), z = s^2: the
// first omitted term, 2 z^7/15, is below 4e-19 relative.  1/(2 + x) comes from
// an FP32 reciprocal refined by one Newton step in double, which leaves a
// relative error near 1e-14 (the square of the FP32 reciprocal's).  Outside
// that range (|J - 1| > 1/8) the library log1p is used.
__device__ __forceinline__ double log1p_d(double x) {
  if (!(fabs(x) <= 0.125)) return log1p(x);
  const double d = 2.0 + x;
  double r = (double)__frcp_rn((float)d);
  r = fma(r, fma(-d, r, 1.0), r);
  const double s = x * r;
  const double z = s * s;
  double t = 2.0 / 13.0;
  t = fma(t, z, 2.0 / 11.0);
  t = fma(t, z, 2.0 / 9.0);
  t = fma(t, z, 2.0 / 7.0);
  t = fma(t, z, 2.0 / 5.0);
  t = fma(t, z, 2.0 / 3.0);
  t = fma(t, z, 2.0);
  return s * t;
}

__device__ __forceinline__ double log1p_s(double x) { return log1p_d(x); }
__device__ __forceinline__ float log1p_s(float x) { return log1pf(x); }

// Resident 128-thread CTAs per SM requested from the register allocator.
#ifndef IBFE_FE_MIN_BLOCKS
#define IBFE_FE_MIN_BLOCKS 3
#endif
#ifndef IBFE_FE_MIN_BLOCKS_ADJ
#define IBFE_FE_MIN_BLOCKS_ADJ 3
#endif

template <typename Real, bool kAdj>
constexpr int fe_min_blocks() {
  return sizeof(Real) == 8 ? 2 : (kAdj ? IBFE_FE_MIN_BLOCKS_ADJ : IBFE_FE_MIN_BLOCKS);
}

// Exact volumetric invariant (IB_FP32_SPLIT_DFVOL plans): J - 1 at force
// point q of element e as (det(DX + DU) - det(DX)) / det(DX), with
// DX = sum_a dX_a (x) dN_a/dxi and DU = sum_a du_a (x) dN_a/dxi, from node
// differences formed without rounding (integer cells, FP32 offsets, FP32
// reference coordinates: TwoSum), the expansion
//   det(A + B) - det(A) = cof(A) : B + A : cof(B) + det(B),
// and every step in double-float.  Near incompressibility |J - 1| << |F - I|,
// and J - 1 from the FP32 displacement gradient would carry a relative error
// near eps |F - I| / |J - 1|; here it is near 2^-44 |F - I| / |J - 1|.  The
// shape-function derivatives are the force kernel's FP32 constants, so both
// describe the same element.  One thread per (q, e), q-major; the result is
// stored as a (hi, lo) pair for the force kernel.
__device__ __forceinline__ void cof3(const df M[3][3], df C[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
      C[i][j] = dadd(dmul(M[i1][j1], M[i2][j2]), neg(dmul(M[i1][j2], M[i2][j1])));
    }
}

template <int kEl, int Q>
__device__ __forceinline__ df exact_jm1_at(const FeArgs<float>& A, int e) {
  using EL = El<kEl>;
  const int E = A.E;
  const int n0 = __ldg(A.conn + e);
  int c0[3];
  float o0[3], X0[3];
  A.pos.load(n0, c0, o0);
#pragma unroll
  for (int d = 0; d < 3; ++d) X0[d] = __ldg(A.X + d * A.N + n0);
  const df h(A.h, A.hlo);
  df M[3][3], B[3][3];
#pragma unroll
  for (int a = 1; a < EL::C; ++a) {
    const int na = __ldg(A.conn + a * E + e);
    int c[3];
    float o[3];
    A.pos.load(na, c, o);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const df od = two_sum(o[d], -o0[d]);                    // exact
      const df sc = two_sum(float(c[d] - c0[d]), od.hi);      // exact
      const df dx = dmul(df(sc.hi, __fadd_rn(sc.lo, od.lo)), h);
      const df dX = two_sum(__ldg(A.X + d * A.N + na), -X0[d]);  // exact
      const df du = dadd(dx, neg(dX));
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        M[d][j] = dfma(M[d][j], dX, float(EL::dxi(a, Q, j)));
        B[d][j] = dfma(B[d][j], du, float(EL::dxi(a, Q, j)));
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      M[i][j] = norm(M[i][j]);
      B[i][j] = norm(B[i][j]);
    }
  df CM[3][3], CB[3][3];
  cof3(M, CM);
  cof3(B, CB);
  df t, j0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      t = dfma(t, CM[i][j], B[i][j]);
      t = dfma(t, M[i][j], CB[i][j]);
    }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    t = dfma(t, B[0][j], CB[0][j]);
    j0 = dfma(j0, M[0][j], CM[0][j]);
  }
  return ddiv(norm(t), norm(j0));
}

template <int kEl>
__global__ void __launch_bounds__(128) k_exact_jm1(FeArgs<float> A, float2* __restrict__ jx) {
  using EL = El<kEl>;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)EL::QF * A.E) return;
  const int q = (int)(t / A.E), e = (int)(t % A.E);
  df r;
  switch (q) {  // q is uniform across a warp except where two q blocks meet
    case 0: r = exact_jm1_at<kEl, 0>(A, e); break;
    case 1: if constexpr (EL::QF > 1) r = exact_jm1_at<kEl, 1 % EL::QF>(A, e); break;
    case 2: if constexpr (EL::QF > 2) r = exact_jm1_at<kEl, 2 % EL::QF>(A, e); break;
    case 3: if constexpr (EL::QF > 3) r = exact_jm1_at<kEl, 3 % EL::QF>(A, e); break;
    case 4: if constexpr (EL::QF > 4) r = exact_jm1_at<kEl, 4 % EL::QF>(A, e); break;
    case 5: if constexpr (EL::QF > 5) r = exact_jm1_at<kEl, 5 % EL::QF>(A, e); break;
    case 6: if constexpr (EL::QF > 6) r = exact_jm1_at<kEl, 6 % EL::QF>(A, e); break;
    default: if constexpr (EL::QF > 7) r = exact_jm1_at<kEl, 7 % EL::QF>(A, e); break;
  }
  jx[t] = make_float2(r.hi, r.lo);
}

// Shape-function derivative dN_a/dxi_j of the trilinear hexahedron at Gauss
// point q, for a q known only at run time (the lane-per-point kernel): the
// compile-time table's three magnitudes, chosen by how many of the other two
// axes' corner signs match the point's, and the corner's sign along j.  The
// values are the same floats as Real(El<IB_ELEM_HEX8>::dxi(a, q, j)).
template <typename Real, int a, int j>
__device__ __forceinline__ Real hex_dxi(int q) {
  constexpr Real kAA = Real(0.5 * (kA * kA)), kAB = Real(0.5 * (kA * kB)),
                 kBB = Real(0.5 * (kB * kB));
  constexpr int k1 = (j + 1) % 3, k2 = (j + 2) % 3;
  // corner a's sign bits (bit k set: + along axis k); q's bit k set: + along k
  constexpr int sa = (corner_sign(a, 0) > 0) | (corner_sign(a, 1) > 0) << 1 |
                     (corner_sign(a, 2) > 0) << 2;
  const int diff = (sa ^ q) & ((1 << k1) | (1 << k2));  // the other two axes that differ
  const Real m = diff == 0 ? kAA : (__popc(diff) == 1 ? kAB : kBB);
  return corner_sign(a, j) > 0 ? m : -m;
}

// Butterfly reduce-scatter over the 8 lanes of an element (lane = Gauss
// point g): on entry each lane holds its point's corner contributions
// G[a][i], a = 0..7; on exit lane g holds the sum over the 8 points of
// corner g's, summed in a fixed tree (lanes 4 apart, then 2, then 1).
template <typename Real>
__device__ __forceinline__ void reduce_scatter8(Real G[8][3], int g, Real out[3]) {
  const unsigned full = 0xffffffffu;
  Real h4[4][3];  // after the first level: the 4 corners with bit 2 = g's
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const bool hi = g & 4;
      const Real keep = hi ? G[4 + k][i] : G[k][i], send = hi ? G[k][i] : G[4 + k][i];
      h4[k][i] = keep + __shfl_xor_sync(full, send, 4);
    }
  Real h2[2][3];  // corners with bits 2, 1 = g's
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const bool hi = g & 2;
      const Real keep = hi ? h4[2 + k][i] : h4[k][i], send = hi ? h4[k][i] : h4[2 + k][i];
      h2[k][i] = keep + __shfl_xor_sync(full, send, 2);
    }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const bool hi = g & 1;
    const Real keep = hi ? h2[1][i] : h2[0][i], send = hi ? h2[0][i] : h2[1][i];
    out[i] = keep + __shfl_xor_sync(full, send, 1);
  }
}

// Sum over the 8 lanes of an element, in a fixed tree (every lane gets it).
template <typename T>
__device__ __forceinline__ T sum8(T v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// One element's nodal forces (or their adjoint).  kLanes = false: one thread
// per element, its force points unrolled with compile-time shape values.
// kLanes = true (hexahedra): eight consecutive lanes per element, lane g
// evaluating Gauss point g; the corner data are exchanged by shuffles, and
// lane g writes corner g's force (valid = false: a lane of a padding element
// takes part in the shuffles and stores nothing).
// kPacked: an element of a packed plan (its instance's h; its material row in
// the device table); false: the plan's h and the table passed by value.
template <typename Real, typename S, bool kEnergy, bool kAdj, bool kParams, int kLaws, int kEl,
          bool kLanes = false, bool kPacked = false>
__device__ __forceinline__ void fe_element(const FeArgs<Real>& A, const MatTable& mt, int e,
                                           bool valid = true) {
  using EL = El<kEl>;
  static_assert(!kLanes || kEl == IB_ELEM_HEX8, "eight lanes per element: hexahedra");
  const int E = A.E;
  constexpr bool volx = (kLaws & kLawVolX) != 0;
  static_assert(!volx || (std::is_same<Real, float>::value && std::is_same<S, df>::value),
                "the exact volumetric invariant is a split-precision option");
  const int g = threadIdx.x & 7;  // kLanes: this lane's Gauss point and corner

  // reference and current coordinates relative to corner 0 (kLanes: this
  // lane's corner only; the others arrive by shuffles)
  constexpr int kNodes = kLanes ? 1 : EL::C;
  // grid spacing of the element's structure
  Real h = A.h;
  if constexpr (kPacked) h = Real(__ldg(&A.inst[__ldg(A.elem_inst + e)].h));
  Real dX[kNodes][3], du[kNodes][3];
  Real vv[kAdj ? kNodes : 1][3];
  {
    int node[kNodes];
#pragma unroll
    for (int a = 0; a < kNodes; ++a) node[a] = __ldg(A.conn + (kLanes ? g : a) * E + e);
    int c0[3];
    Real o0[3], X0[3];
    if constexpr (kLanes) {
      int c[3];
      Real o[3];
      A.pos.load(node[0], c, o);
      const unsigned full = 0xffffffffu;
      const int src = threadIdx.x & 24;  // lane 0 of this element's group
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        c0[d] = __shfl_sync(full, c[d], src);
        o0[d] = __shfl_sync(full, o[d], src);
        const Real X = __ldg(A.X + d * A.N + node[0]);
        X0[d] = __shfl_sync(full, X, src);
        dX[0][d] = X - X0[d];
        const Real dx = (Real(c[d] - c0[d]) + (o[d] - o0[d])) * h;
        du[0][d] = dx - dX[0][d];
      }
    } else {
      A.pos.load(node[0], c0, o0);
#pragma unroll
      for (int d = 0; d < 3; ++d) X0[d] = __ldg(A.X + d * A.N + node[0]);
#pragma unroll
      for (int a = 0; a < kNodes; ++a) {
        int c[3];
        Real o[3];
        if (a == 0) {
#pragma unroll
          for (int d = 0; d < 3; ++d) { dX[0][d] = Real(0); du[0][d] = Real(0); }
          continue;
        }
        A.pos.load(node[a], c, o);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          dX[a][d] = __ldg(A.X + d * A.N + node[a]) - X0[d];
          Real dx = (Real(c[d] - c0[d]) + (o[d] - o0[d])) * h;
          du[a][d] = dx - dX[a][d];
        }
      }
    }
    if (kAdj) {
#pragma unroll
      for (int a = 0; a < kNodes; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) vv[a][d] = __ldg(A.v + d * A.N + node[a]);
    }
  }

  const int mid = A.mat_id ? __ldg(A.mat_id + e) : 0;
  // the material row: the table passed by value, or the device table
  int model;
  if constexpr (kPacked)
    model = __ldg(&A.mats[mid].model);
  else
    model = mt.model[mid];
  const auto prm = [&](int k) -> double {
    if constexpr (kPacked) return __ldg(&A.mats[mid].p[k]);
    return mt.p[mid][k];
  };
  // a parameter in Real: FP32 plans read the table's FP32 roundings (the same
  // values a conversion here would give, without the FP64-rate conversion)
  const auto prmr = [&](int k) -> Real {
    if constexpr (sizeof(Real) == 4) {
      if constexpr (kPacked) return __ldg(&A.mats[mid].pf[k]);
      return mt.pf[mid][k];
    }
    return Real(prm(k));
  };
  const bool ta_on = kPacked ? __ldg(&A.mats[mid].act) != 0 : mt.act[mid] != 0;
  // the laws this instantiation handles (kLaws bit m: ib_model m; bit
  // kLawActBit: the active term); the host picks an instantiation whose set
  // covers the material table, and every other branch compiles away
  const bool lawNH = (kLaws & 1) && model == IB_NEO_HOOKEAN;
  const bool lawF1 = (kLaws & 2) && model == IB_FIBRE1;
  const bool lawHO = (kLaws & 4) && model == IB_HO;
  const bool lawSR = (kLaws & 8) && model == IB_STD_REINF;
  const bool lawF2 = (kLaws & 16) && model == IB_FIBRE2;
  Real ef[3] = {Real(1), Real(0), Real(0)}, es[3] = {Real(0), Real(1), Real(0)};
  if (A.fib) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      ef[i] = __ldg(A.fib + i * E + e);
      es[i] = __ldg(A.fib + (3 + i) * E + e);
    }
  }
  // |e|^2 - 1 and e_f . e_s as compensated sums of exact products in S
  const S efn1 = dacc(dacc(dacc(S(-1), ef[0], ef[0]), ef[1], ef[1]), ef[2], ef[2]);
  const S esn1 = dacc(dacc(dacc(S(-1), es[0], es[0]), es[1], es[1]), es[2], es[2]);
  const S efes = dacc(dacc(dacc(S(0), ef[0], es[0]), ef[1], es[1]), ef[2], es[2]);
  const Real esn1r = Real(esn1), efesr = Real(efes);

  // material constants (unused entries of a model are never read by its branches)
  const Real kap = prmr(lawNH ? 1 : (lawHO ? 8 : (lawF2 ? 4 : 3)));
  const Real pa = prmr(0), pb = prmr(1);
  const Real paf = prmr(lawF1 ? 1 : 2), pbf = prmr(lawF1 ? 2 : 3);
  const Real pas = prmr(4), pbs = prmr(5), pafs = prmr(6), pbfs = prmr(7);
  // active fibre tension (Section 6.1); the parameter adjoint always needs
  // its fibre kinematics for d/dT_a
  static_assert(!kParams || (kLaws & kLawAct), "the parameter adjoint computes d/dT_a");
  const Real Ta = prmr(kTa);
  const bool act = (kLaws & kLawAct) && (kParams || ta_on);

  double en = 0.0;
  Real gp[kParamRow];
#pragma unroll
  for (int k = 0; k < kParamRow; ++k) gp[k] = Real(0);
  bool inverted = false;

  // One force point q: from J0 = sum_a dX_a (x) dN_a/dxi, Du = sum_a du_a (x)
  // dN_a/dxi and (adjoint) Dvv = sum_a v_a (x) dN_a/dxi, the stress (or its
  // derivative) as Qm = P J0^-T w j0, whose product with dN_a/dxi is corner
  // a's contribution; the energy and parameter sums accumulate in en, gp.
  auto point = [&](int q, const Real (&J0)[3][3], const Real (&Du)[3][3],
                   const Real (&Dvv)[3][3], Real (&Qm)[3][3]) {
    Real cJ[3][3];
    cofactor(J0, cJ);
    const Real j0 = J0[0][0] * cJ[0][0] + J0[0][1] * cJ[0][1] + J0[0][2] * cJ[0][2];
    if (!(j0 > Real(0))) inverted = true;
    const Real wj = j0 * Real(EL::wF);  // the force rule's weight times det dX/dxi
    const Real ij0 = Real(1) / j0;
    // J0^-1 = cof(J0)^T / det
    Real Ji[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Ji[i][j] = cJ[j][i] * ij0;
    Real H[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        H[i][j] = Du[i][0] * Ji[0][j] + Du[i][1] * Ji[1][j] + Du[i][2] * Ji[2][j];

    // ---- invariants --------------------------------------------------------
    // J - 1 = tr H + ((tr H)^2 - tr(H^2))/2 + det H, the middle term written as
    // the sum of the principal 2x2 minors H_ii H_jj - H_ij H_ji: a compensated
    // sum in S of the FP32 entries of H and of their exact pairwise products
    // (near incompressibility tr H cancels to |J - 1| << |H|); det H (third
    // order) is taken in Real.
    S Jm1;
    if constexpr (volx) {
      const float2 jq = __ldg(A.jx + (int64_t)q * E + e);
      Jm1 = S(jq.x, jq.y);
    } else {
      Jm1 = dacc(S(0), H[0][0], H[1][1]);
      Jm1 = dacc(Jm1, H[0][0], H[2][2]);
      Jm1 = dacc(Jm1, H[1][1], H[2][2]);
      Jm1 = dacc(Jm1, -H[0][1], H[1][0]);
      Jm1 = dacc(Jm1, -H[0][2], H[2][0]);
      Jm1 = dacc(Jm1, -H[1][2], H[2][1]);
      Jm1 = sacc(sacc(sacc(sacc(Jm1, H[0][0]), H[1][1]), H[2][2]), det3(H));
    }
    const S lnJs = log1p_s(Jm1);
    const Real lnJ = Real(lnJs);
    const Real J = Real(1) + Real(Jm1);
    Real F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) F[i][j] = H[i][j] + (i == j ? Real(1) : Real(0));
    Real FiT[3][3];
    cofactor(F, FiT);
    const Real iJ = Real(1) / J;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) FiT[i][j] *= iJ;
    Real HH = Real(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) HH += H[i][j] * H[i][j];
    const Real I1m3 = Real(2) * (H[0][0] + H[1][1] + H[2][2]) + HH;
    const Real Jm23m1 = expm1(Real(-2.0 / 3.0) * lnJ);
    const Real Jm23 = Real(1) + Jm23m1;
    const Real Ibm3 = Jm23 * I1m3 + Real(3) * Jm23m1;  // I1bar - 3
    const Real I1o3 = Real(1) + I1m3 * Real(1.0 / 3.0);
    Real Dv[3][3];  // J^-2/3 (F - I1/3 F^-T)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Dv[i][j] = Jm23 * (F[i][j] - I1o3 * FiT[i][j]);

    // ---- constitutive law -----------------------------------------------------
    Real ciso;
    Real eiso = Real(1);  // Psi_4: exp(b (I1bar - 3)); Psi_3: exp(C01 (I1bar - 3))
    if (lawHO) {
      eiso = exp(pb * Ibm3);
      ciso = pa * eiso;
    } else if (lawF2) {
      eiso = exp(pb * Ibm3);
      ciso = Real(2) * pa * pb * eiso;
    } else if (lawSR) {
      ciso = pa;  // G_T
    } else {
      ciso = Real(2) * pa;
    }
    // Fibre family f (the fibre of Psi_2 and of Psi_4): I4f - 1 combined in S.
    // Its exponential factor and coefficient are then products of that small
    // number, with no cancellation left, and are formed in Real.
    Fibre<Real, S> f1;
    Fibre<Real, Real> f2;
    Real d1 = Real(0), cf1 = Real(0), ef1 = Real(1), cf2 = Real(0), ef2 = Real(1);
    const bool has_f = lawF1 || lawHO || lawSR || lawF2 || act;
    const bool has_s = lawHO;
    // active stress P^a = T F e (x) e, T = T_a g, g = 1 + 4.9 (sqrt(I4f) - 1)
    // with sqrt(I4f) - 1 = (I4f - 1)/(sqrt(I4f) + 1); T is added to the fibre
    // coefficient cf1
    Real sq4 = Real(1), gact = Real(1), Tact = Real(0);
    // Psi_1 (model 3): the I4f term (E_L + G_T - 4 G_L)/2 (I4f - 1) F e (x) e,
    // k4 = (E_L + G_T - 4 G_L)/2, and the I5f term
    // (G_T - G_L)(2 Fe (x) e - Fe (x) Ce - FCe (x) e) = -(G_T - G_L)(Fe (x) w + Fw (x) e)
    // with C e = e + w, w = H e + H^T e + H^T H e (no cancellation for small H)
    const Real k4 = lawSR ? Real(0.5) * (prmr(2) + pa - Real(4) * pb) : Real(0);
    const Real c5 = lawSR ? pa - pb : Real(0);
    Real w5[3] = {Real(0), Real(0), Real(0)}, Fw5[3] = {Real(0), Real(0), Real(0)};
    if (has_f) {
      fibre_kin<Real, S>(H, ef, efn1, f1, lawF1 || lawHO);
      d1 = Real(f1.d);
      if (lawSR) {
        cf1 = k4 * d1;
        Real He[3], HtHe[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) He[i] = f1.Fe[i] - ef[i];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          HtHe[j] = H[0][j] * He[0] + H[1][j] * He[1] + H[2][j] * He[2];
          w5[j] = He[j] + (H[0][j] * ef[0] + H[1][j] * ef[1] + H[2][j] * ef[2]) + HtHe[j];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
          Fw5[i] = w5[i] + H[i][0] * w5[0] + H[i][1] * w5[1] + H[i][2] * w5[2];
      } else if (lawF1 || lawHO || lawF2) {
        ef1 = exp(pbf * d1 * d1);
        cf1 = Real(2) * paf * d1 * ef1;
      }
      if (act) {
        const Real d4 = Real(f1.d4);
        sq4 = sqrt(Real(1) + d4);
        gact = Real(1) + Real(4.9) * (d4 / (sq4 + Real(1)));
        Tact = Ta * gact;
      }
    }
    // Sheet family and the fibre-sheet coupling (HO only) in Real, with the
    // same cancellation-free formulas.
    Real Fef[3], Fes[3];
    Real I8 = Real(0), e8 = Real(1), c8 = Real(0);
    if (has_s) {
      fibre_kin<Real, Real>(H, es, esn1r, f2);
      ef2 = exp(pbs * f2.d * f2.d);
      cf2 = Real(2) * pas * f2.d * ef2;
      Real Hef[3], Hes[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        Hef[i] = H[i][0] * ef[0] + H[i][1] * ef[1] + H[i][2] * ef[2];
        Hes[i] = H[i][0] * es[0] + H[i][1] * es[1] + H[i][2] * es[2];
        Fef[i] = ef[i] + Hef[i];
        Fes[i] = es[i] + Hes[i];
      }
      I8 = efesr;
#pragma unroll
      for (int i = 0; i < 3; ++i) I8 += ef[i] * Hes[i] + es[i] * Hef[i] + Hef[i] * Hes[i];
      e8 = exp(pbfs * I8 * I8);
      c8 = pafs * I8 * e8;
    }

    if (kEnergy) {
      double psi = 0.5 * double(kap) * double(lnJs) * double(lnJs);
      if (lawNH || lawF1) psi += prm(0) * double(Ibm3);
      else if (lawHO) psi += prm(0) / (2.0 * prm(1)) * expm1(prm(1) * double(Ibm3));
      else if (lawSR) psi += 0.5 * prm(0) * double(Ibm3);
      else if (lawF2) psi += prm(0) * expm1(prm(1) * double(Ibm3));
      if (lawSR) {
        const double ww = double(w5[0]) * w5[0] + double(w5[1]) * w5[1] + double(w5[2]) * w5[2];
        psi += 0.5 * double(c5) * (double(efn1) - ww) + 0.25 * double(k4) * double(f1.d) * double(f1.d);
      } else if (lawF1 || lawHO || lawF2) {  // the exponential fibre term of Psi_2, Psi_3, Psi_4
        const double af = prm(lawF1 ? 1 : 2), bf = prm(lawF1 ? 2 : 3);
        psi += af / (2.0 * bf) * expm1(bf * double(f1.d) * double(f1.d));
      }
      if (has_s) {
        psi += prm(4) / (2.0 * prm(5)) * expm1(prm(5) * double(f2.d) * double(f2.d));
        psi += prm(6) / (2.0 * prm(7)) * expm1(prm(7) * double(I8) * double(I8));
      }
      if (act) {
        // T_a/2 [(1 - 4.9)(I4 - 1) + 4.9 (2/3)(I4^(3/2) - 1)] with
        // I4^(3/2) - 1 = (I4 - 1)(I4 + sqrt(I4) + 1)/(sqrt(I4) + 1)
        const double d4 = double(f1.d4), r = sqrt(1.0 + d4);
        psi += 0.5 * prm(kTa) * d4 * ((1.0 - 4.9) + 4.9 * (2.0 / 3.0) * (2.0 + d4 + r) / (r + 1.0));
      }
      en += psi * double(wj);
    }

    // stress (forward) or its directional derivative (adjoint)
    Real P[3][3];
    if (!kAdj) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) P[i][j] = ciso * Dv[i][j] + kap * lnJ * FiT[i][j];
      if (has_f) {
        const Real c = cf1 + Tact;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) P[i][j] += c * f1.Fe[i] * ef[j];
      }
      if (lawSR) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) P[i][j] -= c5 * (f1.Fe[i] * w5[j] + Fw5[i] * ef[j]);
      }
      if (has_s) {
        const Real c = Real(cf2), k8 = Real(c8);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j)
            P[i][j] += c * f2.Fe[i] * es[j] + k8 * (Fef[i] * es[j] + Fes[i] * ef[j]);
      }
    } else {
      // dF = Dvv J0^-1
      Real dF[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          dF[i][j] = Dvv[i][0] * Ji[0][j] + Dvv[i][1] * Ji[1][j] + Dvv[i][2] * Ji[2][j];
      // delta = d ln J = F^-T : dF ; dI1 = 2 F : dF ; d F^-T = -F^-T dF^T F^-T
      Real dl = Real(0), dI1 = Real(0), DdF = Real(0);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          dl += FiT[i][j] * dF[i][j];
          dI1 += Real(2) * F[i][j] * dF[i][j];
          DdF += Dv[i][j] * dF[i][j];
        }
      Real M[3][3];  // F^-T dF^T
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          M[i][j] = FiT[i][0] * dF[j][0] + FiT[i][1] * dF[j][1] + FiT[i][2] * dF[j][2];
      Real dFiT[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          dFiT[i][j] = -(M[i][0] * FiT[0][j] + M[i][1] * FiT[1][j] + M[i][2] * FiT[2][j]);
      const Real I1 = Real(3) + I1m3;
      const Real dbeta = Jm23 * (dI1 - Real(2.0 / 3.0) * I1 * dl);
      Real dciso = Real(0);
      if (lawHO || lawF2) dciso = ciso * pb * dbeta;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const Real dD = Real(-2.0 / 3.0) * dl * Dv[i][j] +
                          Jm23 * (dF[i][j] - dI1 * Real(1.0 / 3.0) * FiT[i][j] -
                                  I1o3 * dFiT[i][j]);
          P[i][j] = ciso * dD + dciso * Dv[i][j] + kap * (dl * FiT[i][j] + lnJ * dFiT[i][j]);
        }
      Real dI4f = Real(0), dI4s = Real(0), dI8 = Real(0);
      if (has_f) {
        Real dFe[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) dFe[i] = dF[i][0] * ef[0] + dF[i][1] * ef[1] + dF[i][2] * ef[2];
        dI4f = Real(2) * (f1.Fe[0] * dFe[0] + f1.Fe[1] * dFe[1] + f1.Fe[2] * dFe[2]);
        Real dc = Real(0);
        if (lawSR)
          dc = k4 * dI4f;
        else if (lawF2 || ((lawF1 || lawHO) && d1 > Real(0)))
          dc = Real(2) * paf * ef1 * (Real(1) + Real(2) * pbf * d1 * d1) * dI4f;
        if (act) dc += Ta * Real(4.9 / 2.0) * dI4f / sq4;  // dT = T_a 4.9 dI4f / (2 sqrt(I4f))
        const Real c = cf1 + Tact;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) P[i][j] += (dc * f1.Fe[i] + c * dFe[i]) * ef[j];
      }
      // Psi_1's I5f term: d[-(G_T - G_L)(Fe (x) w + Fw (x) e)] with
      // dw = dF e + dF^T e + dF^T H e + H^T dF e
      Real X5 = Real(0);  // (Fe (x) w + Fw (x) e) : dF
      if (lawSR) {
        Real dFe[3], dFw[3], dw[3], Fdw[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          dFe[i] = dF[i][0] * ef[0] + dF[i][1] * ef[1] + dF[i][2] * ef[2];
          dFw[i] = dF[i][0] * w5[0] + dF[i][1] * w5[1] + dF[i][2] * w5[2];
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          Real t = dFe[j];
#pragma unroll
          for (int i = 0; i < 3; ++i)
            t += dF[i][j] * f1.Fe[i] + H[i][j] * dFe[i];  // dF^T (e + He) + H^T dF e
          dw[j] = t;
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
          Fdw[i] = dw[i] + H[i][0] * dw[0] + H[i][1] * dw[1] + H[i][2] * dw[2];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j)
            P[i][j] -= c5 * (dFe[i] * w5[j] + f1.Fe[i] * dw[j] + dFw[i] * ef[j] + Fdw[i] * ef[j]);
        X5 = f1.Fe[0] * dFw[0] + f1.Fe[1] * dFw[1] + f1.Fe[2] * dFw[2] + Fw5[0] * dFe[0] +
             Fw5[1] * dFe[1] + Fw5[2] * dFe[2];
      }
      if (has_s) {
        Real dFs[3], dFf[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          dFs[i] = dF[i][0] * es[0] + dF[i][1] * es[1] + dF[i][2] * es[2];
          dFf[i] = dF[i][0] * ef[0] + dF[i][1] * ef[1] + dF[i][2] * ef[2];
        }
        dI4s = Real(2) * (f2.Fe[0] * dFs[0] + f2.Fe[1] * dFs[1] + f2.Fe[2] * dFs[2]);
        const Real dc =
            f2.d > Real(0)
                ? Real(2) * pas * ef2 * (Real(1) + Real(2) * pbs * f2.d * f2.d) * dI4s
                : Real(0);
        const Real c = Real(cf2);
        dI8 = dFf[0] * Fes[0] + dFf[1] * Fes[1] + dFf[2] * Fes[2] + Fef[0] * dFs[0] +
              Fef[1] * dFs[1] + Fef[2] * dFs[2];
        const Real dk8 = pafs * e8 * (Real(1) + Real(2) * pbfs * I8 * I8) * dI8;
        const Real k8 = c8;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j)
            P[i][j] += (dc * f2.Fe[i] + c * dFs[i]) * es[j] +
                       dk8 * (Fef[i] * es[j] + Fes[i] * ef[j]) +
                       k8 * (dFf[i] * es[j] + dFs[i] * ef[j]);
      }
      if (kParams) {
        // gparams_k = -sum_q w j0 (dP/dtheta_k : dF): the element's eight
        // terms in Real, the sums over elements in double
        const Real w = wj;
        const Real vol = lnJ * dl;
        gp[kTa] -= w * gact * Real(0.5) * dI4f;  // (g F e (x) e) : dF
        if (lawNH) {
          gp[0] -= w * Real(2) * DdF;
          gp[1] -= w * vol;
        } else if (lawF1) {
          gp[0] -= w * Real(2) * DdF;
          gp[1] -= w * d1 * ef1 * dI4f;
          gp[2] -= w * paf * d1 * d1 * d1 * ef1 * dI4f;
          gp[3] -= w * vol;
        } else if (lawSR) {  // {G_T, G_L, E_L, kappa}; (Fe (x) e) : dF = dI4f / 2
          const Real y4 = Real(0.5) * dI4f;
          gp[0] -= w * (DdF - X5 + Real(0.5) * d1 * y4);
          gp[1] -= w * (X5 - Real(2) * d1 * y4);
          gp[2] -= w * (Real(0.5) * d1 * y4);
          gp[3] -= w * vol;
        } else if (lawF2) {  // {C10, C01, af, bf, kappa}
          gp[0] -= w * Real(2) * pb * eiso * DdF;
          gp[1] -= w * Real(2) * pa * eiso * (Real(1) + pb * Ibm3) * DdF;
          gp[2] -= w * d1 * ef1 * dI4f;
          gp[3] -= w * paf * d1 * d1 * d1 * ef1 * dI4f;
          gp[4] -= w * vol;
        } else if (lawHO) {
          gp[0] -= w * eiso * DdF;
          gp[1] -= w * pa * Ibm3 * eiso * DdF;
          gp[2] -= w * d1 * ef1 * dI4f;
          gp[3] -= w * paf * d1 * d1 * d1 * ef1 * dI4f;
          gp[4] -= w * f2.d * ef2 * dI4s;
          gp[5] -= w * pas * f2.d * f2.d * f2.d * ef2 * dI4s;
          gp[6] -= w * I8 * e8 * dI8;
          gp[7] -= w * pafs * I8 * I8 * I8 * e8 * dI8;
          gp[8] -= w * vol;
        }
      }
    }

    // corner forces: G_a -= (P J0^-T w j0) dN_a/dxi
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        Qm[i][k] = (P[i][0] * Ji[k][0] + P[i][1] * Ji[k][1] + P[i][2] * Ji[k][2]) * wj;
  };

  if constexpr (!kLanes) {
    Real Ge[EL::C][3];
#pragma unroll
    for (int a = 0; a < EL::C; ++a)
#pragma unroll
      for (int d = 0; d < 3; ++d) Ge[a][d] = Real(0);
#pragma unroll
    for (int q = 0; q < EL::QF; ++q) {
      Real J0[3][3], Du[3][3], Dvv[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          Real s = Real(0), t = Real(0), w = Real(0);
#pragma unroll
          for (int a = 1; a < EL::C; ++a) {
            s += dX[a][i] * Real(EL::dxi(a, q, j));
            t += du[a][i] * Real(EL::dxi(a, q, j));
          }
          if (kAdj) {
#pragma unroll
            for (int a = 0; a < EL::C; ++a) w += vv[a][i] * Real(EL::dxi(a, q, j));
          }
          J0[i][j] = s;
          Du[i][j] = t;
          Dvv[i][j] = w;
        }
      Real Qm[3][3];
      point(q, J0, Du, Dvv, Qm);
#pragma unroll
      for (int a = 0; a < EL::C; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i)
          Ge[a][i] -= Qm[i][0] * Real(EL::dxi(a, q, 0)) + Qm[i][1] * Real(EL::dxi(a, q, 1)) +
                      Qm[i][2] * Real(EL::dxi(a, q, 2));
    }
    if (inverted) set_status(A.status, kStatInverted);
#pragma unroll
    for (int a = 0; a < EL::C; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) A.out[(a * 3 + i) * E + e] = Ge[a][i];
    if (kEnergy) A.epart[e] = en;
    if (kParams) {
#pragma unroll
      for (int k = 0; k < kParamRow; ++k) reinterpret_cast<Real*>(A.epart)[(int64_t)k * E + e] = gp[k];
    }
  } else {
    // the corners' data from their lanes, accumulated into this lane's point
    const unsigned full = 0xffffffffu;
    const int base = threadIdx.x & 24;
    Real J0[3][3], Du[3][3], Dvv[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) J0[i][j] = Du[i][j] = Dvv[i][j] = Real(0);
    auto gather = [&](auto a_) {
      constexpr int a = decltype(a_)::value;
      const Real dn[3] = {hex_dxi<Real, a, 0>(g), hex_dxi<Real, a, 1>(g),
                          hex_dxi<Real, a, 2>(g)};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const Real xa = __shfl_sync(full, dX[0][i], base + a);
        const Real ua = __shfl_sync(full, du[0][i], base + a);
        const Real va = kAdj ? __shfl_sync(full, vv[0][i], base + a) : Real(0);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          if (a > 0) {
            J0[i][j] += xa * dn[j];
            Du[i][j] += ua * dn[j];
          }
          if (kAdj) Dvv[i][j] += va * dn[j];
        }
      }
    };
    gather(std::integral_constant<int, 0>{});
    gather(std::integral_constant<int, 1>{});
    gather(std::integral_constant<int, 2>{});
    gather(std::integral_constant<int, 3>{});
    gather(std::integral_constant<int, 4>{});
    gather(std::integral_constant<int, 5>{});
    gather(std::integral_constant<int, 6>{});
    gather(std::integral_constant<int, 7>{});
    Real Qm[3][3];
    point(g, J0, Du, Dvv, Qm);
    Real Gq[8][3];
    auto corner = [&](auto a_) {
      constexpr int a = decltype(a_)::value;
      const Real d0 = hex_dxi<Real, a, 0>(g), d1 = hex_dxi<Real, a, 1>(g),
                 d2 = hex_dxi<Real, a, 2>(g);
#pragma unroll
      for (int i = 0; i < 3; ++i) Gq[a][i] = -(Qm[i][0] * d0 + Qm[i][1] * d1 + Qm[i][2] * d2);
    };
    corner(std::integral_constant<int, 0>{});
    corner(std::integral_constant<int, 1>{});
    corner(std::integral_constant<int, 2>{});
    corner(std::integral_constant<int, 3>{});
    corner(std::integral_constant<int, 4>{});
    corner(std::integral_constant<int, 5>{});
    corner(std::integral_constant<int, 6>{});
    corner(std::integral_constant<int, 7>{});
    Real mine[3];
    reduce_scatter8(Gq, g, mine);
    if (kEnergy) en = sum8(en);
    if (kParams) {
#pragma unroll
      for (int k = 0; k < kParamRow; ++k) gp[k] = sum8(gp[k]);
    }
    if (valid) {
      if (inverted) set_status(A.status, kStatInverted);
#pragma unroll
      for (int i = 0; i < 3; ++i) A.out[(g * 3 + i) * E + e] = mine[i];
      if (g == 0) {
        if (kEnergy) A.epart[e] = en;
        if (kParams) {
#pragma unroll
          for (int k = 0; k < kParamRow; ++k) reinterpret_cast<Real*>(A.epart)[(int64_t)k * E + e] = gp[k];
        }
      }
    }
  }
}

// Persistent grid (a fixed number of CTAs per SM, fewer than fit): the SM
// room the kernel leaves lets the Gauss-point binning and the interpolation,
// issued on another stream, run beside it.
// CTAs take blocks of elements from a counter, so a CTA that becomes resident
// late (its SM busy with those kernels) simply takes fewer.
template <typename Real, typename S, bool kEnergy, bool kAdj, bool kParams, int kLaws, int kEl>
__global__ void __launch_bounds__(128, fe_min_blocks<Real, kAdj>())
    k_fe(FeArgs<Real> A, MatTable mt) {
  __shared__ int base;
  for (;;) {
    if (threadIdx.x == 0) base = atomicAdd(A.next, 1) * (int)blockDim.x;
    __syncthreads();
    const int b = base;
    __syncthreads();
    if (b >= A.E) break;
    if (b + (int)threadIdx.x < A.E)
      fe_element<Real, S, kEnergy, kAdj, kParams, kLaws, kEl>(A, mt, b + (int)threadIdx.x);
  }
}

// Hexahedra: eight lanes per element (lane g: Gauss point g), sixteen
// elements per 128-thread CTA, blocks of elements taken from a counter.
template <typename Real, bool kAdj>
constexpr int fe8_min_blocks() {
  return sizeof(Real) == 8 ? 2 : (kAdj ? 4 : 5);
}

template <typename Real, typename S, bool kEnergy, bool kAdj, bool kParams, int kLaws,
          bool kPacked = false>
__global__ void __launch_bounds__(128, fe8_min_blocks<Real, kAdj>())
    k_fe8(FeArgs<Real> A, MatTable mt) {
  constexpr int kPer = 128 / 8;
  __shared__ int base;
  for (;;) {
    if (threadIdx.x == 0) base = atomicAdd(A.next, 1) * kPer;
    __syncthreads();
    const int b = base;
    __syncthreads();
    if (b >= A.E) break;
    const int e = b + (int)(threadIdx.x >> 3);
    fe_element<Real, S, kEnergy, kAdj, kParams, kLaws, IB_ELEM_HEX8, true, kPacked>(
        A, mt, e < A.E ? e : A.E - 1, e < A.E);
  }
}

template <typename Real>
FeArgs<Real> make_args(ib_plan* p, const void* xa, const float* off, const void* v, void* out);

template <>
inline FeArgs<float> make_args<float>(ib_plan* p, const void* xa, const float* off, const void* v,
                               void* out) {
  FeArgs<float> A;
  A.E = p->E;
  A.N = p->N;
  A.conn = p->conn;
  A.X = (const float*)p->X;
  A.fib = (const float*)p->fibres;
  A.mat_id = p->mat_id;
  A.pos.cell = (const int32_t*)xa;
  A.pos.off = off;
  A.pos.N = p->N;
  A.h = (float)p->grid.h;
  A.hlo = (float)(p->grid.h - (double)A.h);
  A.jx = (const float2*)p->vol_jm1;
  A.v = (const float*)v;
  A.out = (float*)out;
  A.epart = p->epart;
  A.status = p->dstatus;
  A.next = p->tile_counters + 6;
  A.inst = p->n_inst > 1 ? p->inst : nullptr;
  A.elem_inst = p->n_inst > 1 ? p->elem_inst : nullptr;
  A.mats = p->mat_dev;
  return A;
}

template <>
inline FeArgs<double> make_args<double>(ib_plan* p, const void* xa, const float*, const void* v,
                                 void* out) {
  FeArgs<double> A;
  A.E = p->E;
  A.N = p->N;
  A.conn = p->conn;
  A.X = (const double*)p->X;
  A.fib = (const double*)p->fibres;
  A.mat_id = p->mat_id;
  A.pos.x64 = (const double*)xa;
  A.pos.N = p->N;
  for (int d = 0; d < 3; ++d) A.pos.origin[d] = p->grid.origin[d];
  A.pos.inv_h = 1.0 / p->grid.h;
  A.h = p->grid.h;
  A.hlo = 0.f;
  A.jx = nullptr;
  A.v = (const double*)v;
  A.out = (double*)out;
  A.epart = p->epart;
  A.status = p->dstatus;
  A.next = p->tile_counters + 6;
  A.inst = nullptr;  // packed plans are FP32
  A.elem_inst = nullptr;
  A.mats = nullptr;
  return A;
}

}  // namespace

// The force launch of packed plans (FP32 split, hexahedra, no energy): declared
// here, defined and instantiated in fe_force_batch.cu only.
template <bool kAdj, bool kParams, int kLaws>
ib_status fe_run_packed(ib_plan* p, const MatTable& mt, const void* xa, const float* off,
                        const void* v, void* out, cudaStream_t s);

// Launch the force kernel for one (precision, output, law set, element) choice.
template <typename Real, typename S, bool kEnergy, bool kAdj, bool kParams, int kLaws, int kEl>
ib_status fe_run(ib_plan* p, const MatTable& mt, const void* xa, const float* off, const void* v,
                 void* out, cudaStream_t s) {
  if (p->E == 0) return IB_OK;
  if (p->n_inst > 1) {  // packed plans: FP32 split hexahedra, no energy
    if constexpr (kEl == IB_ELEM_HEX8 && std::is_same<Real, float>::value &&
                  std::is_same<S, df>::value && !kEnergy && (kLaws & kLawVolX) == 0)
      return fe_run_packed<kAdj, kParams, kLaws>(p, mt, xa, off, v, out, s);
    else
      return IB_ERR_INVALID_ARG;
  }
  FeArgs<Real> A = make_args<Real>(p, xa, off, v, out);
  const int threads = 128;
  // elements per CTA step: one per thread, or one per eight lanes (hexahedra)
  constexpr bool lanes = kEl == IB_ELEM_HEX8;
  const int per_cta = lanes ? threads / 8 : threads;
  // the forward runs beside the sort and interpolation; the adjoint runs alone
  const int per_sm = kAdj ? (lanes ? fe8_min_blocks<Real, kAdj>() : fe_min_blocks<Real, kAdj>())
                          : p->fe_ctas;
  const int blocks = std::min((p->E + per_cta - 1) / per_cta, p->sm_count * per_sm);
  if (cudaMemsetAsync(A.next, 0, sizeof(int), s) != cudaSuccess) return IB_ERR_CUDA;
  if constexpr ((kLaws & kLawVolX) != 0) {
    if (!p->vol_jm1) return IB_ERR_INVALID_ARG;
    const int64_t n = (int64_t)El<kEl>::QF * p->E;
    k_exact_jm1<kEl><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(A, (float2*)p->vol_jm1);
  }
  if constexpr (lanes)
    k_fe8<Real, S, kEnergy, kAdj, kParams, kLaws><<<blocks, threads, 0, s>>>(A, mt);
  else
    k_fe<Real, S, kEnergy, kAdj, kParams, kLaws, kEl><<<blocks, threads, 0, s>>>(A, mt);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

}  // namespace ibfe
