// Device helpers: trilinear-hex Gauss tables, the 4-point delta weights and
// position loading.  Shared by the kernels of libibfe (not by the oracle).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ib_internal.cuh"

namespace ibfe {

// ---------------------------------------------------------------------------
// Trilinear hexahedron at the 2x2x2 Gauss points (+-1/sqrt(3), unit weights).
// Corner a has signs c_a in VTK order; Gauss point q = b0 + 2 b1 + 4 b2 has
// signs s_q = 2 b - 1.  Per axis the linear factor (1 + c xi)/2 at xi = s g is
// kA = (1+g)/2 when c == s and kB = (1-g)/2 otherwise; N_a(xi_q) is the
// product of the three factors and dN_a/dxi_d = (c_ad / 2) * (product of the
// other two factors).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int corner_sign(int a, int d) {
  // VTK: 0(-,-,-) 1(+,-,-) 2(+,+,-) 3(-,+,-) 4(-,-,+) 5(+,-,+) 6(+,+,+) 7(-,+,+)
  return d == 0 ? ((a & 3) == 1 || (a & 3) == 2 ? 1 : -1)
                : (d == 1 ? ((a & 3) >= 2 ? 1 : -1) : (a >= 4 ? 1 : -1));
}
__host__ __device__ constexpr int gauss_sign(int q, int d) { return ((q >> d) & 1) ? 1 : -1; }
constexpr double kG = 0.57735026918962576451;  // 1/sqrt(3)
constexpr double kA = 0.5 * (1.0 + kG);
constexpr double kB = 0.5 * (1.0 - kG);
__host__ __device__ constexpr double lin_factor(int a, int q, int d) {
  return corner_sign(a, d) == gauss_sign(q, d) ? kA : kB;
}
__host__ __device__ constexpr double shapeN(int a, int q) {
  return lin_factor(a, q, 0) * lin_factor(a, q, 1) * lin_factor(a, q, 2);
}
__host__ __device__ constexpr double shape_dxi(int a, int q, int d) {
  return 0.5 * corner_sign(a, d) *
         (d == 0 ? lin_factor(a, q, 1) * lin_factor(a, q, 2)
                 : (d == 1 ? lin_factor(a, q, 0) * lin_factor(a, q, 2)
                           : lin_factor(a, q, 0) * lin_factor(a, q, 1)));
}

// ---------------------------------------------------------------------------
// Element types.  El<IB_ELEM_HEX8>: the trilinear hexahedron above; its force
// and its coupling points use the 2x2x2 Gauss rule (unit weights).
// El<IB_ELEM_TET4>: the linear tetrahedron on the unit reference tetrahedron
// (N_0 = 1 - xi - eta - zeta, N_1 = xi, N_2 = eta, N_3 = zeta; constant
// gradients); its coupling points are the symmetric 4-point rule of degree 2
// (barycentric (a, b, b, b) and permutations, point q nearest corner q,
// weights 1/24), and its force, whose integrand is constant, is evaluated
// once at the centroid with the whole reference volume 1/6.
// El<IB_ELEM_TET10>: the quadratic tetrahedron (P2), VTK node order (the 4
// vertices, then the nodes of edges 01, 12, 02, 03, 13, 23); with the
// barycentric coordinates L_i of P1, N = L_i (2 L_i - 1) at a vertex and
// 4 L_i L_j at the node of edge (i, j).  The same 4-point rule serves the
// force (degree 2: exact for P : grad N of an affine element under an affine
// deformation) and the coupling; its lumped mass scales the element's
// diagonal sum_q w_q j0 N_a^2 to the element's volume (kScaledMass).
//   C: nodes, Q: coupling points, QF: force points, N(a, q): shape value at
//   coupling point q, dxi(a, q, d): reference gradient at force point q,
//   wQ / wF: reference weights of the two rules.
// ---------------------------------------------------------------------------
template <int kEl>
struct El;

template <>
struct El<IB_ELEM_HEX8> {
  static constexpr int C = 8, Q = 8, QF = 8;
  static constexpr double wQ = 1.0, wF = 1.0;
  static constexpr bool kScaledMass = false;
  __host__ __device__ static constexpr double N(int a, int q) { return shapeN(a, q); }
  __host__ __device__ static constexpr double dxi(int a, int q, int d) {
    return shape_dxi(a, q, d);
  }
};

template <>
struct El<IB_ELEM_TET4> {
  static constexpr int C = 4, Q = 4, QF = 1;
  static constexpr double wQ = 1.0 / 24.0, wF = 1.0 / 6.0;
  static constexpr bool kScaledMass = false;
  static constexpr double kTa = 0.58541019662496845446;  // (5 + 3 sqrt 5) / 20
  static constexpr double kTb = 0.13819660112501051518;  // (5 - sqrt 5) / 20
  __host__ __device__ static constexpr double N(int a, int q) { return a == q ? kTa : kTb; }
  __host__ __device__ static constexpr double dxi(int a, int, int d) {
    return a == 0 ? -1.0 : (a - 1 == d ? 1.0 : 0.0);
  }
};

template <>
struct El<IB_ELEM_TET10> {
  static constexpr int C = 10, Q = 4, QF = 4;
  static constexpr double wQ = 1.0 / 24.0, wF = 1.0 / 24.0;
  static constexpr bool kScaledMass = true;
  // barycentric coordinate i at rule point q and its (constant) xi-gradient
  __host__ __device__ static constexpr double L(int i, int q) {
    return i == q ? El<IB_ELEM_TET4>::kTa : El<IB_ELEM_TET4>::kTb;
  }
  __host__ __device__ static constexpr double dL(int i, int d) {
    return El<IB_ELEM_TET4>::dxi(i, 0, d);
  }
  // vertices of the edge of node 4 + k
  __host__ __device__ static constexpr int ev0(int k) { return k == 1 ? 1 : (k == 4 ? 1 : (k == 5 ? 2 : 0)); }
  __host__ __device__ static constexpr int ev1(int k) { return k == 0 ? 1 : (k <= 2 ? 2 : 3); }
  __host__ __device__ static constexpr double N(int a, int q) {
    return a < 4 ? L(a, q) * (2.0 * L(a, q) - 1.0) : 4.0 * L(ev0(a - 4), q) * L(ev1(a - 4), q);
  }
  __host__ __device__ static constexpr double dxi(int a, int q, int d) {
    return a < 4 ? (4.0 * L(a, q) - 1.0) * dL(a, d)
                 : 4.0 * (L(ev0(a - 4), q) * dL(ev1(a - 4), d) + L(ev1(a - 4), q) * dL(ev0(a - 4), d));
  }
};

// ---------------------------------------------------------------------------
// 4-point delta weights.  For a point at t (grid units, staggering removed)
// with theta = t - floor(t) in [0,1), the four faces floor(t)-1 .. floor(t)+2
// are at distances r = theta+1, theta, theta-1, theta-2.  With
// q = sqrt(1 + 4 theta (1 - theta)) both branches of the kernel reduce to
//   phi(theta+1) = (3 - 2 theta - q)/8      phi(theta)   = (3 - 2 theta + q)/8
//   phi(theta-1) = (1 + 2 theta + q)/8      phi(theta-2) = (1 + 2 theta - q)/8
// evaluated here with q - 1 = 4 theta (1-theta) / (1 + q) so that the two
// weights that vanish at the support edge carry no cancellation error.
// Derivatives d phi/dr at the same r, with g = (2 - 4 theta)/q:
//   (-2 - g)/8, (-2 + g)/8, (2 + g)/8, (2 - g)/8.
// ---------------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ void delta_weights(Real th, Real w[4]) {
  Real om = Real(1) - th;
  Real p = Real(4) * th * om;
  Real q = sqrt(Real(1) + p);
  Real qm1 = p / (Real(1) + q);
  w[0] = (Real(2) * om - qm1) * Real(0.125);
  w[1] = (Real(2) * om + Real(2) + qm1) * Real(0.125);
  w[2] = (Real(2) * th + Real(2) + qm1) * Real(0.125);
  w[3] = (Real(2) * th - qm1) * Real(0.125);
}

template <typename Real>
__device__ __forceinline__ void delta_weights_d(Real th, Real w[4], Real dw[4]) {
  Real om = Real(1) - th;
  Real p = Real(4) * th * om;
  Real q = sqrt(Real(1) + p);
  Real qm1 = p / (Real(1) + q);
  w[0] = (Real(2) * om - qm1) * Real(0.125);
  w[1] = (Real(2) * om + Real(2) + qm1) * Real(0.125);
  w[2] = (Real(2) * th + Real(2) + qm1) * Real(0.125);
  w[3] = (Real(2) * th - qm1) * Real(0.125);
  Real g = (Real(2) - Real(4) * th) / q;
  dw[0] = (Real(-2) - g) * Real(0.125);
  dw[1] = (Real(-2) + g) * Real(0.125);
  dw[2] = (Real(2) + g) * Real(0.125);
  dw[3] = (Real(2) - g) * Real(0.125);
}

// Stencil start and fraction along one axis for a point with in-cell offset
// `off` in [0,1) and staggering s (0 or 1/2): t = cell + off - s,
// floor(t) = cell + (off < s ? -1 : 0); the first face is floor(t) - 1.
template <typename Real>
__device__ __forceinline__ int stencil_axis(Real off, bool half, Real& theta) {
  if (!half) {
    theta = off;
    return -1;
  }
  if (off < Real(0.5)) {
    theta = off + Real(0.5);
    return -2;
  }
  theta = off - Real(0.5);
  return -1;
}

__device__ __forceinline__ int wrap_idx(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

__device__ __forceinline__ int32_t pack_cell(int x, int y, int z) {
  return x | (y << kPackBits) | (z << (2 * kPackBits));
}
__device__ __forceinline__ void unpack_cell(int32_t p, int& x, int& y, int& z) {
  x = p & ((1 << kPackBits) - 1);
  y = (p >> kPackBits) & ((1 << kPackBits) - 1);
  z = (p >> (2 * kPackBits)) & ((1 << kPackBits) - 1);
}

// Grid of the structure that owns a tile (or an element): its sizes, tiles
// per dimension, first tile and instance number.  kPacked false: a plan of
// one structure, its own grid, 0 and 0 (compile-time; nothing is loaded);
// true: the packed batch's InstDev row of table[idx].
struct TileGeo {
  int n[3];
  int nt[3];
  int base;
  int inst;
};
template <bool kPacked>
__device__ __forceinline__ TileGeo tile_geo(const GridDev& g, const InstDev* inst,
                                            const int32_t* table, int idx) {
  TileGeo t;
  if constexpr (kPacked) {
    const int i = __ldg(table + idx);
    const InstDev* r = inst + i;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      t.n[d] = __ldg(&r->n[d]);
      t.nt[d] = __ldg(&r->nt[d]);
    }
    t.base = __ldg(&r->tile_base);
    t.inst = i;
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      t.n[d] = g.n[d];
      t.nt[d] = g.nt[d];
    }
    t.base = 0;
    t.inst = 0;
  }
  return t;
}
// tile coordinates of a tile within its structure's grid
__device__ __forceinline__ void tile_coords(const TileGeo& t, int tile, int& tx, int& ty,
                                            int& tz) {
  const int l = tile - t.base;
  tx = l % t.nt[0];
  ty = (l / t.nt[0]) % t.nt[1];
  tz = l / (t.nt[0] * t.nt[1]);
}

// Node position as (integer cell, offset in cell units).  FP32 split plans
// read the stored pair; FP64 plans derive it from the absolute coordinate.
template <typename Real>
struct NodeLoader;

template <>
struct NodeLoader<float> {
  const int32_t* cell;
  const float* off;
  int64_t N;
  __device__ __forceinline__ void load(int node, int c[3], float o[3]) const {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      c[d] = __ldg(cell + d * N + node);
      o[d] = __ldg(off + d * N + node);
    }
  }
};

template <>
struct NodeLoader<double> {
  const double* x64;
  int64_t N;
  double origin[3];
  double inv_h;
  __device__ __forceinline__ void load(int node, int c[3], double o[3]) const {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double t = (__ldg(x64 + d * N + node) - origin[d]) * inv_h;
      double f = floor(t);
      c[d] = (int)f;
      o[d] = t - f;
    }
  }
};

__device__ __forceinline__ void set_status(int* st, int bit) { atomicOr(st, bit); }

// Exclusive prefix sum of one int per thread across the block (blockDim.x a
// multiple of 32, at most 1024).  `tmp` is 32 ints of shared memory; `total`
// receives the block sum.  Contains barriers: call from every thread.
__device__ __forceinline__ int block_exclusive_scan(int v, int* tmp, int& total) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(full, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) tmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < nw ? tmp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(full, w, o);
      if (lane >= o) w += y;
    }
    tmp[lane] = w;
  }
  __syncthreads();
  total = tmp[nw - 1];
  const int pre = (warp > 0 ? tmp[warp - 1] : 0) + x - v;
  __syncthreads();
  return pre;
}

}  // namespace ibfe
