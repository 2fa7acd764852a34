// Interpolation of a MAC field at the Gauss points (Section 4.4):
//   U^IB_q^c = sum_faces u^c(face) prod_d phi(r_d)      (h^3 delta_h = prod phi)
// and the position derivatives of the same sums, used by the adjoints:
//   d/dchi_d sum_faces u^c prod phi = h^-1 sum_faces u^c phi'(r_d) prod_{d'!=d} phi(r_d').
// One thread per Gauss point, visiting points in tile-sorted order so that the
// 4x4x4 stencils of neighbouring threads overlap in cache; each result is
// written at the point's original index gq = q*E + e for the element-wise
// projection that follows.
//
// Modes
//   0: a[c][gq] = w j0 * vscale * S_c                      (S_c = sum u^c prod phi)
//   1: a as mode 0, and b[d][gq] = gscale * sum_c val_c dS_c/dr_d
//   2: b only.
#include "ib_device.cuh"

namespace ibfe {
namespace {

template <typename Real>
struct InterpArgs {
  GridDev g;
  int64_t Q;
  const int32_t* p_cell;
  const Real* p_off;
  const Real* p_val;
  const int32_t* p_idx;
  const Real* wj0;
  const Real* u;
  Real vscale, gscale;
  Real* out_a;
  Real* out_b;
};

__device__ __forceinline__ int wrap_near(int i, int n) {
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

template <typename Real, int MODE>
__global__ void __launch_bounds__(128) k_interp(InterpArgs<Real> A) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.Q) return;
  const int n0 = A.g.n[0], n1 = A.g.n[1], n2 = A.g.n[2];
  const int64_t cells = (int64_t)n0 * n1 * n2;
  int cx, cy, cz;
  unpack_cell(__ldg(A.p_cell + i), cx, cy, cz);
  const Real off[3] = {__ldg(A.p_off + i), __ldg(A.p_off + A.Q + i), __ldg(A.p_off + 2 * A.Q + i)};
  const int cc[3] = {cx, cy, cz};
  const int nn[3] = {n0, n1, n2};
  const int gq = __ldg(A.p_idx + i);
  Real val[3] = {Real(0), Real(0), Real(0)};
  if (MODE != 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) val[c] = __ldg(A.p_val + c * A.Q + i);
  }
  Real S[3];
  Real grad[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Real w[3][4], dw[3][4];
    int idx[3][4];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      Real th;
      const int s = stencil_axis(off[d], d != c, th);
      if (MODE == 0)
        delta_weights(th, w[d]);
      else
        delta_weights_d(th, w[d], dw[d]);
#pragma unroll
      for (int j = 0; j < 4; ++j) idx[d][j] = wrap_near(cc[d] + s + j, nn[d]);
    }
    const Real* uc = A.u + c * cells;
    Real tot = Real(0), gx = Real(0), gy = Real(0), gz = Real(0);
#pragma unroll
    for (int kz = 0; kz < 4; ++kz) {
      Real py = Real(0), pdy = Real(0), pdx = Real(0);
#pragma unroll
      for (int ky = 0; ky < 4; ++ky) {
        const Real* row = uc + ((int64_t)idx[2][kz] * n1 + idx[1][ky]) * n0;
        Real rx = Real(0), rdx = Real(0);
#pragma unroll
        for (int kx = 0; kx < 4; ++kx) {
          const Real v = __ldg(row + idx[0][kx]);
          rx += w[0][kx] * v;
          if (MODE != 0) rdx += dw[0][kx] * v;
        }
        py += w[1][ky] * rx;
        if (MODE != 0) {
          pdy += dw[1][ky] * rx;
          pdx += w[1][ky] * rdx;
        }
      }
      tot += w[2][kz] * py;
      if (MODE != 0) {
        gz += dw[2][kz] * py;
        gy += w[2][kz] * pdy;
        gx += w[2][kz] * pdx;
      }
    }
    S[c] = tot;
    if (MODE != 0) {
      grad[0] += val[c] * gx;
      grad[1] += val[c] * gy;
      grad[2] += val[c] * gz;
    }
  }
  if (MODE != 2) {
    const Real wq = __ldg(A.wj0 + gq) * A.vscale;
#pragma unroll
    for (int c = 0; c < 3; ++c) A.out_a[c * A.Q + gq] = wq * S[c];
  }
  if (MODE != 0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) A.out_b[d * A.Q + gq] = A.gscale * grad[d];
  }
}

template <typename Real>
ib_status interp_t(ib_plan* p, const void* u, int mode, double vscale, double gscale,
                   cudaStream_t s) {
  if (p->Q == 0) return IB_OK;
  InterpArgs<Real> A;
  A.g = p->grid;
  A.Q = p->Q;
  A.p_cell = p->p_cell;
  A.p_off = (const Real*)p->p_off;
  A.p_val = (const Real*)p->p_val;
  A.p_idx = p->p_idx;
  A.wj0 = (const Real*)p->wj0;
  A.u = (const Real*)u;
  A.vscale = (Real)vscale;
  A.gscale = (Real)gscale;
  A.out_a = (Real*)p->gq_a;
  A.out_b = (Real*)p->gq_b;
  const int threads = 128;
  const int blocks = (int)((p->Q + threads - 1) / threads);
  if (mode == 0)
    k_interp<Real, 0><<<blocks, threads, 0, s>>>(A);
  else if (mode == 1)
    k_interp<Real, 1><<<blocks, threads, 0, s>>>(A);
  else
    k_interp<Real, 2><<<blocks, threads, 0, s>>>(A);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

}  // namespace

ib_status launch_interp_points(ib_plan* p, const void* u, int mode, double vscale,
                               double gscale, cudaStream_t s) {
  return p->precision == IB_FP64 ? interp_t<double>(p, u, mode, vscale, gscale, s)
                                 : interp_t<float>(p, u, mode, vscale, gscale, s);
}

}  // namespace ibfe
