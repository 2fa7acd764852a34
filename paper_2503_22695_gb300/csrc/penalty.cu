// Penalty tethers of the solid boundary (Section 5: the fixed face of Cook's
// membrane, kappa = 1e6; the fixed outer tube of the aortic valve,
// kappa = 5e6).  Each tethered node a is pulled towards its reference
// position by
//   G_a -= kappa w_a (x_a - X_a),   energy kappa/2 sum_a w_a |x_a - X_a|^2,
// with w_a the node's lumped mass (its volume weight, the nodal-rule weight of
// Section 4.4) unless the caller gives weights (an area weight for a face,
// say).  The force is linear in x, so its Jacobian is -kappa w_a I on the
// tethered nodes and the adjoint adds -kappa w_a v_a.  x_a - X_a is formed in
// double from the split position (origin + (cell + off) h - X), exact to
// double rounding however small the displacement.
#include <cmath>

#include "ib_device.cuh"

namespace ibfe {
namespace {

constexpr int kPenCTAs = 64;  // blocks of the fixed-shape energy reduction

template <typename Real>
struct PenArgs {
  const int32_t* nodes;
  int n;
  const Real* w;       // [n] or null: lumped mass
  const Real* mass;    // [N]
  const Real* X;       // [3][N]
  int64_t N;
  // positions: split (cell, off) or x64
  const int32_t* cell;
  const float* off;
  const double* x64;
  double origin[3], h;
  double kappa;
};

template <typename Real>
__device__ __forceinline__ double pen_disp(const PenArgs<Real>& A, int a, int d) {
  const double X = double(A.X[d * A.N + a]);
  if (A.x64) return A.x64[d * A.N + a] - X;
  return (A.origin[d] + (double(A.cell[d * A.N + a]) + double(A.off[d * A.N + a])) * A.h) - X;
}

template <typename Real>
__device__ __forceinline__ double pen_weight(const PenArgs<Real>& A, int t, int a) {
  return double(A.w ? A.w[t] : A.mass[a]);
}

__device__ __forceinline__ double block_sum_pen(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;
}

// G_a -= kappa w (x_a - X_a) for the tethered nodes (distinct); with epart,
// CTA b also writes the energy of its chunk of the node list to epart[b].
template <typename Real>
__global__ void __launch_bounds__(256) k_penalty(PenArgs<Real> A, Real* __restrict__ G,
                                                 double* __restrict__ epart) {
  __shared__ double sh[32];
  const int chunk = (A.n + gridDim.x - 1) / gridDim.x;
  const int t0 = blockIdx.x * chunk, t1 = min(A.n, t0 + chunk);
  double e = 0.0;
  for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
    const int a = A.nodes[t];
    if (a < 0 || a >= A.N) continue;
    const double kw = A.kappa * pen_weight(A, t, a);
    double dd = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double u = pen_disp(A, a, d);
      G[d * A.N + a] -= Real(kw * u);
      dd += u * u;
    }
    e += 0.5 * kw * dd;
  }
  if (epart) {
    e = block_sum_pen(e, sh);
    if (threadIdx.x == 0) epart[blockIdx.x] = e;
  }
}

// Hv_a -= kappa w v_a (the tethers' share of the force adjoint)
template <typename Real>
__global__ void __launch_bounds__(256) k_penalty_adj(PenArgs<Real> A, const Real* __restrict__ v,
                                                     Real* __restrict__ Hv, Real mul) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.n) return;
  const int a = A.nodes[t];
  if (a < 0 || a >= A.N) return;
  const Real kw = Real(A.kappa * pen_weight(A, t, a)) * mul;
#pragma unroll
  for (int d = 0; d < 3; ++d) Hv[d * A.N + a] -= kw * v[d * A.N + a];
}

__global__ void __launch_bounds__(64) k_penalty_sum(const double* __restrict__ epart,
                                                    double* __restrict__ out) {
  __shared__ double sh[32];
  const double e = block_sum_pen(threadIdx.x < kPenCTAs ? epart[threadIdx.x] : 0.0, sh);
  if (threadIdx.x == 0) *out = e;
}

template <typename Real>
PenArgs<Real> pen_args(const ib_plan* p, const ib_pos* x) {
  PenArgs<Real> A;
  A.nodes = p->pen_nodes;
  A.n = p->pen_n;
  A.w = (const Real*)p->pen_w;
  A.mass = (const Real*)p->mass;
  A.X = (const Real*)p->X;
  A.N = p->N;
  A.cell = x->cell;
  A.off = x->off;
  A.x64 = p->precision == IB_FP64 ? x->x64 : nullptr;
  for (int d = 0; d < 3; ++d) A.origin[d] = p->grid.origin[d];
  A.h = p->grid.h;
  A.kappa = p->pen_kappa;
  return A;
}

}  // namespace

bool penalty_on(const ib_plan* p) { return p->pen_n > 0 && p->pen_kappa != 0.0; }

ib_status launch_penalty(ib_plan* p, const ib_pos* x, void* G, bool energy, cudaStream_t s) {
  if (!penalty_on(p)) return IB_OK;
  double* ep = energy ? p->pen_part : nullptr;
  if (p->precision == IB_FP64)
    k_penalty<double><<<kPenCTAs, 256, 0, s>>>(pen_args<double>(p, x), (double*)G, ep);
  else
    k_penalty<float><<<kPenCTAs, 256, 0, s>>>(pen_args<float>(p, x), (float*)G, ep);
  if (energy) k_penalty_sum<<<1, 64, 0, s>>>(p->pen_part, p->pen_part + kPenCTAs);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

const double* penalty_energy_dev(const ib_plan* p) { return p->pen_part + kPenCTAs; }

ib_status launch_penalty_adj(ib_plan* p, const void* v, void* Hv, cudaStream_t s, double mul) {
  if (!penalty_on(p)) return IB_OK;
  const int g = (p->pen_n + 255) / 256;
  ib_pos none{nullptr, nullptr, nullptr, 0.0};
  if (p->precision == IB_FP64)
    k_penalty_adj<double><<<g, 256, 0, s>>>(pen_args<double>(p, &none), (const double*)v,
                                            (double*)Hv, mul);
  else
    k_penalty_adj<float><<<g, 256, 0, s>>>(pen_args<float>(p, &none), (const float*)v,
                                           (float*)Hv, (float)mul);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

size_t penalty_scratch_doubles() { return kPenCTAs + 1; }

}  // namespace ibfe

extern "C" ib_status ib_plan_set_penalty(ib_plan* p, const int32_t* nodes, int32_t n,
                                         const void* weights, double kappa) {
  if (!p || n < 0 || (n > 0 && !nodes) || !std::isfinite(kappa) || kappa < 0.0)
    return IB_ERR_INVALID_ARG;
  if (n > p->N) return IB_ERR_INVALID_ARG;
  p->pen_nodes = n > 0 ? nodes : nullptr;
  p->pen_n = n;
  p->pen_w = n > 0 ? weights : nullptr;
  p->pen_kappa = kappa;
  return IB_OK;
}
