// Deterministic element<->node transfers and the plan's static geometry.
//
// No sparse matrix is formed (the paper's design rule, abstract): nodal sums
// are gathers over a static node -> (element, corner) incidence list, visited
// in a fixed order (ascending element, then corner), so every nodal value is
// summed in the same order on every call and no floating-point atomics occur.
#include "ib_device.cuh"

namespace ibfe {
namespace {

constexpr int kIncShift = 28;  // incidence entry: corner << 28 | element (as uint32)

// out[c][n] = add[c][n] + scale[n] * sum_{(a,e) in inc(n)} elem[(a*ncomp + c)*E + e]
// (add and scale optional; add may be out itself)
template <typename Real, int NC>
__global__ void __launch_bounds__(256) k_node_gather(const int32_t* __restrict__ inc_off,
                                                     const int32_t* __restrict__ inc_idx,
                                                     const Real* __restrict__ elem,
                                                     const Real* __restrict__ scale,
                                                     const Real* add, int N, int E, Real* out,
                                                     Real mul) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  Real acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = Real(0);
  const int b = __ldg(inc_off + n), en = __ldg(inc_off + n + 1);
  for (int k = b; k < en; ++k) {
    // unsigned: corners 8 and 9 of a P2 element set the top bit
    const uint32_t v = static_cast<uint32_t>(__ldg(inc_idx + k));
    const int a = (int)(v >> kIncShift), e = (int)(v & ((1u << kIncShift) - 1u));
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] += __ldg(elem + (int64_t)(a * NC + c) * E + e);
  }
  const Real s = (scale ? __ldg(scale + n) : Real(1)) * mul;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int64_t o = (int64_t)c * N + n;
    out[o] = add ? add[o] + acc[c] * s : acc[c] * s;
  }
}

// out[(a*NC + c)*E + e] = sum_q N_a(xi_q) w[q*E + e] vals[c][q*E + e]
// (w: the points' weights w_q j0, or null for 1)
template <typename Real, int NC, int kEl>
__global__ void __launch_bounds__(256) k_elem_project(const Real* __restrict__ vals,
                                                      const Real* __restrict__ w, int E,
                                                      Real* __restrict__ out) {
  using EL = El<kEl>;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int64_t Q = (int64_t)EL::Q * E;
  Real wq[EL::Q];
#pragma unroll
  for (int q = 0; q < EL::Q; ++q) wq[q] = w ? __ldg(w + (int64_t)q * E + e) : Real(1);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    Real v[EL::Q];
#pragma unroll
    for (int q = 0; q < EL::Q; ++q) v[q] = __ldg(vals + c * Q + (int64_t)q * E + e) * wq[q];
#pragma unroll
    for (int a = 0; a < EL::C; ++a) {
      Real s = Real(0);
#pragma unroll
      for (int q = 0; q < EL::Q; ++q) s += Real(EL::N(a, q)) * v[q];
      out[(int64_t)(a * NC + c) * E + e] = s;
    }
  }
}

// out[i] = add[i] + src[i] (add optional, may alias out)
template <typename Real>
__global__ void k_node_copy(const Real* __restrict__ src, const Real* add, int64_t n, Real* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = add ? add[i] + src[i] : src[i];
}

// w_q j0 at the coupling points of each element (the element rule's weight
// times det dX/dxi; for the tetrahedron the Jacobian is constant).
template <typename Real, int kEl>
__global__ void __launch_bounds__(128) k_wj0(const int32_t* __restrict__ conn,
                                             const Real* __restrict__ X, int E, int64_t N,
                                             Real* __restrict__ wj0, int* status) {
  using EL = El<kEl>;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  Real dX[EL::C][3];
  const int n0 = __ldg(conn + e);
  for (int a = 0; a < EL::C; ++a) {
    const int n = __ldg(conn + a * E + e);
    for (int d = 0; d < 3; ++d) dX[a][d] = __ldg(X + d * N + n) - __ldg(X + d * N + n0);
  }
  bool bad = false;
#pragma unroll
  for (int q = 0; q < EL::Q; ++q) {
    Real J0[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Real s = Real(0);
#pragma unroll
        for (int a = 1; a < EL::C; ++a) s += dX[a][i] * Real(EL::dxi(a, q, j));
        J0[i][j] = s;
      }
    const Real det = J0[0][0] * (J0[1][1] * J0[2][2] - J0[1][2] * J0[2][1]) +
                     J0[0][1] * (J0[1][2] * J0[2][0] - J0[1][0] * J0[2][2]) +
                     J0[0][2] * (J0[1][0] * J0[2][1] - J0[1][1] * J0[2][0]);
    if (!(det > Real(0))) bad = true;
    wj0[(int64_t)q * E + e] = Real(EL::wQ) * det;
  }
  if (bad) set_status(status, kStatInverted);
}

// Per-element lumped mass in double from the weights w_q j0 (Real): for
// hexahedra and P1 the row sums sum_q N_a(xi_q) w_q j0; for P2 the diagonal
// d_a = sum_q N_a(xi_q)^2 w_q j0 scaled by V / sum_b d_b, V = sum_q w_q j0
// (every mass positive, the element's masses summing to its volume).  The
// node gather then sums in double, so the rounded FP32 mass is, in
// practice, independent of the order in which the elements are listed (the
// point values carried by spreading divide by it).
template <typename Real, int kEl>
__global__ void __launch_bounds__(256) k_mass_corner_d(const Real* __restrict__ wj0, int E,
                                                       double* __restrict__ out) {
  using EL = El<kEl>;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double w[EL::Q], d[EL::C], V = 0.0, D = 0.0;
#pragma unroll
  for (int q = 0; q < EL::Q; ++q) {
    w[q] = double(__ldg(wj0 + (int64_t)q * E + e));
    V += w[q];
  }
#pragma unroll
  for (int a = 0; a < EL::C; ++a) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < EL::Q; ++q)
      s += (EL::kScaledMass ? EL::N(a, q) * EL::N(a, q) : EL::N(a, q)) * w[q];
    d[a] = s;
    D += s;
  }
#pragma unroll
  for (int a = 0; a < EL::C; ++a) out[(int64_t)a * E + e] = EL::kScaledMass ? d[a] * (V / D) : d[a];
}

__global__ void k_mass_round(const double* __restrict__ md, float* __restrict__ m,
                             float* __restrict__ im, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  m[n] = float(md[n]);
  // nodes that belong to no element carry no mass and receive zero
  im[n] = md[n] > 0.0 ? float(1.0 / md[n]) : 0.f;
}

template <typename Real>
__global__ void k_invert(const Real* __restrict__ m, Real* __restrict__ im, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  // nodes that belong to no element carry no mass and receive zero
  if (n < N) im[n] = m[n] > Real(0) ? Real(1) / m[n] : Real(0);
}

template <typename Real>
ib_status gather_t(ib_plan* p, const void* elem, const void* scale, const void* add, void* out,
                   int nc, cudaStream_t s, double mul = 1.0) {
  if (p->N == 0) return IB_OK;
  const int blocks = (p->N + 255) / 256;
  if (nc == 3)
    k_node_gather<Real, 3><<<blocks, 256, 0, s>>>(p->inc_off, p->inc_idx, (const Real*)elem,
                                                  (const Real*)scale, (const Real*)add, p->N,
                                                  p->E, (Real*)out, (Real)mul);
  else
    k_node_gather<Real, 1><<<blocks, 256, 0, s>>>(p->inc_off, p->inc_idx, (const Real*)elem,
                                                  (const Real*)scale, (const Real*)add, p->N,
                                                  p->E, (Real*)out, (Real)mul);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

template <typename Real>
ib_status project_t(ib_plan* p, const void* vals, const void* w, void* out, int nc,
                    cudaStream_t s) {
  if (p->E == 0) return IB_OK;
  const int blocks = (p->E + 255) / 256;
  with_elem(p->elem, [&](auto el) {
    constexpr int kE = decltype(el)::value;
    if (nc == 3)
      k_elem_project<Real, 3, kE><<<blocks, 256, 0, s>>>((const Real*)vals, (const Real*)w,
                                                         p->E, (Real*)out);
    else
      k_elem_project<Real, 1, kE><<<blocks, 256, 0, s>>>((const Real*)vals, (const Real*)w,
                                                         p->E, (Real*)out);
  });
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

template <typename Real>
ib_status static_t(ib_plan* p, cudaStream_t s) {
  if (p->E > 0) {
    with_elem(p->elem, [&](auto el) {
      constexpr int kE = decltype(el)::value;
      k_wj0<Real, kE><<<(p->E + 127) / 128, 128, 0, s>>>(p->conn, (const Real*)p->X, p->E, p->N,
                                                       (Real*)p->wj0, p->dstatus);
    });
    if (cudaGetLastError() != cudaSuccess) return IB_ERR_CUDA;
  }
  // m_a = sum over the elements containing a of the element's lumped mass
  if (sizeof(Real) == 4 || p->elem == IB_ELEM_TET10) {  // accumulated in double
    double *ed = nullptr, *md = nullptr;
    if (cudaMalloc(&ed, sizeof(double) * p->nc * (size_t)(p->E > 0 ? p->E : 1)) != cudaSuccess ||
        cudaMalloc(&md, sizeof(double) * (size_t)p->N) != cudaSuccess) {
      cudaFree(ed);
      return IB_ERR_CUDA;
    }
    if (p->E > 0)
      with_elem(p->elem, [&](auto el) {
        constexpr int kE = decltype(el)::value;
        k_mass_corner_d<Real, kE><<<(p->E + 255) / 256, 256, 0, s>>>((const Real*)p->wj0, p->E,
                                                                     ed);
      });
    k_node_gather<double, 1><<<(p->N + 255) / 256, 256, 0, s>>>(
        p->inc_off, p->inc_idx, ed, nullptr, nullptr, p->N, p->E, md, 1.0);
    if (sizeof(Real) == 4)
      k_mass_round<<<(p->N + 255) / 256, 256, 0, s>>>(md, (float*)p->mass, (float*)p->inv_mass,
                                                      p->N);
    else if (p->N > 0) {
      cudaMemcpyAsync(p->mass, md, sizeof(double) * p->N, cudaMemcpyDeviceToDevice, s);
      k_invert<double><<<(p->N + 255) / 256, 256, 0, s>>>(md, (double*)p->inv_mass, p->N);
    }
    const bool good = cudaStreamSynchronize(s) == cudaSuccess;
    cudaFree(ed);
    cudaFree(md);
    return good && cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
  }
  ib_status st = project_t<Real>(p, p->wj0, nullptr, p->elem_scratch, 1, s);
  if (st != IB_OK) return st;
  st = gather_t<Real>(p, p->elem_scratch, nullptr, nullptr, p->mass, 1, s);
  if (st != IB_OK) return st;
  if (p->N > 0)
    k_invert<Real><<<(p->N + 255) / 256, 256, 0, s>>>((const Real*)p->mass, (Real*)p->inv_mass,
                                                      p->N);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

}  // namespace

ib_status launch_node_gather(ib_plan* p, const void* elem, const void* scale, void* out,
                             cudaStream_t s, const void* add, double mul) {
  return p->precision == IB_FP64 ? gather_t<double>(p, elem, scale, add, out, 3, s, mul)
                                 : gather_t<float>(p, elem, scale, add, out, 3, s, mul);
}

ib_status launch_node_copy(ib_plan* p, const void* src, void* out, const void* add,
                           cudaStream_t s) {
  const int64_t n = 3LL * p->N;
  if (n == 0) return IB_OK;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (p->precision == IB_FP64)
    k_node_copy<double><<<blocks, 256, 0, s>>>((const double*)src, (const double*)add, n,
                                               (double*)out);
  else
    k_node_copy<float><<<blocks, 256, 0, s>>>((const float*)src, (const float*)add, n,
                                              (float*)out);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

ib_status launch_elem_project(ib_plan* p, const void* vals, bool weighted, void* out,
                              cudaStream_t s) {
  const void* w = weighted ? p->wj0 : nullptr;
  return p->precision == IB_FP64 ? project_t<double>(p, vals, w, out, 3, s)
                                 : project_t<float>(p, vals, w, out, 3, s);
}

ib_status launch_plan_static(ib_plan* p, cudaStream_t s) {
  return p->precision == IB_FP64 ? static_t<double>(p, s) : static_t<float>(p, s);
}

}  // namespace ibfe
