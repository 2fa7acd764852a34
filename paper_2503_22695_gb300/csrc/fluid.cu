// Fluid step of the explicit IB scheme (Section 4.2): Chorin's projection on
// the periodic MAC grid,
//   rho/dt (u* - u^n) - mu Lap_h u* = f          (Helmholtz, per component)
//   Lap_h p = div_h u* / dt                       (Poisson, cell centres)
//   u^{n+1} = u* - dt grad_h p                    (correction)
// with a geometric multigrid for both solves (the paper accelerates its
// solvers with geometric multigrid).
//
// Layout: fields [3][n2][n1][n0] as in the coupling operators (component c on
// the lower c-faces), p [n2][n1][n0] at cell centres, so that
//   (div u)(i) = sum_c (u^c(i + e_c) - u^c(i)) / h,
//   (grad p)^c(i) = (p(i) - p(i - e_c)) / h,   div grad = Lap_h (7 points).
// In the periodic box every component lives on a translated copy of the same
// n0 x n1 x n2 lattice with the same operator, so one scalar multigrid for
// A = alpha - beta Lap_h serves the three velocity components (solved
// together, one launch per kernel) and the pressure (alpha = 0, whose
// constant mode is fixed by a zero mean).
//
// Multigrid: V-cycles over levels that halve every dimension while all are
// even and the largest exceeds 16 (rediscretised operator, h doubled per
// level); red-black Gauss-Seidel smoothing; the residual and its restriction
// (mean of the 8 children) in one kernel, which also zeroes the coarse
// correction; trilinear (cell-centred) prolongation added to the fine
// iterate; on the coarsest level one CTA per component solves in shared
// memory with a fixed number of red-black sweeps (weighted Jacobi when a
// dimension is odd).  Every reduction has a fixed shape, so results are
// bitwise reproducible; the cycle counts are fixed (no host round trip), so
// a step can be captured in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ib_device.cuh"

struct ib_fluid {
  int precision;
  size_t rsize;
  int n[3];
  double h, rho, mu, dt;
  static constexpr int kMaxLevels = 16;
  int nlev;
  int ln[kMaxLevels][3];   // lattice of each level
  void* lphi[kMaxLevels];  // levels >= 1: correction [3][cells]
  void* lrhs[kMaxLevels];  // levels >= 1: right-hand side [3][cells]
  int cyc_h, cyc_p, pre, post, coarse_sweeps;
  void* rhs0;              // [3][cells] Helmholtz right-hand side
  void* div;               // [cells] Poisson right-hand side
  void* ptmp;              // [cells] pressure when the caller passes none
  double* red;             // reduction partials
  int sm_count;
  size_t coarse_smem;
};

namespace ibfe {
namespace {

constexpr int kFluidRedCTAs = 256;   // first-level reduction CTAs
constexpr int kCoarseMax = 16;       // coarsest level: every dimension <= 16 (or odd)
constexpr int kCoarseCells = 8192;   // shared-memory limit of the coarsest solve

bool ok(cudaError_t e) { return e == cudaSuccess; }

__device__ __forceinline__ int wrap_up(int i, int n) { return i + 1 == n ? 0 : i + 1; }
__device__ __forceinline__ int wrap_dn(int i, int n) { return i == 0 ? n - 1 : i - 1; }

// sum of the six lattice neighbours of (i, j, k) (periodic)
template <typename Real>
__device__ __forceinline__ Real nb_sum(const Real* __restrict__ f, int i, int j, int k, int n0,
                                       int n1, int n2) {
  const int64_t row = ((int64_t)k * n1 + j) * n0;
  const Real sx = f[row + wrap_up(i, n0)] + f[row + wrap_dn(i, n0)];
  const Real sy = f[((int64_t)k * n1 + wrap_up(j, n1)) * n0 + i] +
                  f[((int64_t)k * n1 + wrap_dn(j, n1)) * n0 + i];
  const Real sz = f[((int64_t)wrap_up(k, n2) * n1 + j) * n0 + i] +
                  f[((int64_t)wrap_dn(k, n2) * n1 + j) * n0 + i];
  return sx + sy + sz;
}

// One colour of a red-black Gauss-Seidel sweep for (alpha - beta Lap) phi = rhs
// on ncomp stacked lattices: cells with (i + j + k) even (colour 0) or odd.
// phi_i = (rhs_i + b sum_nb phi) / (alpha + 6 b), b = beta / h^2.  n0 even.
template <typename Real>
__global__ void __launch_bounds__(256) k_rb_smooth(Real* __restrict__ phi,
                                                   const Real* __restrict__ rhs, int n0, int n1,
                                                   int n2, int ncomp, Real b, Real dinv,
                                                   int color) {
  const int h0 = n0 >> 1;
  const int64_t cells = (int64_t)n0 * n1 * n2;
  const int64_t per = (int64_t)h0 * n1 * n2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < per * ncomp;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / per);
    const int64_t r = t - c * per;
    const int m = (int)(r % h0);
    const int64_t jk = r / h0;
    const int j = (int)(jk % n1), k = (int)(jk / n1);
    const int i = 2 * m + ((j + k + color) & 1);
    Real* f = phi + c * cells;
    const int64_t idx = ((int64_t)k * n1 + j) * n0 + i;
    f[idx] = (rhs[c * cells + idx] + b * nb_sum(f, i, j, k, n0, n1, n2)) * dinv;
  }
}

// Residual rhs - A phi of the 8 children of each coarse cell, averaged into
// the coarse right-hand side; the coarse correction is zeroed.
template <typename Real>
__global__ void __launch_bounds__(256) k_restrict(const Real* __restrict__ phi,
                                                  const Real* __restrict__ rhs,
                                                  Real* __restrict__ rc, Real* __restrict__ pc,
                                                  int n0, int n1, int n2, int ncomp, Real b,
                                                  Real diag) {
  const int m0 = n0 >> 1, m1 = n1 >> 1, m2 = n2 >> 1;
  const int64_t cells = (int64_t)n0 * n1 * n2, ccells = (int64_t)m0 * m1 * m2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ccells * ncomp;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / ccells);
    const int64_t r = t - c * ccells;
    const int I = (int)(r % m0);
    const int64_t JK = r / m0;
    const int J = (int)(JK % m1), K = (int)(JK / m1);
    const Real* f = phi + c * cells;
    const Real* g = rhs + c * cells;
    Real s = Real(0);
#pragma unroll
    for (int dk = 0; dk < 2; ++dk)
#pragma unroll
      for (int dj = 0; dj < 2; ++dj)
#pragma unroll
        for (int di = 0; di < 2; ++di) {
          const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
          const int64_t idx = ((int64_t)k * n1 + j) * n0 + i;
          s += g[idx] - diag * f[idx] + b * nb_sum(f, i, j, k, n0, n1, n2);
        }
    rc[t] = s * Real(0.125);
    pc[t] = Real(0);
  }
}

// phi_fine += trilinear (cell-centred) interpolation of the coarse correction:
// per axis 3/4 of the parent and 1/4 of the parent's neighbour on the side of
// the child.
template <typename Real>
__global__ void __launch_bounds__(256) k_prolong(const Real* __restrict__ pc,
                                                 Real* __restrict__ phi, int n0, int n1, int n2,
                                                 int ncomp) {
  const int m0 = n0 >> 1, m1 = n1 >> 1, m2 = n2 >> 1;
  const int64_t cells = (int64_t)n0 * n1 * n2, ccells = (int64_t)m0 * m1 * m2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cells * ncomp;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t / cells);
    const int64_t r = t - c * cells;
    const int i = (int)(r % n0);
    const int64_t jk = r / n0;
    const int j = (int)(jk % n1), k = (int)(jk / n1);
    const int I = i >> 1, J = j >> 1, K = k >> 1;
    const int I2 = (i & 1) ? wrap_up(I, m0) : wrap_dn(I, m0);
    const int J2 = (j & 1) ? wrap_up(J, m1) : wrap_dn(J, m1);
    const int K2 = (k & 1) ? wrap_up(K, m2) : wrap_dn(K, m2);
    const Real* q = pc + c * ccells;
    auto at = [&](int a, int bb, int cc) { return q[((int64_t)cc * m1 + bb) * m0 + a]; };
    const Real w1 = Real(0.75), w2 = Real(0.25);
    const Real zK = w1 * (w1 * (w1 * at(I, J, K) + w2 * at(I2, J, K)) +
                          w2 * (w1 * at(I, J2, K) + w2 * at(I2, J2, K)));
    const Real zK2 = w1 * (w1 * at(I, J, K2) + w2 * at(I2, J, K2)) +
                     w2 * (w1 * at(I, J2, K2) + w2 * at(I2, J2, K2));
    phi[t] += zK + w2 * zK2;
  }
}

// Fixed-shape block sum in double (thread 0 holds the result).
__device__ __forceinline__ double block_sum_fl(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
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

// Coarsest level: one CTA per component solves A phi = rhs in shared memory
// from phi = 0 with `sweeps` red-black sweeps (all dimensions even) or
// weighted Jacobi sweeps (omega = 6/7); for the singular Poisson operator the
// mean is removed at the end.
template <typename Real>
__global__ void __launch_bounds__(1024) k_coarse(Real* __restrict__ phi,
                                                 const Real* __restrict__ rhs, int n0, int n1,
                                                 int n2, Real b, Real dinv, int sweeps,
                                                 int even, int singular) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double shr[32];
  const int cells = n0 * n1 * n2;
  Real* sp = reinterpret_cast<Real*>(smem_raw);
  Real* sr = sp + cells;
  Real* st = sr + cells;  // Jacobi only
  const int c = blockIdx.x;
  for (int t = threadIdx.x; t < cells; t += blockDim.x) {
    sr[t] = rhs[(int64_t)c * cells + t];
    sp[t] = Real(0);
  }
  __syncthreads();
  for (int s = 0; s < sweeps; ++s) {
    if (even) {
      for (int color = 0; color < 2; ++color) {
        const int half = cells >> 1;
        for (int t = threadIdx.x; t < half; t += blockDim.x) {
          const int m = t % (n0 >> 1), jk = t / (n0 >> 1);
          const int j = jk % n1, k = jk / n1;
          const int i = 2 * m + ((j + k + color) & 1);
          const int idx = (k * n1 + j) * n0 + i;
          sp[idx] = (sr[idx] + b * nb_sum(sp, i, j, k, n0, n1, n2)) * dinv;
        }
        __syncthreads();
      }
    } else {
      const Real w = Real(6.0 / 7.0);
      for (int t = threadIdx.x; t < cells; t += blockDim.x) {
        const int i = t % n0, jk = t / n0, j = jk % n1, k = jk / n1;
        const Real nv = (sr[t] + b * nb_sum(sp, i, j, k, n0, n1, n2)) * dinv;
        st[t] = sp[t] + w * (nv - sp[t]);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < cells; t += blockDim.x) sp[t] = st[t];
      __syncthreads();
    }
  }
  Real mean = Real(0);
  if (singular) {
    double v = 0.0;
    for (int t = threadIdx.x; t < cells; t += blockDim.x) v += double(sp[t]);
    v = block_sum_fl(v, shr);
    if (threadIdx.x == 0) shr[0] = v / cells;
    __syncthreads();
    mean = Real(shr[0]);
  }
  for (int t = threadIdx.x; t < cells; t += blockDim.x)
    phi[(int64_t)c * cells + t] = sp[t] - mean;
}

// rhs0 = rho/dt u^n + f and the initial iterate u* = u^n (u_next may alias u).
template <typename Real>
__global__ void __launch_bounds__(256) k_fluid_rhs(const Real* u, const Real* __restrict__ f,
                                                   Real* __restrict__ rhs0, Real* ustar,
                                                   int64_t n, Real a) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const Real v = u[t];
    rhs0[t] = a * v + (f ? f[t] : Real(0));
    ustar[t] = v;
  }
}

// div = (div_h u*) / dt at the cell centres (scale = 1 / (h dt)); p = 0.
template <typename Real>
__global__ void __launch_bounds__(256) k_divergence(const Real* __restrict__ u,
                                                    Real* __restrict__ div,
                                                    Real* __restrict__ p, int n0, int n1,
                                                    int n2, Real scale) {
  const int64_t cells = (int64_t)n0 * n1 * n2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cells;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % n0);
    const int64_t jk = t / n0;
    const int j = (int)(jk % n1), k = (int)(jk / n1);
    const Real dx = u[((int64_t)k * n1 + j) * n0 + wrap_up(i, n0)] - u[t];
    const Real dy = u[cells + ((int64_t)k * n1 + wrap_up(j, n1)) * n0 + i] - u[cells + t];
    const Real dz = u[2 * cells + ((int64_t)wrap_up(k, n2) * n1 + j) * n0 + i] - u[2 * cells + t];
    div[t] = (dx + dy + dz) * scale;
    p[t] = Real(0);
  }
}

// u^{n+1} = u* - dt grad_h p (in place; scale = dt / h)
template <typename Real>
__global__ void __launch_bounds__(256) k_project(Real* __restrict__ u, const Real* __restrict__ p,
                                                 int n0, int n1, int n2, Real scale) {
  const int64_t cells = (int64_t)n0 * n1 * n2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cells;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % n0);
    const int64_t jk = t / n0;
    const int j = (int)(jk % n1), k = (int)(jk / n1);
    const Real pc = p[t];
    u[t] -= scale * (pc - p[((int64_t)k * n1 + j) * n0 + wrap_dn(i, n0)]);
    u[cells + t] -= scale * (pc - p[((int64_t)k * n1 + wrap_dn(j, n1)) * n0 + i]);
    u[2 * cells + t] -= scale * (pc - p[((int64_t)wrap_dn(k, n2) * n1 + j) * n0 + i]);
  }
}

// Fixed-shape sums: CTA b sums a contiguous chunk of x (and of x^2, and of
// the squared residual of A phi = rhs when phi is given) into part[b][3].
template <typename Real>
__global__ void __launch_bounds__(256) k_sums_l1(const Real* __restrict__ x, int64_t n,
                                                 double* __restrict__ part) {
  __shared__ double sh[32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t e0 = blockIdx.x * chunk, e1 = std::min<int64_t>(n, e0 + chunk);
  double s = 0.0;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) s += double(x[e]);
  s = block_sum_fl(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

template <typename Real>
__global__ void __launch_bounds__(256) k_resid_l1(const Real* __restrict__ phi,
                                                  const Real* __restrict__ rhs, int n0, int n1,
                                                  int n2, int ncomp, Real b, Real diag,
                                                  double* __restrict__ part) {
  __shared__ double sh[32];
  const int64_t cells = (int64_t)n0 * n1 * n2, n = cells * ncomp;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t e0 = blockIdx.x * chunk, e1 = std::min<int64_t>(n, e0 + chunk);
  double rr = 0.0, bb = 0.0;
  for (int64_t t = e0 + threadIdx.x; t < e1; t += blockDim.x) {
    const int c = (int)(t / cells);
    const int64_t r = t - c * cells;
    const int i = (int)(r % n0);
    const int64_t jk = r / n0;
    const int j = (int)(jk % n1), k = (int)(jk / n1);
    const Real* f = phi + c * cells;
    const double res = double(rhs[t]) - double(diag) * double(f[r]) +
                       double(b) * double(nb_sum(f, i, j, k, n0, n1, n2));
    rr += res * res;
    bb += double(rhs[t]) * double(rhs[t]);
  }
  rr = block_sum_fl(rr, sh);
  bb = block_sum_fl(bb, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = rr;
    part[2 * blockIdx.x + 1] = bb;
  }
}

// out[k] = sum_b part[b * stride + k] for k < stride (one CTA)
__global__ void __launch_bounds__(256) k_sums_l2(const double* __restrict__ part, int nblk,
                                                 int stride, double* __restrict__ out) {
  __shared__ double sh[32];
  for (int k = 0; k < stride; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b * stride + k];
    s = block_sum_fl(s, sh);
    if (threadIdx.x == 0) out[k] = s;
    __syncthreads();
  }
}

// x -= (*sum) / n
template <typename Real>
__global__ void __launch_bounds__(256) k_sub_mean(Real* __restrict__ x, int64_t n,
                                                  const double* __restrict__ sum) {
  const Real m = Real(*sum / double(n));
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    x[t] -= m;
}

int grid_for(const ib_fluid* fl, int64_t work) {
  const int64_t want = (work + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)fl->sm_count * 8));
}

template <typename Real>
struct Fluid {
  static ib_status smooth(ib_fluid* fl, Real* phi, const Real* rhs, const int* n, int ncomp,
                          double alpha, double beta, double h, int sweeps, cudaStream_t s) {
    const double b = beta / (h * h);
    const Real dinv = Real(1.0 / (alpha + 6.0 * b));
    const int64_t work = (int64_t)(n[0] / 2) * n[1] * n[2] * ncomp;
    const int g = grid_for(fl, work);
    for (int sw = 0; sw < sweeps; ++sw)
      for (int color = 0; color < 2; ++color)
        k_rb_smooth<Real><<<g, 256, 0, s>>>(phi, rhs, n[0], n[1], n[2], ncomp, Real(b), dinv,
                                            color);
    return IB_OK;
  }

  // one V-cycle from level l (phi, rhs of that level)
  static ib_status vcycle(ib_fluid* fl, int l, Real* phi, const Real* rhs, int ncomp,
                          double alpha, double beta, bool singular, cudaStream_t s) {
    const int* n = fl->ln[l];
    const double h = fl->h * double(1 << l);
    const double b = beta / (h * h);
    if (l == fl->nlev - 1) {
      const bool even = n[0] % 2 == 0 && n[1] % 2 == 0 && n[2] % 2 == 0;
      k_coarse<Real><<<ncomp, 1024, fl->coarse_smem, s>>>(
          phi, rhs, n[0], n[1], n[2], Real(b), Real(1.0 / (alpha + 6.0 * b)),
          fl->coarse_sweeps, even ? 1 : 0, singular ? 1 : 0);
      return IB_OK;
    }
    smooth(fl, phi, rhs, n, ncomp, alpha, beta, h, fl->pre, s);
    Real* pc = (Real*)fl->lphi[l + 1];
    Real* rc = (Real*)fl->lrhs[l + 1];
    const int64_t cc = (int64_t)fl->ln[l + 1][0] * fl->ln[l + 1][1] * fl->ln[l + 1][2];
    k_restrict<Real><<<grid_for(fl, cc * ncomp), 256, 0, s>>>(
        phi, rhs, rc, pc, n[0], n[1], n[2], ncomp, Real(b), Real(alpha + 6.0 * b));
    vcycle(fl, l + 1, pc, rc, ncomp, alpha, beta, singular, s);
    const int64_t cells = (int64_t)n[0] * n[1] * n[2];
    k_prolong<Real><<<grid_for(fl, cells * ncomp), 256, 0, s>>>(pc, phi, n[0], n[1], n[2],
                                                                  ncomp);
    smooth(fl, phi, rhs, n, ncomp, alpha, beta, h, fl->post, s);
    return IB_OK;
  }

  // relative residual ||rhs - A phi|| / ||rhs|| (synchronises s)
  static double residual(ib_fluid* fl, const Real* phi, const Real* rhs, int ncomp, double alpha,
                         double beta, cudaStream_t s) {
    const int* n = fl->n;
    const double b = beta / (fl->h * fl->h);
    k_resid_l1<Real><<<kFluidRedCTAs, 256, 0, s>>>(phi, rhs, n[0], n[1], n[2], ncomp, Real(b),
                                                   Real(alpha + 6.0 * b), fl->red);
    k_sums_l2<<<1, 256, 0, s>>>(fl->red, kFluidRedCTAs, 2, fl->red + 2 * kFluidRedCTAs);
    double out[2] = {0.0, 0.0};
    if (!ok(cudaMemcpyAsync(out, fl->red + 2 * kFluidRedCTAs, sizeof(out),
                            cudaMemcpyDeviceToHost, s)) ||
        !ok(cudaStreamSynchronize(s)))
      return -1.0;
    return out[1] > 0.0 ? std::sqrt(out[0] / out[1]) : std::sqrt(out[0]);
  }

  static void sub_mean(ib_fluid* fl, Real* x, int64_t n, cudaStream_t s) {
    k_sums_l1<Real><<<kFluidRedCTAs, 256, 0, s>>>(x, n, fl->red);
    k_sums_l2<<<1, 256, 0, s>>>(fl->red, kFluidRedCTAs, 1, fl->red + 2 * kFluidRedCTAs);
    k_sub_mean<Real><<<grid_for(fl, n), 256, 0, s>>>(x, n, fl->red + 2 * kFluidRedCTAs);
  }

  static ib_status step(ib_fluid* fl, const Real* u, const Real* f, Real* un, Real* p,
                        double* residuals, cudaStream_t s) {
    const int* n = fl->n;
    const int64_t cells = (int64_t)n[0] * n[1] * n[2];
    const double a = fl->rho / fl->dt;
    Real* rhs0 = (Real*)fl->rhs0;
    Real* div = (Real*)fl->div;
    k_fluid_rhs<Real><<<grid_for(fl, 3 * cells), 256, 0, s>>>(u, f, rhs0, un, 3 * cells,
                                                               Real(a));
    for (int c = 0; c < fl->cyc_h; ++c) vcycle(fl, 0, un, rhs0, 3, a, fl->mu, false, s);
    double rh = 0.0, rp = 0.0;
    if (residuals) rh = residual(fl, un, rhs0, 3, a, fl->mu, s);
    k_divergence<Real><<<grid_for(fl, cells), 256, 0, s>>>(un, div, p, n[0], n[1], n[2],
                                                            Real(1.0 / (fl->h * fl->dt)));
    sub_mean(fl, div, cells, s);  // exact zero mean (periodic box) up to rounding
    for (int c = 0; c < fl->cyc_p; ++c) vcycle(fl, 0, p, div, 1, 0.0, -1.0, true, s);
    if (residuals) rp = residual(fl, p, div, 1, 0.0, -1.0, s);
    sub_mean(fl, p, cells, s);
    k_project<Real><<<grid_for(fl, cells), 256, 0, s>>>(un, p, n[0], n[1], n[2],
                                                         Real(fl->dt / fl->h));
    if (residuals) {
      residuals[0] = rh;
      residuals[1] = rp;
    }
    return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
  }
};

// x^{n+1} = x^n + dt U on split positions: the offset moves by dt U / h
// cells and whole cells carry into the integer part (t - floor(t) is exact
// in FP32 for |t| < 2^23, and lies in [0, 1)).
__global__ void __launch_bounds__(256) k_advance_split(int32_t* __restrict__ cell,
                                                       float* __restrict__ off,
                                                       const float* __restrict__ U, int64_t n,
                                                       float scale) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float v = off[t] + scale * U[t];
    const float fl = floorf(v);
    off[t] = v - fl;
    cell[t] += (int32_t)fl;
  }
}

__global__ void __launch_bounds__(256) k_advance_x64(double* __restrict__ x,
                                                     const double* __restrict__ U, int64_t n,
                                                     double dt) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    x[t] += dt * U[t];
}

}  // namespace

ib_status launch_advance_positions(ib_plan* p, const ib_pos* x, const void* U, double dt,
                                   cudaStream_t s) {
  const int64_t n = 3 * (int64_t)p->N;
  if (n == 0) return IB_OK;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
  if (p->precision == IB_FP64)
    k_advance_x64<<<g, 256, 0, s>>>(const_cast<double*>(x->x64), (const double*)U, n, dt);
  else
    k_advance_split<<<g, 256, 0, s>>>(const_cast<int32_t*>(x->cell), const_cast<float*>(x->off),
                                      (const float*)U, n, (float)(dt / p->grid.h));
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

// Advance the fluid one step (internal entry shared with ib_step).
ib_status fluid_step_async(ib_fluid* fl, const void* u, const void* f, void* u_next, void* p,
                           double* residuals, cudaStream_t s) {
  void* pp = p ? p : fl->ptmp;
  if (fl->precision == IB_FP64)
    return Fluid<double>::step(fl, (const double*)u, (const double*)f, (double*)u_next,
                               (double*)pp, residuals, s);
  return Fluid<float>::step(fl, (const float*)u, (const float*)f, (float*)u_next, (float*)pp,
                            residuals, s);
}

bool fluid_matches(const ib_fluid* fl, const ib_plan* p) {
  return fl && p && fl->n[0] == p->grid.n[0] && fl->n[1] == p->grid.n[1] &&
         fl->n[2] == p->grid.n[2] && fl->h == p->grid.h &&
         (fl->precision == IB_FP64) == (p->precision == IB_FP64);
}

double fluid_dt(const ib_fluid* fl) { return fl->dt; }

}  // namespace ibfe

extern "C" {

ib_status ib_fluid_create(const ib_grid* grid, int32_t precision, double rho, double mu,
                          double dt, void* stream, ib_fluid** out) {
  using namespace ibfe;
  if (!grid || !out) return IB_ERR_INVALID_ARG;
  *out = nullptr;
  if (precision != IB_FP32_SPLIT && precision != IB_FP64 && precision != IB_FP32_SPLIT_F32STAB)
    return IB_ERR_INVALID_ARG;
  if (!(grid->h > 0.0) || !std::isfinite(grid->h) || !(rho > 0.0) || !std::isfinite(rho) ||
      !(mu >= 0.0) || !std::isfinite(mu) || !(dt > 0.0) || !std::isfinite(dt))
    return IB_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d)
    if (grid->n[d] < 4 || grid->n[d] > 4096) return IB_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d)
    if (grid->n[d] % 2) return IB_ERR_UNSUPPORTED;  // red-black colouring of the periodic lattice
  ib_fluid* fl = new ib_fluid();
  std::memset(fl, 0, sizeof(*fl));
  fl->precision = precision;
  fl->rsize = precision == IB_FP64 ? 8 : 4;
  for (int d = 0; d < 3; ++d) fl->n[d] = grid->n[d];
  fl->h = grid->h;
  fl->rho = rho;
  fl->mu = mu;
  fl->dt = dt;
  fl->cyc_h = 2;
  fl->cyc_p = 8;
  fl->pre = 2;
  fl->post = 2;
  fl->coarse_sweeps = 40;
  // level sizes
  int l = 0;
  for (int d = 0; d < 3; ++d) fl->ln[0][d] = grid->n[d];
  for (;;) {
    const int* c = fl->ln[l];
    const bool even = c[0] % 2 == 0 && c[1] % 2 == 0 && c[2] % 2 == 0;
    const int mx = std::max(c[0], std::max(c[1], c[2]));
    const int mn = std::min(c[0], std::min(c[1], c[2]));
    if (!even || mx <= kCoarseMax || mn < 4 || l + 1 >= ib_fluid::kMaxLevels) break;
    for (int d = 0; d < 3; ++d) fl->ln[l + 1][d] = c[d] / 2;
    ++l;
  }
  fl->nlev = l + 1;
  const int* cn = fl->ln[l];
  const int64_t ccells = (int64_t)cn[0] * cn[1] * cn[2];
  if (ccells > kCoarseCells) {
    delete fl;
    return IB_ERR_UNSUPPORTED;  // the coarsest lattice must fit one CTA's shared memory
  }
  fl->coarse_smem = 3 * (size_t)ccells * fl->rsize;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&fl->sm_count, cudaDevAttrMultiProcessorCount, dev);
  bool good = true;
  const int64_t cells = (int64_t)grid->n[0] * grid->n[1] * grid->n[2];
  good = good && ok(cudaMalloc(&fl->rhs0, 3 * cells * fl->rsize));
  good = good && ok(cudaMalloc(&fl->div, cells * fl->rsize));
  good = good && ok(cudaMalloc(&fl->ptmp, cells * fl->rsize));
  good = good && ok(cudaMalloc(&fl->red, sizeof(double) * (2 * kFluidRedCTAs + 4)));
  for (int k = 1; good && k < fl->nlev; ++k) {
    const int64_t c = (int64_t)fl->ln[k][0] * fl->ln[k][1] * fl->ln[k][2];
    good = ok(cudaMalloc(&fl->lphi[k], 3 * c * fl->rsize)) &&
           ok(cudaMalloc(&fl->lrhs[k], 3 * c * fl->rsize));
  }
  if (good) {
    // dynamic shared memory of the coarsest solve: the limit is a property of
    // the kernel, shared by every solver object, so it is set to the largest
    // coarsest level any object may have
    good = precision == IB_FP64
               ? ok(cudaFuncSetAttribute(k_coarse<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         3 * kCoarseCells * (int)sizeof(double)))
               : ok(cudaFuncSetAttribute(k_coarse<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         3 * kCoarseCells * (int)sizeof(float)));
  }
  if (!good) {
    ib_fluid_destroy(fl);
    return IB_ERR_CUDA;
  }
  (void)stream;
  *out = fl;
  return IB_OK;
}

ib_status ib_fluid_destroy(ib_fluid* fl) {
  if (!fl) return IB_ERR_INVALID_ARG;
  cudaFree(fl->rhs0);
  cudaFree(fl->div);
  cudaFree(fl->ptmp);
  cudaFree(fl->red);
  for (int k = 1; k < fl->nlev; ++k) {
    cudaFree(fl->lphi[k]);
    cudaFree(fl->lrhs[k]);
  }
  delete fl;
  return IB_OK;
}

ib_status ib_fluid_set_cycles(ib_fluid* fl, int32_t helmholtz_cycles, int32_t poisson_cycles) {
  if (!fl || helmholtz_cycles < 1 || helmholtz_cycles > 100 || poisson_cycles < 1 ||
      poisson_cycles > 100)
    return IB_ERR_INVALID_ARG;
  fl->cyc_h = helmholtz_cycles;
  fl->cyc_p = poisson_cycles;
  return IB_OK;
}

ib_status ib_fluid_levels(const ib_fluid* fl, int32_t* levels) {
  if (!fl || !levels) return IB_ERR_INVALID_ARG;
  *levels = fl->nlev;
  return IB_OK;
}

ib_status ib_fluid_step(ib_fluid* fl, const void* u, const void* f, void* u_next, void* p,
                        double* residuals, void* stream) {
  if (!fl || !u || !u_next) return IB_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  ib_status st = ibfe::fluid_step_async(fl, u, f, u_next, p, residuals, s);
  if (st != IB_OK) return st;
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

}  // extern "C"
