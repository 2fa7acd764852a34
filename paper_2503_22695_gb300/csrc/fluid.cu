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
// even and the largest exceeds 8 (rediscretised operator, h doubled per
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
  double* red;             // reduction partials (sums) and results
  double* rpart;           // residual partials, one pair per CTA of the finest grid
  int sm_count;
  size_t coarse_smem;
  // the step's launches captured once per set of field pointers and cycle
  // counts, replayed with one graph launch
  cudaStream_t cap;
  cudaGraphExec_t gexec;
  const void* gkey[4];
  int gcyc[2];
};

namespace ibfe {
namespace {

constexpr int kFluidRedCTAs = 1024;  // first-level reduction CTAs
constexpr int kCoarseMax = 8;        // coarsest level: every dimension <= 8 (or odd)
constexpr int kCoarseCells = 8192;   // shared-memory limit of the coarsest solve

bool ok(cudaError_t e) { return e == cudaSuccess; }

__device__ __forceinline__ int wrap_up(int i, int n) { return i + 1 == n ? 0 : i + 1; }
__device__ __forceinline__ int wrap_dn(int i, int n) { return i == 0 ? n - 1 : i - 1; }

// Kernels run on 3-D grids: x over i (or i/2), y over j, z over (component,
// k) as z = c n2 + k, so no index is divided per element.  Offsets within a
// component are 32-bit (every lattice has fewer than 2^31 / 3 cells).
struct Lat {
  int n0, n1, n2;
  __device__ __forceinline__ int at(int i, int j, int k) const { return (k * n1 + j) * n0 + i; }
  __device__ __forceinline__ int64_t cells() const { return (int64_t)n0 * n1 * n2; }
};

__device__ __forceinline__ bool thread_cell(int nx, const Lat& L, int& x, int& j, int& k,
                                            int& c) {
  x = blockIdx.x * blockDim.x + threadIdx.x;
  j = blockIdx.y * blockDim.y + threadIdx.y;
  c = blockIdx.z / L.n2;
  k = blockIdx.z - c * L.n2;
  return x < nx && j < L.n1;
}

// sum of the six lattice neighbours of (i, j, k) (periodic)
template <typename Real>
__device__ __forceinline__ Real nb_sum(const Real* __restrict__ f, const Lat& L, int i, int j,
                                       int k) {
  const int row = (k * L.n1 + j) * L.n0;
  const int plane = L.n0 * L.n1;
  const int k_up = k + 1 == L.n2 ? -k * plane : plane;
  const int k_dn = k == 0 ? (L.n2 - 1) * plane : -plane;
  const int j_up = j + 1 == L.n1 ? -j * L.n0 : L.n0;
  const int j_dn = j == 0 ? (L.n1 - 1) * L.n0 : -L.n0;
  const int idx = row + i;
  const Real sx = f[row + wrap_up(i, L.n0)] + f[row + wrap_dn(i, L.n0)];
  const Real sy = f[idx + j_up] + f[idx + j_dn];
  const Real sz = f[idx + k_up] + f[idx + k_dn];
  return sx + sy + sz;
}

// One colour of a red-black Gauss-Seidel sweep for (alpha - beta Lap) phi = rhs
// on ncomp stacked lattices: cells with (i + j + k) even (colour 0) or odd.
// phi_i = (rhs_i + b sum_nb phi) / (alpha + 6 b), b = beta / h^2.  n0 even;
// x runs over i / 2.
template <typename Real>
__global__ void __launch_bounds__(256) k_rb_smooth(Real* __restrict__ phi,
                                                   const Real* __restrict__ rhs, Lat L, Real b,
                                                   Real dinv, int color) {
  int m, j, k, c;
  if (!thread_cell(L.n0 >> 1, L, m, j, k, c)) return;
  const int i = 2 * m + ((j + k + color) & 1);
  const int64_t off = c * L.cells();
  Real* f = phi + off;
  const int idx = L.at(i, j, k);
  f[idx] = (rhs[off + idx] + b * nb_sum(f, L, i, j, k)) * dinv;
}

// Residual rhs - A phi of the 8 children of each coarse cell, averaged into
// the coarse right-hand side; the coarse correction is zeroed.  Grid over
// the coarse lattice Lc.
template <typename Real>
__global__ void __launch_bounds__(256) k_restrict(const Real* __restrict__ phi,
                                                  const Real* __restrict__ rhs,
                                                  Real* __restrict__ rc, Real* __restrict__ pc,
                                                  Lat L, Lat Lc, Real b, Real diag) {
  int I, J, K, c;
  if (!thread_cell(Lc.n0, Lc, I, J, K, c)) return;
  const int64_t off = c * L.cells();
  const Real* f = phi + off;
  const Real* g = rhs + off;
  Real s = Real(0);
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        const int i = 2 * I + di, j = 2 * J + dj, k = 2 * K + dk;
        const int idx = L.at(i, j, k);
        s += g[idx] - diag * f[idx] + b * nb_sum(f, L, i, j, k);
      }
  const int64_t t = c * Lc.cells() + Lc.at(I, J, K);
  rc[t] = s * Real(0.125);
  pc[t] = Real(0);
}

// phi_fine += trilinear (cell-centred) interpolation of the coarse correction:
// per axis 3/4 of the parent and 1/4 of the parent's neighbour on the side of
// the child.  One thread per coarse column I and fine (j, k): the two fine
// cells 2I (neighbour I-1) and 2I+1 (neighbour I+1) share the parent loads.
template <typename Real>
__global__ void __launch_bounds__(256) k_prolong(const Real* __restrict__ pc,
                                                 Real* __restrict__ phi, Lat L, Lat Lc) {
  int I, j, k, c;
  if (!thread_cell(Lc.n0, L, I, j, k, c)) return;
  const int J = j >> 1, K = k >> 1;
  const int J2 = (j & 1) ? wrap_up(J, Lc.n1) : wrap_dn(J, Lc.n1);
  const int K2 = (k & 1) ? wrap_up(K, Lc.n2) : wrap_dn(K, Lc.n2);
  const int Im = wrap_dn(I, Lc.n0), Ip = wrap_up(I, Lc.n0);
  const Real* q = pc + c * Lc.cells();
  const Real w1 = Real(0.75), w2 = Real(0.25);
  // the (J, K) plane weights folded first: column values at Im, I, Ip
  const Real* r00 = q + (K * Lc.n1 + J) * Lc.n0;
  const Real* r10 = q + (K * Lc.n1 + J2) * Lc.n0;
  const Real* r01 = q + (K2 * Lc.n1 + J) * Lc.n0;
  const Real* r11 = q + (K2 * Lc.n1 + J2) * Lc.n0;
  auto col = [&](int a) {
    return w1 * (w1 * r00[a] + w2 * r10[a]) + w2 * (w1 * r01[a] + w2 * r11[a]);
  };
  const Real cm = col(Im), c0 = col(I), cp = col(Ip);
  Real* f = phi + c * L.cells() + L.at(2 * I, j, k);
  f[0] += w1 * c0 + w2 * cm;
  f[1] += w1 * c0 + w2 * cp;
}

// Fixed-shape block sum in double (thread 0 holds the result).
__device__ __forceinline__ double block_sum_fl(double v, double* sh) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthr = blockDim.x * blockDim.y * blockDim.z;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < (nthr >> 5) ? sh[lane] : 0.0;
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
  const Lat L{n0, n1, n2};
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
          sp[idx] = (sr[idx] + b * nb_sum(sp, L, i, j, k)) * dinv;
        }
        __syncthreads();
      }
    } else {
      const Real w = Real(6.0 / 7.0);
      for (int t = threadIdx.x; t < cells; t += blockDim.x) {
        const int i = t % n0, jk = t / n0, j = jk % n1, k = jk / n1;
        const Real nv = (sr[t] + b * nb_sum(sp, L, i, j, k)) * dinv;
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
                                                   Real* __restrict__ rhs0, Real* ustar, int n,
                                                   Real a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const Real v = u[t];
  rhs0[t] = a * v + (f ? f[t] : Real(0));
  if (ustar != u) ustar[t] = v;
}

// div = (div_h u*) / dt at the cell centres (scale = 1 / (h dt)); p = 0.
template <typename Real>
__global__ void __launch_bounds__(256) k_divergence(const Real* __restrict__ u,
                                                    Real* __restrict__ div,
                                                    Real* __restrict__ p, Lat L, Real scale) {
  int i, j, k, c;
  if (!thread_cell(L.n0, L, i, j, k, c)) return;
  const int cells = (int)L.cells();
  const int t = L.at(i, j, k);
  const Real dx = u[L.at(wrap_up(i, L.n0), j, k)] - u[t];
  const Real dy = u[cells + L.at(i, wrap_up(j, L.n1), k)] - u[cells + t];
  const Real dz = u[2 * cells + L.at(i, j, wrap_up(k, L.n2))] - u[2 * cells + t];
  div[t] = (dx + dy + dz) * scale;
  p[t] = Real(0);
}

// u^{n+1} = u* - dt grad_h p (in place; scale = dt / h)
template <typename Real>
__global__ void __launch_bounds__(256) k_project(Real* __restrict__ u, const Real* __restrict__ p,
                                                 Lat L, Real scale) {
  int i, j, k, c;
  if (!thread_cell(L.n0, L, i, j, k, c)) return;
  const int cells = (int)L.cells();
  const int t = L.at(i, j, k);
  const Real pc = p[t];
  u[t] -= scale * (pc - p[L.at(wrap_dn(i, L.n0), j, k)]);
  u[cells + t] -= scale * (pc - p[L.at(i, wrap_dn(j, L.n1), k)]);
  u[2 * cells + t] -= scale * (pc - p[L.at(i, j, wrap_dn(k, L.n2))]);
}

// Fixed-shape sums: CTA b sums a contiguous chunk of x into part[b].  Each
// thread accumulates its (about 64) elements in Real, the CTA's threads in
// double: the sum only sets a mean that is removed, and on GB300 a double
// add per element would make this pass FP64-bound.
template <typename Real>
__global__ void __launch_bounds__(256) k_sums_l1(const Real* __restrict__ x, int n,
                                                 double* __restrict__ part) {
  __shared__ double sh[32];
  const int chunk = (n + gridDim.x - 1) / gridDim.x;
  const int e0 = blockIdx.x * chunk, e1 = min(n, e0 + chunk);
  Real s = Real(0);
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) s += x[e];
  const double t = block_sum_fl(double(s), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Squared residual of A phi = rhs and squared rhs, one partial pair per CTA
// of the 3-D grid (the grid's shape fixes the summation order).
template <typename Real>
__global__ void __launch_bounds__(256) k_resid_l1(const Real* __restrict__ phi,
                                                  const Real* __restrict__ rhs, Lat L, Real b,
                                                  Real diag, double* __restrict__ part) {
  __shared__ double sh[32];
  int i, j, k, c;
  double rr = 0.0, bb = 0.0;
  if (thread_cell(L.n0, L, i, j, k, c)) {
    const int64_t off = c * L.cells();
    const Real* f = phi + off;
    const int t = L.at(i, j, k);
    const double g = double(rhs[off + t]);
    const double res = g - double(diag) * double(f[t]) + double(b) * double(nb_sum(f, L, i, j, k));
    rr = res * res;
    bb = g * g;
  }
  rr = block_sum_fl(rr, sh);
  bb = block_sum_fl(bb, sh);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const int blk = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    part[2 * blk] = rr;
    part[2 * blk + 1] = bb;
  }
}

// out[k] = sum_b part[b * stride + k] for k < stride (one CTA); out[stride]
// = out[0] * scale
__global__ void __launch_bounds__(256) k_sums_l2(const double* __restrict__ part, int nblk,
                                                 int stride, double* __restrict__ out,
                                                 double scale) {
  __shared__ double sh[32];
  for (int k = 0; k < stride; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[b * stride + k];
    s = block_sum_fl(s, sh);
    if (threadIdx.x == 0) {
      out[k] = s;
      if (k == 0) out[stride] = s * scale;
    }
    __syncthreads();
  }
}

// x -= *mean
template <typename Real>
__global__ void __launch_bounds__(256) k_sub_mean(Real* __restrict__ x, int n,
                                                  const double* __restrict__ mean) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) x[t] -= Real(*mean);
}

// Block of 256 threads for a lattice row range of width nx: x as wide as the
// row allows (up to 64), y the rest.
dim3 block_for(int nx) {
  int bx = 64;
  while (bx > 8 && bx >= 2 * nx) bx >>= 1;
  return dim3(bx, 256 / bx, 1);
}

dim3 grid_for(int nx, int n1, int nz, dim3 blk) {
  return dim3((nx + blk.x - 1) / blk.x, (n1 + blk.y - 1) / blk.y, nz);
}

int blocks1d(int64_t n) { return (int)((n + 255) / 256); }

template <typename Real>
struct Fluid {
  static Lat lat(const int* n) { return Lat{n[0], n[1], n[2]}; }

  // `sweeps` red-black sweeps on phi (two colour passes each)
  static void smooth(Real* phi, const Real* rhs, const int* n, int ncomp, double alpha,
                     double beta, double h, int sweeps, cudaStream_t s) {
    const double b = beta / (h * h);
    const Real dinv = Real(1.0 / (alpha + 6.0 * b));
    const dim3 blk = block_for(n[0] / 2);
    const dim3 grd = grid_for(n[0] / 2, n[1], n[2] * ncomp, blk);
    for (int sw = 0; sw < sweeps; ++sw)
      for (int color = 0; color < 2; ++color)
        k_rb_smooth<Real><<<grd, blk, 0, s>>>(phi, rhs, lat(n), Real(b), dinv, color);
  }

  // one V-cycle from level l (phi, rhs of that level)
  static void vcycle(ib_fluid* fl, int l, Real* phi, const Real* rhs, int ncomp, double alpha,
                     double beta, bool singular, cudaStream_t s) {
    const int* n = fl->ln[l];
    const double h = fl->h * double(1 << l);
    const double b = beta / (h * h);
    if (l == fl->nlev - 1) {
      const bool even = n[0] % 2 == 0 && n[1] % 2 == 0 && n[2] % 2 == 0;
      k_coarse<Real><<<ncomp, 1024, fl->coarse_smem, s>>>(
          phi, rhs, n[0], n[1], n[2], Real(b), Real(1.0 / (alpha + 6.0 * b)),
          fl->coarse_sweeps, even ? 1 : 0, singular ? 1 : 0);
      return;
    }
    smooth(phi, rhs, n, ncomp, alpha, beta, h, fl->pre, s);
    Real* pc = (Real*)fl->lphi[l + 1];
    Real* rc = (Real*)fl->lrhs[l + 1];
    const int* m = fl->ln[l + 1];
    const dim3 bc = block_for(m[0]);
    k_restrict<Real><<<grid_for(m[0], m[1], m[2] * ncomp, bc), bc, 0, s>>>(
        phi, rhs, rc, pc, lat(n), lat(m), Real(b), Real(alpha + 6.0 * b));
    vcycle(fl, l + 1, pc, rc, ncomp, alpha, beta, singular, s);
    const dim3 bf = block_for(m[0]);
    k_prolong<Real><<<grid_for(m[0], n[1], n[2] * ncomp, bf), bf, 0, s>>>(pc, phi, lat(n),
                                                                          lat(m));
    smooth(phi, rhs, n, ncomp, alpha, beta, h, fl->post, s);
  }

  // relative residual ||rhs - A phi|| / ||rhs|| on the finest level
  // (synchronises s)
  static double residual(ib_fluid* fl, const Real* phi, const Real* rhs, int ncomp, double alpha,
                         double beta, cudaStream_t s) {
    const int* n = fl->n;
    const double b = beta / (fl->h * fl->h);
    const dim3 blk = block_for(n[0]);
    const dim3 grd = grid_for(n[0], n[1], n[2] * ncomp, blk);
    const int nblk = (int)(grd.x * grd.y * grd.z);
    double* part = fl->rpart;
    k_resid_l1<Real><<<grd, blk, 0, s>>>(phi, rhs, lat(n), Real(b), Real(alpha + 6.0 * b), part);
    k_sums_l2<<<1, 256, 0, s>>>(part, nblk, 2, fl->red + 2 * kFluidRedCTAs, 1.0);
    double out[2] = {0.0, 0.0};
    if (!ok(cudaMemcpyAsync(out, fl->red + 2 * kFluidRedCTAs, sizeof(out),
                            cudaMemcpyDeviceToHost, s)) ||
        !ok(cudaStreamSynchronize(s)))
      return -1.0;
    return out[1] > 0.0 ? std::sqrt(out[0] / out[1]) : std::sqrt(out[0]);
  }

  static void sub_mean(ib_fluid* fl, Real* x, int n, cudaStream_t s) {
    k_sums_l1<Real><<<kFluidRedCTAs, 256, 0, s>>>(x, n, fl->red);
    k_sums_l2<<<1, 256, 0, s>>>(fl->red, kFluidRedCTAs, 1, fl->red + 2 * kFluidRedCTAs,
                                1.0 / double(n));
    k_sub_mean<Real><<<blocks1d(n), 256, 0, s>>>(x, n, fl->red + 2 * kFluidRedCTAs + 1);
  }

  static ib_status step(ib_fluid* fl, const Real* u, const Real* f, Real* un, Real* p,
                        double* residuals, cudaStream_t s) {
    const int* n = fl->n;
    const int cells = n[0] * n[1] * n[2];
    const double a = fl->rho / fl->dt;
    Real* rhs0 = (Real*)fl->rhs0;
    Real* div = (Real*)fl->div;
    k_fluid_rhs<Real><<<blocks1d(3 * (int64_t)cells), 256, 0, s>>>(u, f, rhs0, un, 3 * cells,
                                                                    Real(a));
    for (int c = 0; c < fl->cyc_h; ++c) vcycle(fl, 0, un, rhs0, 3, a, fl->mu, false, s);
    double rh = 0.0, rp = 0.0;
    if (residuals) rh = residual(fl, un, rhs0, 3, a, fl->mu, s);
    const dim3 blk = block_for(n[0]);
    const dim3 grd = grid_for(n[0], n[1], n[2], blk);
    k_divergence<Real><<<grd, blk, 0, s>>>(un, div, p, lat(n), Real(1.0 / (fl->h * fl->dt)));
    sub_mean(fl, div, cells, s);  // exact zero mean (periodic box) up to rounding
    for (int c = 0; c < fl->cyc_p; ++c) vcycle(fl, 0, p, div, 1, 0.0, -1.0, true, s);
    if (residuals) rp = residual(fl, p, div, 1, 0.0, -1.0, s);
    sub_mean(fl, p, cells, s);
    k_project<Real><<<grd, blk, 0, s>>>(un, p, lat(n), Real(fl->dt / fl->h));
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

namespace {
ib_status step_direct(ib_fluid* fl, const void* u, const void* f, void* un, void* p,
                      double* residuals, cudaStream_t s) {
  if (fl->precision == IB_FP64)
    return Fluid<double>::step(fl, (const double*)u, (const double*)f, (double*)un, (double*)p,
                               residuals, s);
  return Fluid<float>::step(fl, (const float*)u, (const float*)f, (float*)un, (float*)p,
                            residuals, s);
}
}  // namespace

// Advance the fluid one step (internal entry shared with ib_step).  Without
// residuals (which need host round trips) the step's ~300 launches run as
// one CUDA graph, captured on the solver's own stream the first time a set
// of field pointers is seen; a caller's stream that is itself being
// captured gets the launches directly.
ib_status fluid_step_async(ib_fluid* fl, const void* u, const void* f, void* u_next, void* p,
                           double* residuals, cudaStream_t s) {
  void* pp = p ? p : fl->ptmp;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (residuals || !ok(cudaStreamIsCapturing(s, &cs)) || cs != cudaStreamCaptureStatusNone)
    return step_direct(fl, u, f, u_next, pp, residuals, s);
  const void* key[4] = {u, f, u_next, pp};
  const bool same = fl->gexec && fl->gcyc[0] == fl->cyc_h && fl->gcyc[1] == fl->cyc_p &&
                    std::memcmp(key, fl->gkey, sizeof(key)) == 0;
  if (!same) {
    if (fl->gexec) {
      cudaGraphExecDestroy(fl->gexec);
      fl->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (!ok(cudaStreamBeginCapture(fl->cap, cudaStreamCaptureModeThreadLocal)))
      return IB_ERR_CUDA;
    const ib_status st = step_direct(fl, u, f, u_next, pp, nullptr, fl->cap);
    const bool ended = ok(cudaStreamEndCapture(fl->cap, &g));
    if (st != IB_OK || !ended || !g) {
      if (g) cudaGraphDestroy(g);
      return st != IB_OK ? st : IB_ERR_CUDA;
    }
    const bool inst = ok(cudaGraphInstantiate(&fl->gexec, g, 0));
    cudaGraphDestroy(g);
    if (!inst) {
      fl->gexec = nullptr;
      return IB_ERR_CUDA;
    }
    std::memcpy(fl->gkey, key, sizeof(key));
    fl->gcyc[0] = fl->cyc_h;
    fl->gcyc[1] = fl->cyc_p;
  }
  return ok(cudaGraphLaunch(fl->gexec, s)) ? IB_OK : IB_ERR_CUDA;
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
  if (3 * (int64_t)grid->n[0] * grid->n[1] * grid->n[2] >= (int64_t(1) << 31))
    return IB_ERR_CAPACITY;  // 32-bit offsets within the stacked velocity components
  ib_fluid* fl = new ib_fluid();
  std::memset(fl, 0, sizeof(*fl));
  fl->precision = precision;
  fl->rsize = precision == IB_FP64 ? 8 : 4;
  for (int d = 0; d < 3; ++d) fl->n[d] = grid->n[d];
  fl->h = grid->h;
  fl->rho = rho;
  fl->mu = mu;
  fl->dt = dt;
  // V-cycles that reach the rounding floor of each precision on the
  // workloads of the tests (FP32: relative residuals ~1e-7 and ~1e-6)
  fl->cyc_h = precision == IB_FP64 ? 3 : 2;
  fl->cyc_p = precision == IB_FP64 ? 12 : 6;
  fl->pre = 2;
  fl->post = 2;
  fl->coarse_sweeps = 20;
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
  good = good && ok(cudaStreamCreateWithFlags(&fl->cap, cudaStreamNonBlocking));
  {
    const dim3 blk = block_for(grid->n[0]);
    const dim3 grd = grid_for(grid->n[0], grid->n[1], grid->n[2] * 3, blk);
    good = good && ok(cudaMalloc(&fl->rpart, sizeof(double) * 2 * grd.x * grd.y * grd.z));
  }
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
  if (fl->gexec) cudaGraphExecDestroy(fl->gexec);
  if (fl->cap) cudaStreamDestroy(fl->cap);
  cudaFree(fl->rhs0);
  cudaFree(fl->div);
  cudaFree(fl->ptmp);
  cudaFree(fl->red);
  cudaFree(fl->rpart);
  for (int k = 0; k < fl->nlev; ++k) {
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

ib_status ib_fluid_get_cycles(const ib_fluid* fl, int32_t cycles[2]) {
  if (!fl || !cycles) return IB_ERR_INVALID_ARG;
  cycles[0] = fl->cyc_h;
  cycles[1] = fl->cyc_p;
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
