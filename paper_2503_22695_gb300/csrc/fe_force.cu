// Host side of the hyperelastic nodal force (Section 4.4) and its adjoints:
// the choice of kernel instantiation per call, and the deterministic
// per-material reductions of energies and parameter gradients.  The device
// code is in fe_kernel.cuh.
#include <algorithm>

#include "dfloat.cuh"
#include "ib_device.cuh"

namespace ibfe {
namespace {

// Deterministic per-material sums of per-element partials in two levels.
// Material m's elements lie in the range mrange[m] (the whole mesh for a
// plan of one structure; its instance's elements in a packed plan): CTA b
// reduces chunk b of that range, all values of the material in one pass, each
// value with its own fixed-shape tree (warp shuffles, then the warp sums; one
// barrier pair per material); then one warp per (material, value) pair sums
// the per-CTA partials with the same tree.  The partition and the trees
// depend only on the range, so an instance of a packed plan gets the bits of
// a plan of its own.
__device__ __forceinline__ double warp_tree(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;  // valid in lane 0
}

constexpr int kRedThreads = 256;

// The block_sum tree for every value k < nvals of a thread at once (one
// barrier pair for all of them); value k's sum is bitwise the one block_sum
// forms for it alone.
__device__ __forceinline__ void block_sum_row(double (&v)[kParamRow], int nvals,
                                              double (*sh)[kParamRow]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kParamRow; ++k)
    if (k < nvals) {
      v[k] = warp_tree(v[k]);
      if (lane == 0) sh[warp][k] = v[k];
    }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < kParamRow; ++k)
      if (k < nvals) v[k] = warp_tree(lane < (int)(blockDim.x >> 5) ? sh[lane][k] : 0.0);
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_reduce_l1(const T* __restrict__ part,
                                                           const int32_t* __restrict__ mat_id,
                                                           const int2* __restrict__ mrange,
                                                           int E, int nvals, int n_mats,
                                                           double* __restrict__ rpart) {
  __shared__ double sh[32][kParamRow];
  for (int m = 0; m < n_mats; ++m) {
    const int2 r = mrange[m];
    const int chunk = (r.y - r.x + gridDim.x - 1) / gridDim.x;
    const int e0 = r.x + blockIdx.x * chunk, e1 = min(r.y, e0 + chunk);
    double s[kParamRow];
#pragma unroll
    for (int k = 0; k < kParamRow; ++k) s[k] = 0.0;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x)
      if ((mat_id ? __ldg(mat_id + e) : 0) == m) {
#pragma unroll
        for (int k = 0; k < kParamRow; ++k)
          if (k < nvals) s[k] += double(__ldg(part + (int64_t)k * E + e));
      }
    block_sum_row(s, nvals, sh);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < kParamRow; ++k)
        if (k < nvals) rpart[((int64_t)blockIdx.x * n_mats + m) * kParamRow + k] = s[k];
    }
  }
}

// One warp per (material, value): the block_sum tree of a kRedThreads-thread
// CTA whose thread t holds partial t (nblk <= kRedThreads), evaluated warp
// by warp.
__global__ void __launch_bounds__(kRedThreads) k_reduce_l2(const double* __restrict__ rpart,
                                                           int nblk, int nvals, int n_mats,
                                                           double* __restrict__ out) {
  const int pair = blockIdx.x * (kRedThreads / 32) + (threadIdx.x >> 5);
  if (pair >= n_mats * nvals) return;
  const int m = pair / nvals, k = pair % nvals, lane = threadIdx.x & 31;
  double ws = 0.0;  // lane w: the tree sum of the partials of thread block w
  for (int w = 0; w < kRedThreads / 32; ++w) {
    const int b = 32 * w + lane;
    double v = 0.0;
    if (b < nblk) v += rpart[((int64_t)b * n_mats + m) * kParamRow + k];
    v = __shfl_sync(0xffffffffu, warp_tree(v), 0);
    if (lane == w) ws = v;
  }
  const double t = warp_tree(ws);
  if (lane == 0) out[m * kParamRow + k] = t;
}

// The smallest instantiated law set covering the material table (every
// model in it, the active term if a material has T_a != 0 or the parameter
// gradients are wanted: they include d/dT_a).
int law_set(const ib_plan* p, const MatTable& mt, bool params) {
  int need = params ? kLawAct : 0;
  if (p->mat_dev) need |= p->mat_need;  // packed plans: the device table's laws
  for (int m = 0; m < mt.n; ++m) {
    need |= 1 << mt.model[m];
    if (mt.p[m][kTa] != 0.0) need |= kLawAct;
  }
  if ((need & ~kLawBase) == 0) return kLawBase;
  if ((need & ~kLawBaseAct) == 0) return kLawBaseAct;
  return kLawAll;
}

}  // namespace

#define IBFE_FE_ARGS p, mt, xa, off, v, out, s
#define HEX IB_ELEM_HEX8

namespace {
// IB_FP32_SPLIT_DFVOL plans: every law, the exact volumetric invariant; one
// instantiation per element and output.
constexpr int kLawVol = kLawAll | kLawVolX;
template <int T>
ib_status vol_force(ib_plan* p, const MatTable& mt, const void* xa, const float* off,
                    const void* v, void* out, bool energy, bool adj, bool params,
                    cudaStream_t s) {
  if (adj)
    return params ? fe_run<float, df, false, true, true, kLawVol, T>(IBFE_FE_ARGS)
                  : fe_run<float, df, false, true, false, kLawVol, T>(IBFE_FE_ARGS);
  return energy ? fe_run<float, df, true, false, false, kLawVol, T>(IBFE_FE_ARGS)
                : fe_run<float, df, false, false, false, kLawVol, T>(IBFE_FE_ARGS);
}

// Tetrahedral meshes (P1 and P2): one instantiation per precision and
// output (all laws).
template <int T>
ib_status tet_force(ib_plan* p, const MatTable& mt, const void* xa, const float* off,
                    const void* v, void* out, bool energy, bool adj, bool params,
                    cudaStream_t s) {
  constexpr int L = kLawAll;
  if (p->precision == IB_FP64) {
    if (adj)
      return params ? fe_run<double, double, false, true, true, L, T>(IBFE_FE_ARGS)
                    : fe_run<double, double, false, true, false, L, T>(IBFE_FE_ARGS);
    return energy ? fe_run<double, double, true, false, false, L, T>(IBFE_FE_ARGS)
                  : fe_run<double, double, false, false, false, L, T>(IBFE_FE_ARGS);
  }
  if (p->precision == IB_FP32_SPLIT_F32STAB) {
    if (adj)
      return params ? fe_run<float, float, false, true, true, L, T>(IBFE_FE_ARGS)
                    : fe_run<float, float, false, true, false, L, T>(IBFE_FE_ARGS);
    return energy ? fe_run<float, float, true, false, false, L, T>(IBFE_FE_ARGS)
                  : fe_run<float, float, false, false, false, L, T>(IBFE_FE_ARGS);
  }
  if (p->precision == IB_FP32_SPLIT_DFVOL) return vol_force<T>(p, mt, xa, off, v, out, energy,
                                                               adj, params, s);
  if (adj)
    return params ? fe_run<float, df, false, true, true, L, T>(IBFE_FE_ARGS)
                  : fe_run<float, df, false, true, false, L, T>(IBFE_FE_ARGS);
  return energy ? fe_run<float, df, true, false, false, L, T>(IBFE_FE_ARGS)
                : fe_run<float, df, false, false, false, L, T>(IBFE_FE_ARGS);
}
}  // namespace

ib_status launch_fe_force(ib_plan* p, const MatTable& mt, const void* xa, const float* off,
                          void* out, bool energy, cudaStream_t s) {
  const void* v = nullptr;
  if (p->elem == IB_ELEM_TET4)
    return tet_force<IB_ELEM_TET4>(p, mt, xa, off, v, out, energy, false, false, s);
  if (p->elem == IB_ELEM_TET10)
    return tet_force<IB_ELEM_TET10>(p, mt, xa, off, v, out, energy, false, false, s);
  const int set = law_set(p, mt, false);
  if (p->precision == IB_FP32_SPLIT_DFVOL)
    return vol_force<HEX>(p, mt, xa, off, v, out, energy, false, false, s);
  if (p->precision == IB_FP64)
    return energy ? fe_run<double, double, true, false, false, kLawAll, HEX>(IBFE_FE_ARGS)
                  : fe_run<double, double, false, false, false, kLawAll, HEX>(IBFE_FE_ARGS);
  if (p->precision == IB_FP32_SPLIT_F32STAB) {
    if (energy) return fe_run<float, float, true, false, false, kLawAll, HEX>(IBFE_FE_ARGS);
    return set == kLawBase
               ? fe_run<float, float, false, false, false, kLawBase, HEX>(IBFE_FE_ARGS)
               : fe_run<float, float, false, false, false, kLawAll, HEX>(IBFE_FE_ARGS);
  }
  if (energy) return fe_run<float, df, true, false, false, kLawAll, HEX>(IBFE_FE_ARGS);
  if (set == kLawBase)
    return fe_run<float, df, false, false, false, kLawBase, HEX>(IBFE_FE_ARGS);
  if (set == kLawBaseAct)
    return fe_run<float, df, false, false, false, kLawBaseAct, HEX>(IBFE_FE_ARGS);
  return fe_run<float, df, false, false, false, kLawAll, HEX>(IBFE_FE_ARGS);
}

ib_status launch_fe_force_adj(ib_plan* p, const MatTable& mt, const void* xa, const float* off,
                              const void* v, void* out, bool params, cudaStream_t s) {
  if (p->elem == IB_ELEM_TET4)
    return tet_force<IB_ELEM_TET4>(p, mt, xa, off, v, out, false, true, params, s);
  if (p->elem == IB_ELEM_TET10)
    return tet_force<IB_ELEM_TET10>(p, mt, xa, off, v, out, false, true, params, s);
  const int set = law_set(p, mt, params);
  if (p->precision == IB_FP32_SPLIT_DFVOL)
    return vol_force<HEX>(p, mt, xa, off, v, out, false, true, params, s);
  if (p->precision == IB_FP64)
    return params ? fe_run<double, double, false, true, true, kLawAll, HEX>(IBFE_FE_ARGS)
                  : fe_run<double, double, false, true, false, kLawAll, HEX>(IBFE_FE_ARGS);
  if (p->precision == IB_FP32_SPLIT_F32STAB)
    return params ? fe_run<float, float, false, true, true, kLawAll, HEX>(IBFE_FE_ARGS)
                  : fe_run<float, float, false, true, false, kLawAll, HEX>(IBFE_FE_ARGS);
  if (params)
    return set == kLawBaseAct
               ? fe_run<float, df, false, true, true, kLawBaseAct, HEX>(IBFE_FE_ARGS)
               : fe_run<float, df, false, true, true, kLawAll, HEX>(IBFE_FE_ARGS);
  if (set == kLawBase) return fe_run<float, df, false, true, false, kLawBase, HEX>(IBFE_FE_ARGS);
  if (set == kLawBaseAct)
    return fe_run<float, df, false, true, false, kLawBaseAct, HEX>(IBFE_FE_ARGS);
  return fe_run<float, df, false, true, false, kLawAll, HEX>(IBFE_FE_ARGS);
}

#undef HEX
#undef IBFE_FE_ARGS

ib_status launch_reduce_parts(ib_plan* p, int nvals, int n_mats, cudaStream_t s,
                              bool real_parts) {
  if (n_mats > p->mat_cap) return IB_ERR_INVALID_ARG;
  if (p->E == 0) {
    cudaMemsetAsync(p->ered, 0, sizeof(double) * kParamRow * p->mat_cap, s);
    return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
  }
  static_assert(kReduceCTAs <= kRedThreads, "one partial per thread of the second level");
  // FP32 partials are widened exactly: the sums are those of their doubles
  if (real_parts && p->precision != IB_FP64)
    k_reduce_l1<float><<<kReduceCTAs, kRedThreads, 0, s>>>(
        reinterpret_cast<const float*>(p->epart), p->mat_id, p->mat_range, p->E, nvals, n_mats,
        p->rpart);
  else
    k_reduce_l1<double><<<kReduceCTAs, kRedThreads, 0, s>>>(p->epart, p->mat_id, p->mat_range,
                                                            p->E, nvals, n_mats, p->rpart);
  const int pairs = n_mats * nvals, per = kRedThreads / 32;
  k_reduce_l2<<<(pairs + per - 1) / per, kRedThreads, 0, s>>>(p->rpart, kReduceCTAs, nvals,
                                                             n_mats, p->ered);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

}  // namespace ibfe
