// Plan-free total elastic energy for callers that cannot allocate device
// memory.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured on its stream, runtimes that hand all device memory to a
// fixed pool up front, or latency-critical loops that must not enter the
// allocator.  ib_fe_energy_noalloc serves them: it needs no plan, and its
// scratch (one partial energy per element, one partial sum per reduction CTA)
// lives in the file-scope device array below, which every GPU that loads this
// library holds until the process exits.  The caller passes the mesh, the
// material table, the positions and a device double for the result.
//
// The scratch is shared by every call on a device and keeps the last call's
// contents; each call overwrites every entry it reads, so nothing has to be
// cleared.  Calls that overlap on the GPU (two streams, or two host threads)
// race on the scratch and must not be issued.
#include <cstring>
#include <mutex>

#include "ib_device.cuh"

namespace ibfe {
namespace {

constexpr int kNoAllocMaxElems = 262144;  // largest mesh accepted (2 MiB of partials)
constexpr int kNoAllocCTAs = 128;         // first-level reduction CTAs
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxElems + kNoAllocCTAs];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kNoAllocMaxDevices] = {nullptr};

template <typename T>
__device__ __forceinline__ T det3_na(const T A[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

// Strain energy of one element, sum over its 8 Gauss points of Psi w_q j0,
// for the laws of Section 3 (Psi_1 to Psi_4) and Section 6.3 (neo-Hookean),
// with the same cancellation-free invariants as the force kernel.  Writes NaN
// for an element with an out-of-range node or material index.
__global__ void __launch_bounds__(128) k_energy_noalloc(const int32_t* __restrict__ conn,
                                                        const float* __restrict__ X,
                                                        const float* __restrict__ fib,
                                                        const int32_t* __restrict__ mat_id,
                                                        const int32_t* __restrict__ cell,
                                                        const float* __restrict__ off, int E,
                                                        int N, float h, MatTable mt,
                                                        double* __restrict__ part) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int node[8];
  bool bad = false;
  for (int a = 0; a < 8; ++a) {
    node[a] = conn[(int64_t)a * E + e];
    if (node[a] < 0 || node[a] >= N) {
      bad = true;
      node[a] = 0;
    }
  }
  const int mid = mat_id ? mat_id[e] : 0;
  if (mid < 0 || mid >= mt.n) bad = true;
  if (bad) {
    part[e] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  float dX[8][3], du[8][3];
  for (int a = 0; a < 8; ++a)
    for (int d = 0; d < 3; ++d) {
      dX[a][d] = X[(int64_t)d * N + node[a]] - X[(int64_t)d * N + node[0]];
      const float dx = (float(cell[(int64_t)d * N + node[a]] - cell[(int64_t)d * N + node[0]]) +
                        (off[(int64_t)d * N + node[a]] - off[(int64_t)d * N + node[0]])) * h;
      du[a][d] = dx - dX[a][d];
    }
  float ef[3] = {1.f, 0.f, 0.f}, es[3] = {0.f, 1.f, 0.f};
  if (fib)
    for (int i = 0; i < 3; ++i) {
      ef[i] = fib[(int64_t)i * E + e];
      es[i] = fib[(int64_t)(3 + i) * E + e];
    }
  const int model = mt.model[mid];
  const double* p = mt.p[mid];
  double en = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float J0[3][3], Du[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        float s = 0.f, t = 0.f;
#pragma unroll
        for (int a = 1; a < 8; ++a) {
          s += dX[a][i] * float(shape_dxi(a, q, j));
          t += du[a][i] * float(shape_dxi(a, q, j));
        }
        J0[i][j] = s;
        Du[i][j] = t;
      }
    const float j0 = det3_na(J0);
    float Ji[3][3];
    Ji[0][0] = (J0[1][1] * J0[2][2] - J0[1][2] * J0[2][1]) / j0;
    Ji[0][1] = (J0[0][2] * J0[2][1] - J0[0][1] * J0[2][2]) / j0;
    Ji[0][2] = (J0[0][1] * J0[1][2] - J0[0][2] * J0[1][1]) / j0;
    Ji[1][0] = (J0[1][2] * J0[2][0] - J0[1][0] * J0[2][2]) / j0;
    Ji[1][1] = (J0[0][0] * J0[2][2] - J0[0][2] * J0[2][0]) / j0;
    Ji[1][2] = (J0[0][2] * J0[1][0] - J0[0][0] * J0[1][2]) / j0;
    Ji[2][0] = (J0[1][0] * J0[2][1] - J0[1][1] * J0[2][0]) / j0;
    Ji[2][1] = (J0[0][1] * J0[2][0] - J0[0][0] * J0[2][1]) / j0;
    Ji[2][2] = (J0[0][0] * J0[1][1] - J0[0][1] * J0[1][0]) / j0;
    float H[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        H[i][j] = Du[i][0] * Ji[0][j] + Du[i][1] * Ji[1][j] + Du[i][2] * Ji[2][j];
    // J - 1, I1 - 3 and the fibre invariants without cancellation, in double
    const double tr = double(H[0][0]) + double(H[1][1]) + double(H[2][2]);
    double trH2 = 0.0, HH = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        trH2 += double(H[i][j]) * double(H[j][i]);
        HH += double(H[i][j]) * double(H[i][j]);
      }
    const double Jm1 = tr + 0.5 * (tr * tr - trH2) + double(det3_na(H));
    const double lnJ = log1p(Jm1);
    const double Jm23m1 = expm1(-2.0 / 3.0 * lnJ);
    const double Ibm3 = (1.0 + Jm23m1) * (2.0 * tr + HH) + 3.0 * Jm23m1;
    auto fibre_d = [&](const float* v, bool clamp) {
      double I4m1 = double(v[0]) * v[0] + double(v[1]) * v[1] + (double(v[2]) * v[2] - 1.0);
      for (int i = 0; i < 3; ++i) {
        const double Hv = double(H[i][0]) * v[0] + double(H[i][1]) * v[1] + double(H[i][2]) * v[2];
        I4m1 += 2.0 * double(v[i]) * Hv + Hv * Hv;
      }
      return (!clamp || I4m1 > 0.0) ? I4m1 : 0.0;
    };
    double psi;
    if (model == IB_NEO_HOOKEAN) {
      psi = p[0] * Ibm3 + 0.5 * p[1] * lnJ * lnJ;
    } else if (model == IB_FIBRE1) {
      const double d = fibre_d(ef, true);
      psi = p[0] * Ibm3 + p[1] / (2.0 * p[2]) * expm1(p[2] * d * d) + 0.5 * p[3] * lnJ * lnJ;
    } else if (model == IB_FIBRE2) {
      const double d = fibre_d(ef, false);
      psi = p[0] * expm1(p[1] * Ibm3) + p[2] / (2.0 * p[3]) * expm1(p[3] * d * d) +
            0.5 * p[4] * lnJ * lnJ;
    } else if (model == IB_STD_REINF) {
      // 2 I4f - I5f - 1 = |e|^2 - 1 - |w|^2 with w = (C - I) e
      //                 = H e + H^T e + H^T H e
      const double d = fibre_d(ef, false);
      double He[3], ww = 0.0;
      for (int i = 0; i < 3; ++i)
        He[i] = double(H[i][0]) * ef[0] + double(H[i][1]) * ef[1] + double(H[i][2]) * ef[2];
      for (int j = 0; j < 3; ++j) {
        double w = He[j];
        for (int i = 0; i < 3; ++i) w += double(H[i][j]) * (double(ef[i]) + He[i]);
        ww += w * w;
      }
      const double en1 = double(ef[0]) * ef[0] + double(ef[1]) * ef[1] + (double(ef[2]) * ef[2] - 1.0);
      psi = 0.5 * p[0] * Ibm3 + 0.5 * (p[0] - p[1]) * (en1 - ww) +
            0.125 * (p[2] + p[0] - 4.0 * p[1]) * d * d + 0.5 * p[3] * lnJ * lnJ;
    } else {
      const double df = fibre_d(ef, true), ds = fibre_d(es, true);
      double I8 = double(ef[0]) * es[0] + double(ef[1]) * es[1] + double(ef[2]) * es[2];
      for (int i = 0; i < 3; ++i) {
        const double Hf = double(H[i][0]) * ef[0] + double(H[i][1]) * ef[1] + double(H[i][2]) * ef[2];
        const double Hs = double(H[i][0]) * es[0] + double(H[i][1]) * es[1] + double(H[i][2]) * es[2];
        I8 += double(ef[i]) * Hs + double(es[i]) * Hf + Hf * Hs;
      }
      psi = p[0] / (2.0 * p[1]) * expm1(p[1] * Ibm3) + p[2] / (2.0 * p[3]) * expm1(p[3] * df * df) +
            p[4] / (2.0 * p[5]) * expm1(p[5] * ds * ds) + p[6] / (2.0 * p[7]) * expm1(p[7] * I8 * I8) +
            0.5 * p[8] * lnJ * lnJ;
    }
    if (p[kTa] != 0.0) {  // potential of the active fibre stress (Section 6.1)
      const double d4 = fibre_d(ef, false), r = sqrt(1.0 + d4);
      psi += 0.5 * p[kTa] * d4 * ((1.0 - 4.9) + 4.9 * (2.0 / 3.0) * (2.0 + d4 + r) / (r + 1.0));
    }
    en += psi * double(j0);
  }
  part[e] = en;
}

__device__ __forceinline__ double block_sum_na(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;
}

// Fixed-shape two-level sum: CTA b sums a contiguous chunk of the partials
// into part[kNoAllocMaxElems + b]; one CTA then sums those.
__global__ void __launch_bounds__(256) k_sum_l1_noalloc(double* __restrict__ part, int E) {
  __shared__ double sh[32];
  const int chunk = (E + gridDim.x - 1) / gridDim.x;
  const int e0 = blockIdx.x * chunk, e1 = min(E, e0 + chunk);
  double s = 0.0;
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) s += part[e];
  s = block_sum_na(s, sh);
  if (threadIdx.x == 0) part[kNoAllocMaxElems + blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_sum_l2_noalloc(const double* __restrict__ part,
                                                        double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < kNoAllocCTAs; b += blockDim.x) s += part[kNoAllocMaxElems + b];
  s = block_sum_na(s, sh);
  if (threadIdx.x == 0) *out = s;
}

}  // namespace
}  // namespace ibfe

extern "C" ib_status ib_fe_energy_noalloc(const ib_mesh* mesh, const ib_material* mats,
                                          int32_t n_mats, const ib_pos* x, double h,
                                          double* energy, void* stream) {
  using namespace ibfe;
  if (!mesh || !mats || !x || !energy || !x->cell || !x->off || !mesh->X) return IB_ERR_INVALID_ARG;
  if (mesh->n_nodes <= 0 || mesh->n_elems < 0 || (mesh->n_elems > 0 && !mesh->conn))
    return IB_ERR_INVALID_ARG;
  if (mesh->elem_type != IB_ELEM_HEX8) return IB_ERR_UNSUPPORTED;  // hexahedra only
  if (!(h > 0.0)) return IB_ERR_INVALID_ARG;
  if (mesh->n_elems > kNoAllocMaxElems) return IB_ERR_CAPACITY;
  if (n_mats <= 0 || n_mats > IB_MAX_MATERIALS) return IB_ERR_INVALID_ARG;
  MatTable mt;
  std::memset(&mt, 0, sizeof(mt));
  mt.n = n_mats;
  for (int m = 0; m < n_mats; ++m) {
    if (!material_valid(mats[m])) return IB_ERR_INVALID_ARG;
    mt.model[m] = mats[m].model;
    for (int k = 0; k < mats[m].n_params; ++k) mt.p[m][k] = mats[m].params[k];
    mt.p[m][kTa] = mats[m].Ta;
    mat_entry_finish(mt.p[m], mt.pf[m], mt.act[m]);
  }
  // once per device, with that device current: the device address of the
  // scratch array (host code only sees a host-side stand-in for the symbol)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices)
    return IB_ERR_CUDA;
  double* scratch;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return IB_ERR_CUDA;
      g_scratch_ptr[dev] = static_cast<double*>(ptr);
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int E = mesh->n_elems;
  if (E > 0)
    k_energy_noalloc<<<(E + 127) / 128, 128, 0, s>>>(
        mesh->conn, static_cast<const float*>(mesh->X), static_cast<const float*>(mesh->fibres),
        mesh->mat_id, x->cell, x->off, E, mesh->n_nodes, (float)h, mt, scratch);
  k_sum_l1_noalloc<<<kNoAllocCTAs, 256, 0, s>>>(scratch, E);
  k_sum_l2_noalloc<<<1, 256, 0, s>>>(scratch, energy);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}
