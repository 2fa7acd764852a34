// Gauss points of the structure as Lagrangian markers, binned by Eulerian tile.
//
// k_points evaluates, per element and Gauss point q (index gq = q*E + e):
//   chi_q = sum_a N_a(xi_q) x_a          (split: integer cell + offset in [0,1))
//   V_q   = w_q j0 sum_a N_a(xi_q) V_a / m_a   (optional carried value; for the
//           spreading of Section 4.4 V = G, the lumped projection of the nodal
//           forces onto the FE space)
// and the sort key tile * 512 + cell-in-tile of the (periodically wrapped)
// cell containing chi_q, for 8^3-cell Eulerian tiles.  The points are then
// ordered by a stable LSD radix sort on that key (8-bit digits, per-block
// digit histograms, a per-digit scan across blocks, stable in-block ranks from
// warp match masks): points are grouped by tile, ordered by cell inside a tile
// (so neighbouring threads read neighbouring faces), and equal keys keep gq
// order, so the sorted sequence -- hence every downstream summation order --
// is identical on every call.  That path serves FP64 plans, whose spreading
// sums doubles in point order.
//
// FP32 plans bin instead of sorting: their spreading accumulates exact
// integers and their interpolation is per point, so a point's place inside
// its tile does not change any result.  k_points counts the points of each
// tile with warp-aggregated integer atomics and keeps each point's slot, one
// scan turns the counts into tile ranges, and one scatter writes the
// tile-grouped arrays.
#include "ib_device.cuh"

namespace ibfe {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortChunk = kSortThreads * kSortItems;
constexpr int kLocalBits = 9;  // cell within an 8^3 tile

template <typename Real>
struct PtArgs {
  int E;
  int64_t N;
  const int32_t* conn;
  NodeLoader<Real> pos;
  const Real* V;         // [3][N] or null
  const Real* inv_mass;  // [N]
  const Real* wj0;       // [nq][E]
  GridDev g;
  const InstDev* inst;   // packed plans: instance table, else null
  const int32_t* elem_inst;  // packed plans: instance of each element
  int32_t* q_cell;
  Real* q_off;           // [3][Q]
  Real* q_val;           // [3][Q]
  uint32_t* key;
  int32_t* val;
  int32_t* count;        // binning: points per tile
  int* status;
};

// Packed cell, and the tile key with either the point's slot in its tile
// (binning: one atomic per distinct tile of the warp) or its index (sorting).
template <typename Real, bool kBin>
__device__ __forceinline__ void bin_point(const PtArgs<Real>& A, int64_t gq, const int cw[3],
                                          const TileGeo& geo) {
  A.q_cell[gq] = pack_cell(cw[0], cw[1], cw[2]);
  const uint32_t tile = (uint32_t)(geo.base + (cw[0] >> kTileShift) +
                                   geo.nt[0] * ((cw[1] >> kTileShift) +
                                                geo.nt[1] * (cw[2] >> kTileShift)));
  if (kBin) {
    const unsigned act = __activemask();
    const unsigned peers = __match_any_sync(act, tile);
    const int leader = __ffs(peers) - 1, lane = threadIdx.x & 31;
    int base = 0;
    if (lane == leader) base = atomicAdd(A.count + tile, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    A.key[gq] = tile;
    A.val[gq] = base + __popc(peers & ((1u << lane) - 1u));
  } else {
    const uint32_t local = (uint32_t)((((cw[2] & 7) << 3) | (cw[1] & 7)) << 3 | (cw[0] & 7));
    A.key[gq] = (tile << kLocalBits) | local;
    A.val[gq] = (int32_t)gq;
  }
}

// kVal: the call carries nodal values (A.V); without them the kernel keeps
// no per-corner values live (fewer registers, more resident warps)
template <typename Real, bool kBin, int kEl, bool kPacked, bool kVal = true>
__global__ void __launch_bounds__(128) k_points(PtArgs<Real> A) {
  using EL = El<kEl>;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= A.E) return;
  const int E = A.E;
  const int64_t Q = (int64_t)EL::Q * E;
  const TileGeo geo = tile_geo<kPacked>(A.g, A.inst, A.elem_inst, e);  // the element's grid
  int c0[3];
  Real o0[3];
  Real dl[EL::C][3];
  Real Vn[EL::C][3];
  bool bad = false;
#pragma unroll
  for (int a = 0; a < EL::C; ++a) {
    const int node = __ldg(A.conn + a * E + e);
    int c[3];
    Real o[3];
    A.pos.load(node, c, o);
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (!(o[d] >= Real(0) && o[d] < Real(1))) bad = true;
    if (a == 0) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        c0[d] = c[d];
        o0[d] = o[d];
        dl[0][d] = Real(0);
      }
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) dl[a][d] = Real(c[d] - c0[d]) + (o[d] - o0[d]);
    }
    if (kVal && A.V) {
      const Real im = __ldg(A.inv_mass + node);
#pragma unroll
      for (int d = 0; d < 3; ++d) Vn[a][d] = __ldg(A.V + d * A.N + node) * im;
    }
  }
  if (bad) {  // keep indices in range; the caller sees IB_ERR_NONFINITE
    set_status(A.status, kStatNonfinite);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      c0[d] = 0;
      o0[d] = Real(0);
#pragma unroll
      for (int a = 0; a < EL::C; ++a) dl[a][d] = Real(0);
    }
  }
#pragma unroll
  for (int q = 0; q < EL::Q; ++q) {
    const int64_t gq = (int64_t)q * E + e;
    int cw[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      Real s = Real(0);
#pragma unroll
      for (int a = 1; a < EL::C; ++a) s += Real(EL::N(a, q)) * dl[a][d];
      Real t = o0[d] + s;
      Real k = floor(t);
      Real off = t - k;
      if (off >= Real(1)) {  // rounding guard: keep the offset in [0,1)
        off = Real(0);
        k += Real(1);
      }
      cw[d] = wrap_idx(c0[d] + (int)k, geo.n[d]);
      A.q_off[d * Q + gq] = off;
    }
    bin_point<Real, kBin>(A, gq, cw, geo);
    if (kVal && A.V) {
      const Real w = __ldg(A.wj0 + gq);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        Real s = Real(0);
#pragma unroll
        for (int a = 0; a < EL::C; ++a) s += Real(EL::N(a, q)) * Vn[a][d];
        A.q_val[d * Q + gq] = w * s;
      }
    }
  }
}

// Nodal quadrature rule (Section 4.4): the coupling points are the nodes,
// chi_a = x_a (gq = a), and a carried value is V_a itself.
template <typename Real, bool kBin>
__global__ void __launch_bounds__(256) k_points_nodal(PtArgs<Real> A) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= A.N) return;
  const int64_t N = A.N;
  int c[3];
  Real o[3];
  A.pos.load(a, c, o);
  bool bad = false;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    if (!(o[d] >= Real(0) && o[d] < Real(1))) bad = true;
  if (bad) {  // keep indices in range; the caller sees IB_ERR_NONFINITE
    set_status(A.status, kStatNonfinite);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      c[d] = 0;
      o[d] = Real(0);
    }
  }
  // (packed plans hold Gauss-rule structures only: the plan's grid)
  const TileGeo geo = tile_geo<false>(A.g, nullptr, nullptr, 0);
  int cw[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    cw[d] = wrap_idx(c[d], geo.n[d]);
    A.q_off[d * N + a] = o[d];
  }
  bin_point<Real, kBin>(A, a, cw, geo);
  if (A.V) {
#pragma unroll
    for (int d = 0; d < 3; ++d) A.q_val[d * N + a] = __ldg(A.V + d * N + a);
  }
}

// Carried values only (positions already built): V_q = w_q j0 sum_a N_a V_a / m_a.
template <typename Real, int kEl>
__global__ void __launch_bounds__(128) k_point_values(int E, int64_t N,
                                                     const int32_t* __restrict__ conn,
                                                     const Real* __restrict__ V,
                                                     const Real* __restrict__ inv_mass,
                                                     const Real* __restrict__ wj0,
                                                     Real* __restrict__ q_val) {
  using EL = El<kEl>;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int64_t Q = (int64_t)EL::Q * E;
  Real Vn[EL::C][3];
#pragma unroll
  for (int a = 0; a < EL::C; ++a) {
    const int node = __ldg(conn + a * E + e);
    const Real im = __ldg(inv_mass + node);
#pragma unroll
    for (int d = 0; d < 3; ++d) Vn[a][d] = __ldg(V + d * N + node) * im;
  }
#pragma unroll
  for (int q = 0; q < EL::Q; ++q) {
    const int64_t gq = (int64_t)q * E + e;
    const Real w = __ldg(wj0 + gq);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      Real s = Real(0);
#pragma unroll
      for (int a = 0; a < EL::C; ++a) s += Real(EL::N(a, q)) * Vn[a][d];
      q_val[d * Q + gq] = w * s;
    }
  }
}

// Largest |value| of each tile (FP32 binning: the fixed-point exponent of the
// spreading): one integer maximum of float bit patterns per group of the
// warp's lanes that share a tile.
__device__ __forceinline__ void tile_vmax_update(uint32_t* vmax, uint32_t tile, float v0, float v1,
                                                 float v2) {
  const uint32_t m = __float_as_uint(fmaxf(fabsf(v0), fmaxf(fabsf(v1), fabsf(v2))));
  const unsigned peers = __match_any_sync(__activemask(), tile);
  const uint32_t mx = __reduce_max_sync(peers, m);
  if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(vmax + tile, mx);
}

// Binned copies of the carried values (and, with kVmax, for FP32 plans, the
// per-tile maxima of their magnitudes).  The tile of a binned point: from
// its cell (one structure), or its binning key, read at its original index
// (packed plans, whose cells are their instance's).
template <typename Real, bool kPacked, bool kVmax>
__global__ void k_permute_values(const int32_t* __restrict__ p_idx, int64_t Q,
                                 const Real* __restrict__ q_val, Real* __restrict__ p_val,
                                 const int32_t* __restrict__ p_cell, GridDev g,
                                 const uint32_t* __restrict__ key,
                                 uint32_t* __restrict__ vmax) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Q) return;
  const int32_t gi = __ldg(p_idx + i);
  Real v[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    v[d] = __ldg(q_val + d * Q + gi);
    p_val[d * Q + i] = v[d];
  }
  if constexpr (sizeof(Real) == 4 && kVmax) {
    uint32_t tile;
    if constexpr (kPacked) {
      tile = __ldg(key + gi);
    } else {
      int cx, cy, cz;
      unpack_cell(__ldg(p_cell + i), cx, cy, cz);
      tile = (uint32_t)((cx >> kTileShift) +
                        g.nt[0] * ((cy >> kTileShift) + g.nt[1] * (cz >> kTileShift)));
    }
    tile_vmax_update(vmax, tile, v[0], v[1], v[2]);
  }
}

// The carried values of k_point_values written straight to their binned
// positions (FP32 binning: a point's position is its tile's start plus its
// slot in the tile, both known since the binning), with the per-tile maxima
// of their magnitudes when kVmax: the same values and maxima as
// k_point_values followed by k_permute_values, one pass instead of two.
template <int kEl, bool kVmax>
__global__ void __launch_bounds__(128) k_point_values_binned(
    int E, int64_t N, const int32_t* __restrict__ conn, const float* __restrict__ V,
    const float* __restrict__ inv_mass, const float* __restrict__ wj0,
    const uint32_t* __restrict__ tile, const int32_t* __restrict__ slot,
    const int32_t* __restrict__ start, float* __restrict__ p_val, uint32_t* __restrict__ vmax) {
  using EL = El<kEl>;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int64_t Q = (int64_t)EL::Q * E;
  float Vn[EL::C][3];
#pragma unroll
  for (int a = 0; a < EL::C; ++a) {
    const int node = __ldg(conn + a * E + e);
    const float im = __ldg(inv_mass + node);
#pragma unroll
    for (int d = 0; d < 3; ++d) Vn[a][d] = __ldg(V + d * N + node) * im;
  }
#pragma unroll
  for (int q = 0; q < EL::Q; ++q) {
    const int64_t gq = (int64_t)q * E + e;
    const uint32_t t = __ldg(tile + gq);
    const int64_t i = __ldg(start + t) + __ldg(slot + gq);
    const float w = __ldg(wj0 + gq);
    float v[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float s = 0.f;
#pragma unroll
      for (int a = 0; a < EL::C; ++a) s += float(EL::N(a, q)) * Vn[a][d];
      v[d] = w * s;
      p_val[d * Q + i] = v[d];
    }
    if constexpr (kVmax) tile_vmax_update(vmax, t, v[0], v[1], v[2]);
  }
}

// ---------------------------------------------------------------------------
// radix sort pieces
// ---------------------------------------------------------------------------
// Each CTA takes a chunk of kSortChunk consecutive items; warp w of the CTA
// owns the kWarpItems items [w kWarpItems, (w+1) kWarpItems) of the chunk, 32
// per round.  Lanes holding the same digit in a round are found with a warp
// match, and one leader lane adds their number.
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kWarpItems = kSortItems * 32;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ key,
                                                             int64_t Q, int shift, int nblk,
                                                             int32_t* __restrict__ hist) {
  __shared__ int cnt[256];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  cnt[t] = 0;
  __syncthreads();
  const int64_t b0 = (int64_t)blockIdx.x * kSortChunk + (int64_t)warp * kWarpItems + lane;
  uint32_t k[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = b0 + r * 32;
    k[r] = i < Q ? __ldg(key + i) : 0u;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const bool valid = b0 + r * 32 < Q;
    const int d = valid ? (int)((k[r] >> shift) & 255u) : 256 + lane;  // unique sentinel
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(&cnt[d], __popc(peers));
  }
  __syncthreads();
  hist[t * nblk + blockIdx.x] = cnt[t];
}

// For each digit (one CTA per digit): exclusive scan, in place, of its
// per-block counts hist[d*nblk .. d*nblk + nblk), and the digit total.
__global__ void __launch_bounds__(256) k_digit_scan(int32_t* __restrict__ hist, int nblk,
                                                    int32_t* __restrict__ dtot) {
  __shared__ int tmp[32];
  int32_t* h = hist + (int64_t)blockIdx.x * nblk;
  int carry = 0;
  for (int b0 = 0; b0 < nblk; b0 += 256) {
    const int i = b0 + threadIdx.x;
    const int v = i < nblk ? h[i] : 0;
    int tot;
    const int pre = block_exclusive_scan(v, tmp, tot);
    if (i < nblk) h[i] = carry + pre;
    carry += tot;
  }
  if (threadIdx.x == 0) dtot[blockIdx.x] = carry;
}

// Stable scatter of one digit pass.  Items keep their input order within a
// digit: the chunk's position of digit d is split among the warps in warp
// order (each warp's count of d), and inside a warp among the rounds in order
// and the lanes of a round in lane order.
__global__ void __launch_bounds__(kSortThreads, 3) k_radix_scatter(
    const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin, int64_t Q, int shift,
    int nblk, const int32_t* __restrict__ offs, const int32_t* __restrict__ dtot,
    uint32_t* __restrict__ kout, int32_t* __restrict__ vout) {
  __shared__ int wpos[kSortWarps][256];
  __shared__ int tmp[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < 256 / 32; ++j) wpos[warp][lane + 32 * j] = 0;
  __syncwarp();
  const int64_t b0 = (int64_t)blockIdx.x * kSortChunk + (int64_t)warp * kWarpItems + lane;
  uint32_t k[kSortItems];
  int32_t v[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = b0 + r * 32;
    k[r] = i < Q ? kin[i] : 0u;
    v[r] = i < Q ? vin[i] : 0;
  }
  unsigned peers[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const bool valid = b0 + r * 32 < Q;
    const int d = valid ? (int)((k[r] >> shift) & 255u) : 256 + lane;
    peers[r] = __match_any_sync(0xffffffffu, d);
    if (valid && lane == __ffs(peers[r]) - 1) atomicAdd(&wpos[warp][d], __popc(peers[r]));
  }
  int total;
  const int dstart = block_exclusive_scan(dtot[t], tmp, total);  // start of digit t
  // (block_exclusive_scan ends with a barrier: every warp's counts are in)
  int base = dstart + offs[t * nblk + blockIdx.x];
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    const int c = wpos[w][t];
    wpos[w][t] = base;
    base += c;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const bool valid = b0 + r * 32 < Q;
    if (valid) {
      const int d = (int)((k[r] >> shift) & 255u);
      const int pos = wpos[warp][d] + __popc(peers[r] & lt);
      kout[pos] = k[r];
      vout[pos] = v[r];
    }
    __syncwarp();
    if (valid && lane == __ffs(peers[r]) - 1) wpos[warp][(k[r] >> shift) & 255u] += __popc(peers[r]);
    __syncwarp();
  }
}

// Binning: every point to start[tile] + slot, with its cell, offset, index
// and (optionally) carried value and the per-tile maxima of its magnitude.
template <typename Real>
__global__ void k_bin_scatter(int64_t Q, const uint32_t* __restrict__ tile,
                              const int32_t* __restrict__ slot, const int32_t* __restrict__ start,
                              const int32_t* __restrict__ q_cell, const Real* __restrict__ q_off,
                              const Real* __restrict__ q_val, int32_t* __restrict__ p_cell,
                              Real* __restrict__ p_off, Real* __restrict__ p_val,
                              int32_t* __restrict__ p_idx, bool with_val,
                              uint32_t* __restrict__ vmax) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Q) return;
  const uint32_t t = __ldg(tile + g);
  const int64_t i = __ldg(start + t) + __ldg(slot + g);
  p_idx[i] = (int32_t)g;
  p_cell[i] = __ldg(q_cell + g);
#pragma unroll
  for (int d = 0; d < 3; ++d) p_off[d * Q + i] = __ldg(q_off + d * Q + g);
  if (with_val) {
    Real v[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      v[d] = __ldg(q_val + d * Q + g);
      p_val[d * Q + i] = v[d];
    }
    if constexpr (sizeof(Real) == 4) tile_vmax_update(vmax, t, v[0], v[1], v[2]);
  }
}

__global__ void k_tile_bounds(const uint32_t* __restrict__ key, int64_t Q,
                              int32_t* __restrict__ start, int32_t* __restrict__ end) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Q) return;
  const uint32_t k = key[i] >> kLocalBits;
  if (i == 0 || (key[i - 1] >> kLocalBits) != k) start[k] = (int32_t)i;
  if (i == Q - 1 || (key[i + 1] >> kLocalBits) != k) end[k] = (int32_t)(i + 1);
}

template <typename Real>
__global__ void k_permute(const int32_t* __restrict__ order, int64_t Q,
                          const int32_t* __restrict__ q_cell, const Real* __restrict__ q_off,
                          const Real* __restrict__ q_val, int32_t* __restrict__ p_cell,
                          Real* __restrict__ p_off, Real* __restrict__ p_val,
                          int32_t* __restrict__ p_idx, bool with_val) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Q) return;
  const int32_t g = order[i];
  p_idx[i] = g;
  p_cell[i] = __ldg(q_cell + g);
#pragma unroll
  for (int d = 0; d < 3; ++d) p_off[d * Q + i] = __ldg(q_off + d * Q + g);
  if (with_val) {
#pragma unroll
    for (int d = 0; d < 3; ++d) p_val[d * Q + i] = __ldg(q_val + d * Q + g);
  }
}

template <typename Real>
ib_status points_t(ib_plan* p, const void* xa, const float* off, const void* nodal,
                   cudaStream_t s);

template <>
ib_status points_t<float>(ib_plan* p, const void* xa, const float* off, const void* nodal,
                          cudaStream_t s) {
  PtArgs<float> A;
  A.E = p->E;
  A.N = p->N;
  A.conn = p->conn;
  A.pos.cell = (const int32_t*)xa;
  A.pos.off = off;
  A.pos.N = p->N;
  A.V = (const float*)nodal;
  A.inv_mass = (const float*)p->inv_mass;
  A.wj0 = (const float*)p->wj0;
  A.g = p->grid;
  A.inst = p->n_inst > 1 ? p->inst : nullptr;
  A.elem_inst = p->n_inst > 1 ? p->elem_inst : nullptr;
  A.q_cell = p->q_cell;
  A.q_off = (float*)p->q_off;
  A.q_val = (float*)p->q_val;
  A.key = p->keys[0];
  A.val = p->vals[0];
  A.status = p->dstatus;
  A.count = p->tile_end;
  cudaMemsetAsync(p->tile_start, 0, sizeof(int32_t) * p->ntiles, s);
  cudaMemsetAsync(p->tile_end, 0, sizeof(int32_t) * p->ntiles, s);
  if (p->quad == IB_QUAD_NODAL)
    k_points_nodal<float, true><<<(p->N + 255) / 256, 256, 0, s>>>(A);
  else
    with_elem(p->elem, [&](auto el) {
      constexpr int kE = decltype(el)::value;
      auto k = p->n_inst > 1 ? (nodal ? k_points<float, true, kE, true, true>
                                      : k_points<float, true, kE, true, false>)
                             : (nodal ? k_points<float, true, kE, false, true>
                                      : k_points<float, true, kE, false, false>);
      k<<<(p->E + 127) / 128, 128, 0, s>>>(A);
    });
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

template <>
ib_status points_t<double>(ib_plan* p, const void* xa, const float*, const void* nodal,
                           cudaStream_t s) {
  PtArgs<double> A;
  A.E = p->E;
  A.N = p->N;
  A.conn = p->conn;
  A.pos.x64 = (const double*)xa;
  A.pos.N = p->N;
  for (int d = 0; d < 3; ++d) A.pos.origin[d] = p->grid.origin[d];
  A.pos.inv_h = 1.0 / p->grid.h;
  A.V = (const double*)nodal;
  A.inv_mass = (const double*)p->inv_mass;
  A.wj0 = (const double*)p->wj0;
  A.g = p->grid;
  A.inst = nullptr;  // packed plans are FP32
  A.elem_inst = nullptr;
  A.q_cell = p->q_cell;
  A.q_off = (double*)p->q_off;
  A.q_val = (double*)p->q_val;
  A.key = p->keys[0];
  A.val = p->vals[0];
  A.status = p->dstatus;
  A.count = nullptr;
  if (p->quad == IB_QUAD_NODAL)
    k_points_nodal<double, false><<<(p->N + 255) / 256, 256, 0, s>>>(A);
  else
    with_elem(p->elem, [&](auto el) {
      k_points<double, false, decltype(el)::value, false><<<(p->E + 127) / 128, 128, 0, s>>>(A);
    });
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

}  // namespace

ib_status launch_points(ib_plan* p, const void* xa, const float* off, const void* nodal,
                        int val_kind, cudaStream_t s) {
  if (p->Q == 0) return IB_OK;
  const void* V = val_kind ? nodal : nullptr;
  return p->precision == IB_FP64 ? points_t<double>(p, xa, off, V, s)
                                 : points_t<float>(p, xa, off, V, s);
}

ib_status launch_sort_points(ib_plan* p, bool with_val, cudaStream_t s) {
  const int64_t Q = p->Q;
  if (p->precision != IB_FP64) {  // binning: counts in tile_end, tile_start zero
    if (Q == 0) {  // no points were built: no counts either
      cudaMemsetAsync(p->tile_start, 0, sizeof(int32_t) * p->ntiles, s);
      cudaMemsetAsync(p->tile_end, 0, sizeof(int32_t) * p->ntiles, s);
    }
    if (launch_classify_tiles(p, s) != IB_OK) return IB_ERR_CUDA;  // also the ranges
    if (Q == 0) return IB_OK;
    const int nb = (int)((Q + 255) / 256);
    if (with_val) cudaMemsetAsync(p->tile_vmax, 0, sizeof(uint32_t) * p->ntiles, s);
    k_bin_scatter<float><<<nb, 256, 0, s>>>(Q, p->keys[0], p->vals[0], p->tile_start, p->q_cell,
                                            (const float*)p->q_off, (const float*)p->q_val,
                                            p->p_cell, (float*)p->p_off, (float*)p->p_val,
                                            p->p_idx, with_val, p->tile_vmax);
    return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
  }
  cudaMemsetAsync(p->tile_start, 0, sizeof(int32_t) * p->ntiles, s);
  cudaMemsetAsync(p->tile_end, 0, sizeof(int32_t) * p->ntiles, s);
  if (Q == 0) return launch_classify_tiles(p, s);
  const int bits = sort_key_bits(p->ntiles);
  const int nblk = p->hist_blocks;
  int cur = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<<<nblk, kSortThreads, 0, s>>>(p->keys[cur], Q, shift, nblk, p->hist);
    k_digit_scan<<<256, 256, 0, s>>>(p->hist, nblk, p->digit_tot);
    k_radix_scatter<<<nblk, kSortThreads, 0, s>>>(p->keys[cur], p->vals[cur], Q, shift, nblk,
                                                  p->hist, p->digit_tot, p->keys[cur ^ 1],
                                                  p->vals[cur ^ 1]);
    cur ^= 1;
  }
  const int tb = 256;
  const int nb = (int)((Q + tb - 1) / tb);
  k_tile_bounds<<<nb, tb, 0, s>>>(p->keys[cur], Q, p->tile_start, p->tile_end);
  if (launch_classify_tiles(p, s) != IB_OK) return IB_ERR_CUDA;
  if (p->precision == IB_FP64)
    k_permute<double><<<nb, tb, 0, s>>>(p->vals[cur], Q, p->q_cell, (const double*)p->q_off,
                                        (const double*)p->q_val, p->p_cell, (double*)p->p_off,
                                        (double*)p->p_val, p->p_idx, with_val);
  else
    k_permute<float><<<nb, tb, 0, s>>>(p->vals[cur], Q, p->q_cell, (const float*)p->q_off,
                                       (const float*)p->q_val, p->p_cell, (float*)p->p_off,
                                       (float*)p->p_val, p->p_idx, with_val);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

ib_status launch_point_values(ib_plan* p, const void* nodal, cudaStream_t s, void* q_out) {
  if (p->Q == 0) return IB_OK;
  void* const q = q_out ? q_out : p->q_val;
  if (p->quad == IB_QUAD_NODAL)  // the nodal values are the point values
    return cudaMemcpyAsync(q, nodal, p->rsize * 3 * (size_t)p->N,
                           cudaMemcpyDeviceToDevice, s) == cudaSuccess
               ? IB_OK
               : IB_ERR_CUDA;
  const int g = (p->E + 127) / 128;
  with_elem(p->elem, [&](auto el) {
    constexpr int kE = decltype(el)::value;
    if (p->precision == IB_FP64)
      k_point_values<double, kE><<<g, 128, 0, s>>>(p->E, p->N, p->conn, (const double*)nodal,
                                                   (const double*)p->inv_mass,
                                                   (const double*)p->wj0, (double*)q);
    else
      k_point_values<float, kE><<<g, 128, 0, s>>>(p->E, p->N, p->conn, (const float*)nodal,
                                                  (const float*)p->inv_mass,
                                                  (const float*)p->wj0, (float*)q);
  });
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

ib_status launch_permute_values(ib_plan* p, cudaStream_t s, bool vmax, const void* q_in,
                                void* p_out, bool zero_vmax) {
  if (p->Q == 0) return IB_OK;
  const int nb = (int)((p->Q + 255) / 256);
  const void* const q = q_in ? q_in : p->q_val;
  void* const out = p_out ? p_out : p->p_val;
  if (p->precision == IB_FP64) {
    k_permute_values<double, false, false><<<nb, 256, 0, s>>>(p->p_idx, p->Q, (const double*)q,
                                                       (double*)out, p->p_cell, p->grid,
                                                       nullptr, nullptr);
  } else {
    if (vmax && zero_vmax) cudaMemsetAsync(p->tile_vmax, 0, sizeof(uint32_t) * p->ntiles, s);
    auto permute = p->n_inst > 1 ? (vmax ? k_permute_values<float, true, true>
                                         : k_permute_values<float, true, false>)
                                  : (vmax ? k_permute_values<float, false, true>
                                          : k_permute_values<float, false, false>);
    permute<<<nb, 256, 0, s>>>(p->p_idx, p->Q, (const float*)q, (float*)out, p->p_cell,
                               p->grid, p->keys[0], p->tile_vmax);
  }
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

ib_status launch_binned_values(ib_plan* p, const void* nodal, cudaStream_t s, bool vmax,
                               void* q_tmp, void* p_out) {
  if (p->Q == 0) return IB_OK;
  // the nodal rule's point values are the nodal values: binned directly
  if (p->quad == IB_QUAD_NODAL) return launch_permute_values(p, s, vmax, nodal, p_out);
  if (p->precision == IB_FP64) {  // sorted points: values, then their sorted copy
    const ib_status st = launch_point_values(p, nodal, s, q_tmp);
    return st == IB_OK ? launch_permute_values(p, s, vmax, q_tmp, p_out) : st;
  }
  float* const out = static_cast<float*>(p_out ? p_out : p->p_val);
  if (vmax) cudaMemsetAsync(p->tile_vmax, 0, sizeof(uint32_t) * p->ntiles, s);
  const int g = (p->E + 127) / 128;
  with_elem(p->elem, [&](auto el) {
    constexpr int kE = decltype(el)::value;
    auto k = vmax ? k_point_values_binned<kE, true> : k_point_values_binned<kE, false>;
    k<<<g, 128, 0, s>>>(p->E, p->N, p->conn, (const float*)nodal, (const float*)p->inv_mass,
                        (const float*)p->wj0, p->keys[0], p->vals[0], p->tile_start, out,
                        p->tile_vmax);
  });
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

int binned_values_launches(const ib_plan* p) {
  return p->quad == IB_QUAD_NODAL || p->precision != IB_FP64 ? 1 : 2;
}

int sort_hist_blocks(int64_t Q) { return (int)((Q + kSortChunk - 1) / kSortChunk); }

int sort_key_bits(int ntiles) {
  int bits = 1;
  while ((1 << bits) < ntiles) ++bits;
  return bits + kLocalBits;
}

}  // namespace ibfe
