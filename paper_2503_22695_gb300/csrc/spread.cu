// Spreading of Gauss-point values onto the periodic MAC grid (Section 4.4):
//   f^c(face) = scale * sum_q V_q^c prod_d phi(r_d),   r_d = (chi_q,d - x_face,d)/h,
// with scale = h^-3 for forces (delta_h carries h^-3) and 1 for the adjoint
// of interpolation.
//
// Three kernels over 8^3-cell Eulerian tiles, no global floating-point
// atomics, bitwise reproducible:
//
// k_spread_zero (side stream, concurrent with the push) -- one warp per
//   "far" tile (no points in its 3x3x3 neighbourhood) writes its zeros with
//   16-byte stores: the bulk of the field's HBM traffic overlaps the
//   accumulation work.
// k_spread_push (persistent CTAs pulling tiles from a work counter) -- a
//   tile holding Gauss points accumulates every stencil entry of its own
//   points into a halo'd 12^3 block per component (its points reach two cells
//   beyond the tile; indices stay unwrapped), one component at a time.
//   Points are staged in batches of 256 (one thread per point computes the
//   3x4 kernel weights); point k of a batch goes to warp k mod 8, each warp
//   adding into its own shared-memory copy, one point per step (32 lanes x 2
//   entries = the 64 stencil entries of one component, all distinct faces),
//   steps ordered by __syncwarp.  The eight copies are summed in warp order
//   and the block is written to the work item's scratch block.  A work item is
//   at most 1024 consecutive points of one tile, so densely populated tiles
//   are shared by several CTAs.
// k_spread_merge -- for every "near" tile, each face sums the blocks of its
//   own tile and of the neighbours whose halo covers it (at most two per
//   axis), in a fixed (z, y, x) source order and, within a source tile, in
//   work-item order, and is written once.  Periodic
//   wrap happens only here, through the neighbour-tile index.
#include "ib_device.cuh"

namespace ibfe {
namespace {

constexpr int W = kSpreadWarps;         // 8 warps
constexpr int kThreads = W * 32;
constexpr int kB = 12;                  // halo'd block edge: tile 8 + 2 + 2
constexpr int kBlk = kB * kB * kB;      // 1728 faces per component
constexpr int kSY = kB;                 // shared y stride
constexpr int kSZ = kB * kB + 1;        // shared z stride (145: spreads (dz,dy) over banks)
constexpr int kAcc = kB * kSZ;          // 1740 per warp copy
constexpr int kBatch = kThreads;        // points staged per batch

template <typename Real>
struct SpreadArgs {
  GridDev g;
  int64_t Q;
  const int32_t* tile_start;
  const int32_t* tile_end;
  const int32_t* tile_slot;    // first work item of each tile
  const int32_t* tile_nitems;  // work items of each tile
  const int32_t* tile_near;
  const int32_t* tile_list;    // tile of each work item
  const int32_t* tile_list_near;
  int32_t* counters;      // [0] non-empty tiles, [1] work counter, [3] near tiles
  const int32_t* p_cell;
  const Real* p_off;
  const Real* p_val;
  Real scale;
  Real* scratch;   // [slots][3][12^3]
  Real* f;
};

// staged point: x/y/z weights, value, row origin in the halo'd block
template <typename Real>
struct alignas(16) Staged {
  Real wx[4];
  Real wy[4];
  Real wz[4];
  Real val;
  int org;
  int pad[2];
};

__device__ __forceinline__ int tile_of(int tx, int ty, int tz, const GridDev& g) {
  return wrap_idx(tx, g.nt[0]) + g.nt[0] * (wrap_idx(ty, g.nt[1]) + g.nt[1] * wrap_idx(tz, g.nt[2]));
}

// One lane adds into one face per step; __syncwarp between steps orders the
// read-modify-writes of different lanes to the same face.
template <typename Real>
__device__ __forceinline__ void add_shared(Real* p, Real v) {
  *p += v;
}

// Work item `slot`: points [start + j kChunk, min(end, start + (j+1) kChunk))
// of `tile`, j = slot - first item of the tile.
template <typename Real>
__device__ __forceinline__ void push_tile(const SpreadArgs<Real>& A, int slot, Staged<Real>* stage,
                                          Real* acc, int tid, int lane, int warp, int nt0,
                                          int nt1) {
  const int tile = A.tile_list[slot];
  const int tx = tile % nt0, ty = (tile / nt0) % nt1, tz = tile / (nt0 * nt1);
  const int s = A.tile_start[tile] + (slot - A.tile_slot[tile]) * kChunk;
  const int e = min(A.tile_end[tile], s + kChunk);
  const int x0 = tx * kTile, y0 = ty * kTile, z0 = tz * kTile;
  Real* my = acc + warp * kAcc;
  // this lane's two stencil entries of a component: row (dz, dy), dx = 2h, 2h+1
  const int r = lane >> 1, dz = r >> 2, dy = r & 3, hx = (lane & 1) * 2;
  const int lane_off = dz * kSZ + dy * kSY + hx;

  for (int c = 0; c < 3; ++c) {
    for (int i = tid; i < W * kAcc; i += kThreads) acc[i] = Real(0);
    for (int b0 = s; b0 < e; b0 += kBatch) {
      const int nb = min(kBatch, e - b0);
      __syncthreads();  // previous batch consumed, accumulators zeroed
      if (tid < nb) {
        const int i = b0 + tid;
        int cx, cy, cz;
        unpack_cell(__ldg(A.p_cell + i), cx, cy, cz);
        Staged<Real> st;
        Real th;
        const int bx = cx - x0 + stencil_axis(__ldg(A.p_off + i), c != 0, th) + 2;
        delta_weights(th, st.wx);
        const int by = cy - y0 + stencil_axis(__ldg(A.p_off + A.Q + i), c != 1, th) + 2;
        delta_weights(th, st.wy);
        const int bz = cz - z0 + stencil_axis(__ldg(A.p_off + 2 * A.Q + i), c != 2, th) + 2;
        delta_weights(th, st.wz);
        st.val = __ldg(A.p_val + c * A.Q + i) * A.scale;
        st.org = bz * kSZ + by * kSY + bx;
        stage[tid] = st;
      }
      __syncthreads();
      // software pipelined: the next point's staged values are read while the
      // current point's read-modify-writes are in flight
      int p = warp;
      Real a0 = Real(0), a1 = Real(0);
      int o = 0;
      if (p < nb) {
        const Staged<Real>& st = stage[p];
        const Real w = st.val * st.wz[dz] * st.wy[dy];
        a0 = w * st.wx[hx];
        a1 = w * st.wx[hx + 1];
        o = st.org + lane_off;
      }
      for (; p < nb; p += W) {
        Real b0 = Real(0), b1 = Real(0);
        int ob = 0;
        if (p + W < nb) {
          const Staged<Real>& st = stage[p + W];
          const Real w = st.val * st.wz[dz] * st.wy[dy];
          b0 = w * st.wx[hx];
          b1 = w * st.wx[hx + 1];
          ob = st.org + lane_off;
        }
        add_shared(my + o, a0);
        add_shared(my + o + 1, a1);
        __syncwarp();
        a0 = b0;
        a1 = b1;
        o = ob;
      }
    }
    __syncthreads();
    Real* out = A.scratch + ((int64_t)slot * 3 + c) * kBlk;
    for (int idx = tid; idx < kBlk; idx += kThreads) {
      const int z = idx / (kB * kB), y = (idx / kB) % kB, x = idx % kB;
      const int o = z * kSZ + y * kSY + x;
      Real sum = Real(0);
#pragma unroll
      for (int w = 0; w < W; ++w) sum += acc[w * kAcc + o];
      out[idx] = sum;
    }
    __syncthreads();
  }
}

template <typename Real>
__global__ void __launch_bounds__(kThreads) k_spread_push(SpreadArgs<Real> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Staged<Real>* stage = reinterpret_cast<Staged<Real>*>(smem_raw);
  Real* acc = reinterpret_cast<Real*>(smem_raw + sizeof(Staged<Real>) * kBatch);
  __shared__ int next;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nt0 = A.g.nt[0], nt1 = A.g.nt[1];
  const int count = A.counters[0];
  for (;;) {
    __syncthreads();
    if (tid == 0) next = atomicAdd(A.counters + 1, 1);
    __syncthreads();
    const int k = next;
    if (k >= count) break;
    push_tile(A, k, stage, acc, tid, lane, warp, nt0, nt1);
  }
}

// Far tiles: one warp per tile, 3 components x 64 rows x 2 x 16-byte zeros.
template <typename Real>
__global__ void __launch_bounds__(kThreads) k_spread_zero(SpreadArgs<Real> A) {
  const int lane = threadIdx.x & 31;
  const int tile = blockIdx.x * W + (threadIdx.x >> 5);
  const int nt0 = A.g.nt[0], nt1 = A.g.nt[1];
  if (tile >= nt0 * nt1 * A.g.nt[2] || A.tile_near[tile]) return;
  const int n0 = A.g.n[0], n1 = A.g.n[1];
  const int64_t cells = (int64_t)n0 * n1 * A.g.n[2];
  const int tx = tile % nt0, ty = (tile / nt0) % nt1, tz = tile / (nt0 * nt1);
  const int x0 = tx * kTile, y0 = ty * kTile, z0 = tz * kTile;
  constexpr int kVec = 16 / sizeof(Real);          // reals per 16-byte store
  constexpr int kPerRow = kTile / kVec;
  for (int idx = lane; idx < 3 * 64 * kPerRow; idx += 32) {
    const int c = idx / (64 * kPerRow), r = (idx / kPerRow) % 64, v = idx % kPerRow;
    const int z = r >> 3, y = r & 7;
    Real* row = A.f + c * cells + ((int64_t)(z0 + z) * n1 + (y0 + y)) * n0 + x0;
    reinterpret_cast<float4*>(row)[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Near tiles: fixed-order sum of the halo'd blocks that cover each face.
template <typename Real>
__global__ void __launch_bounds__(kThreads) k_spread_merge(SpreadArgs<Real> A) {
  __shared__ int src_slot[27], src_n[27];
  const int tid = threadIdx.x;
  const int nt0 = A.g.nt[0], nt1 = A.g.nt[1];
  const int n0 = A.g.n[0], n1 = A.g.n[1];
  const int64_t cells = (int64_t)n0 * n1 * A.g.n[2];
  const int count = A.counters[3];
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    const int tile = A.tile_list_near[k];
    const int tx = tile % nt0, ty = (tile / nt0) % nt1, tz = tile / (nt0 * nt1);
    const int x0 = tx * kTile, y0 = ty * kTile, z0 = tz * kTile;
    __syncthreads();
    if (tid < 27) {
      const int a = tid / 9 - 1, b = (tid / 3) % 3 - 1, c = tid % 3 - 1;
      const int nb = tile_of(tx + c, ty + b, tz + a, A.g);
      src_slot[tid] = A.tile_slot[nb];
      src_n[tid] = A.tile_nitems[nb];
    }
    __syncthreads();
    for (int idx = tid; idx < 3 * 512; idx += kThreads) {
      const int c = idx >> 9, rr = idx & 511;
      const int z = rr >> 6, y = (rr >> 3) & 7, x = rr & 7;
      // source offsets along each axis: own tile, and the neighbour whose halo
      // reaches this face (faces 0..1 from below, 6..7 from above)
      const int lx = x <= 1 ? -1 : 0, ly = y <= 1 ? -1 : 0, lz = z <= 1 ? -1 : 0;
      const int hx = x >= 6 ? 1 : 0, hy = y >= 6 ? 1 : 0, hz = z >= 6 ? 1 : 0;
      Real sum = Real(0);
      for (int oz = lz; oz <= hz; ++oz)
        for (int oy = ly; oy <= hy; ++oy)
          for (int ox = lx; ox <= hx; ++ox) {
            const int si = (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1);
            const int sl = src_slot[si], ns = src_n[si];
            const int bx = x - ox * kTile + 2, by = y - oy * kTile + 2, bz = z - oz * kTile + 2;
            for (int j = 0; j < ns; ++j)  // the tile's work items in order
              sum += A.scratch[((int64_t)(sl + j) * 3 + c) * kBlk + (bz * kB + by) * kB + bx];
          }
      A.f[c * cells + ((int64_t)(z0 + z) * n1 + (y0 + y)) * n0 + (x0 + x)] = sum;
    }
  }
}

template <typename Real>
ib_status spread_t(ib_plan* p, double scale, void* f, cudaStream_t s) {
  SpreadArgs<Real> A;
  A.g = p->grid;
  A.Q = p->Q;
  A.tile_start = p->tile_start;
  A.tile_end = p->tile_end;
  A.tile_slot = p->tile_slot;
  A.tile_nitems = p->tile_nonempty;
  A.tile_near = p->tile_near;
  A.tile_list = p->tile_list;
  A.tile_list_near = p->tile_list_near;
  A.counters = p->tile_counters;
  A.p_cell = p->p_cell;
  A.p_off = (const Real*)p->p_off;
  A.p_val = (const Real*)p->p_val;
  A.scale = (Real)scale;
  A.scratch = (Real*)p->spread_scratch;
  A.f = (Real*)f;
  const size_t smem = sizeof(Staged<Real>) * kBatch + sizeof(Real) * W * kAcc;
  cudaMemsetAsync(p->tile_counters + 1, 0, sizeof(int32_t), s);
  // far-tile zeros on the side stream, concurrent with the push
  cudaEventRecord(p->ev_fork, s);
  cudaStreamWaitEvent(p->side, p->ev_fork, 0);
  k_spread_zero<Real><<<(p->ntiles + W - 1) / W, kThreads, 0, p->side>>>(A);
  cudaEventRecord(p->ev_join, p->side);
  const int push_ctas = min(p->ntiles, p->push_ctas);
  k_spread_push<Real><<<push_ctas, kThreads, smem, s>>>(A);
  const int merge_ctas = min(p->ntiles, p->merge_ctas);
  k_spread_merge<Real><<<merge_ctas, kThreads, 0, s>>>(A);
  cudaStreamWaitEvent(s, p->ev_join, 0);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

}  // namespace

size_t spread_smem_bytes(int precision) {
  return precision == IB_FP64 ? sizeof(Staged<double>) * kBatch + sizeof(double) * W * kAcc
                              : sizeof(Staged<float>) * kBatch + sizeof(float) * W * kAcc;
}

size_t spread_scratch_bytes(int precision, int64_t slots) {
  return (size_t)slots * 3 * kBlk * (precision == IB_FP64 ? sizeof(double) : sizeof(float));
}

ib_status spread_prepare(ib_plan* p) {
  const int smem = (int)spread_smem_bytes(p->precision);
  int dev = 0, sms = 0, per_sm = 0, per_sm_merge = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return IB_ERR_CUDA;
  cudaError_t e;
  if (p->precision == IB_FP64) {
    e = cudaFuncSetAttribute(k_spread_push<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread_push<double>, kThreads, smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_merge, k_spread_merge<double>, kThreads, 0);
  } else {
    e = cudaFuncSetAttribute(k_spread_push<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread_push<float>, kThreads, smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_merge, k_spread_merge<float>, kThreads, 0);
  }
  if (e != cudaSuccess || per_sm < 1 || per_sm_merge < 1) return IB_ERR_CUDA;
  p->sm_count = sms;
  p->push_ctas = sms * per_sm;
  p->merge_ctas = sms * per_sm_merge;
  return IB_OK;
}

int spread_launches() { return 3; }

ib_status launch_spread(ib_plan* p, double scale, void* f, cudaStream_t s) {
  return p->precision == IB_FP64 ? spread_t<double>(p, scale, f, s)
                                 : spread_t<float>(p, scale, f, s);
}

}  // namespace ibfe
