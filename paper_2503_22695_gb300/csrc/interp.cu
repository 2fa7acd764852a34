// Interpolation of a MAC field at the Gauss points (Section 4.4):
//   U^IB_q^c = sum_faces u^c(face) prod_d phi(r_d)      (h^3 delta_h = prod phi)
// and the position derivatives of the same sums, used by the adjoints:
//   d/dchi_d sum_faces u^c prod phi = h^-1 sum_faces u^c phi'(r_d) prod_{d'!=d} phi(r_d').
//
// Persistent CTAs pull work items (at most 1024 consecutive points of one
// 8^3-cell Eulerian tile) from a counter.  The tile's halo'd 12^3 block of
// each velocity component (faces local -2..9 per axis, every face any of its
// points can reach) is staged in shared memory and one thread per point
// evaluates its three 4x4x4 stencils from there.
//
// FP32 plans stage the block with the Tensor Memory Accelerator: one thread
// issues a 4-D tiled bulk copy (x 16 from face -4 so that the start is
// 16-byte aligned, y 12, z 12, all 3 components) of the next item into a
// dense buffer while the CTA evaluates the current item; the dense box is
// then rewritten into the padded block layout (z stride 145, odd in banks)
// that keeps the per-thread stencil gathers spread over the banks.  Tiles
// whose halo crosses the periodic boundary are staged with cp.async and
// explicit wrapping instead.  FP64 plans use the cp.async path throughout,
// one item ahead in a double buffer.
// Results are written at the point's original index gq = q*E + e for the
// element-wise projection that follows.
//
// Modes (the projection to the nodes applies the points' w_q j0 to a)
//   0: a[c][gq] = vscale * S_c                             (S_c = sum u^c prod phi)
//   1: a as mode 0, and b[d][gq] = gscale * sum_c val_c dS_c/dr_d
//   2: b only.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "ib_device.cuh"

namespace ibfe {
namespace {

constexpr int kThreads = 256;
constexpr int kB = 12;
constexpr int kSY = kB;
constexpr int kSZ = kB * kB + 1;
constexpr int kComp = kB * kSZ;  // 1740

template <typename Real>
struct InterpArgs {
  GridDev g;
  const InstDev* inst;       // packed plans: instance table, else null
  const int32_t* tile_inst;  // packed plans: instance of each tile
  const GridCall* calls;     // packed plans: each instance's u, vscale, gscale, else null
  const CUtensorMap* tmaps;  // packed plans: each instance's tensor map of u (FP32)
  int64_t Q;
  const int32_t* tile_start;
  const int32_t* tile_end;
  const int32_t* tile_slot;  // first work item of each tile
  const int32_t* tile_list;  // tile of each work item
  int32_t* counters;      // [0] work items, [2] the values-only mode's work counter
  int32_t* work;          // the gradient modes' work counter (zero at launch)
  const int32_t* p_cell;
  const Real* p_off;
  const Real* p_val;
  const int32_t* p_idx;
  int chunk;               // points per work item
  const Real* u;
  Real vscale, gscale;
  Real* out_a;
  Real* out_b;
  int* status;
  int use_tma;            // FP32: interior tiles staged by the tensor map
};

// The call's field and scalars for the structure `inst` (packed plans: its
// row of the call table; a plan of one structure: the arguments).
template <bool kPacked, typename Real>
__device__ __forceinline__ const Real* call_u(const InterpArgs<Real>& A, int inst) {
  if constexpr (kPacked) return static_cast<const Real*>(A.calls[inst].field);
  return A.u;
}
template <bool kPacked, typename Real>
__device__ __forceinline__ void call_scales(const InterpArgs<Real>& A, int inst, Real& vs,
                                            Real& gs) {
  if constexpr (kPacked) {
    vs = (Real)__ldg(&A.calls[inst].s0);
    gs = (Real)__ldg(&A.calls[inst].s1);
  } else {
    vs = A.vscale;
    gs = A.gscale;
  }
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copy the halo'd 12^3 block of each velocity component around the tile of
// work item `slot` (faces local -2..9, periodically wrapped) into `ub`,
// asynchronously: 16 lanes per 12-face x-row, 16 rows per pass.
template <bool kPacked, typename Real>
__device__ __forceinline__ void stage_block(const InterpArgs<Real>& A, int slot, Real* ub, int tid) {
  const int tile = A.tile_list[slot];
  const TileGeo geo = tile_geo<kPacked>(A.g, A.inst, A.tile_inst, tile);
  int tx, ty, tz;
  tile_coords(geo, tile, tx, ty, tz);
  const int n0 = geo.n[0], n1 = geo.n[1], n2 = geo.n[2];
  const int64_t cells = (int64_t)n0 * n1 * n2;
  const Real* const u = call_u<kPacked>(A, geo.inst);
  const int x0 = tx * kTile, y0 = ty * kTile, z0 = tz * kTile;
  const int bx = tid & 15;
  if (bx >= kB) return;
  for (int row = tid >> 4; row < 3 * kB * kB; row += kThreads / 16) {
    const int c = row / (kB * kB), bz = (row / kB) % kB, by = row % kB;
    int gx = x0 - 2 + bx, gy = y0 - 2 + by, gz = z0 - 2 + bz;  // within one period
    gx += gx < 0 ? n0 : (gx >= n0 ? -n0 : 0);
    gy += gy < 0 ? n1 : (gy >= n1 ? -n1 : 0);
    gz += gz < 0 ? n2 : (gz >= n2 ? -n2 : 0);
    Real* dst = ub + c * kComp + bz * kSZ + by * kSY + bx;
    const Real* src = u + c * cells + ((int64_t)gz * n1 + gy) * n0 + gx;
    if (sizeof(Real) == 4) {
      cp_async4(dst, src);
    } else {
      *dst = *src;
    }
  }
}

template <typename Real, int MODE, bool kPacked>
__device__ __forceinline__ void interp_points(const InterpArgs<Real>& A, int slot, const Real* ub,
                                              int tid);
template <typename Real, int MODE>
__device__ __forceinline__ void interp_one(const InterpArgs<Real>& A, const Real* ub,
                                           const int lc[3], const Real off[3], int gq,
                                           const Real val[3], Real vs, Real gs);

// Persistent CTAs, two-stage pipeline: the velocity block of the next work
// item is fetched while the points of the current one are evaluated.
// The work counter of a call: slot 2 for the values-only mode (never given
// another), the call's own slot for the gradient modes.
template <int MODE, typename Real>
__device__ __forceinline__ int32_t* work_counter(const InterpArgs<Real>& A) {
  return MODE == 0 ? A.counters + 2 : A.work;
}

template <typename Real, int MODE, bool kPacked>
__global__ void __launch_bounds__(kThreads) k_interp_tile(InterpArgs<Real> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* const buf0 = reinterpret_cast<Real*>(smem_raw);
  __shared__ int next;
  const int tid = threadIdx.x;
  const int count = A.counters[0];
  if (tid == 0) next = atomicAdd(work_counter<MODE>(A), 1);
  __syncthreads();
  int cur = next;
  if (cur < count) stage_block<kPacked>(A, cur, buf0, tid);
  cp_async_commit();
  int b = 0;
  while (cur < count) {
    __syncthreads();
    if (tid == 0) next = atomicAdd(work_counter<MODE>(A), 1);
    __syncthreads();
    const int nxt = next;
    if (nxt < count) stage_block<kPacked>(A, nxt, buf0 + (b ^ 1) * 3 * kComp, tid);
    cp_async_commit();
    cp_async_wait_group<1>();  // the current item's block has landed
    __syncthreads();
    interp_points<Real, MODE, kPacked>(A, cur, buf0 + b * 3 * kComp, tid);
    cur = nxt;
    b ^= 1;
  }
  cp_async_wait_group<0>();
}

// ---------------------------------------------------------------------------
// TMA path (FP32)
// ---------------------------------------------------------------------------
constexpr int kDX = 16;                             // dense box x extent (faces -4..11)
constexpr int kDenseFloats = 3 * kB * kB * kDX;     // 6912
constexpr uint32_t kDenseBytes = kDenseFloats * 4;  // 27648 = one box, the tx count
constexpr int kTmaAlign = 1024;
constexpr long long kWaitCycles = 2000000000LL;     // about one second at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bounded wait for phase `parity` of an mbarrier; false after `budget`
// cycles (about 1 s by default).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          long long budget = kWaitCycles) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > budget) return false;
    __nanosleep(64);
  }
}

__device__ __forceinline__ bool tile_interior(const TileGeo& g, int tile) {
  int tx, ty, tz;
  tile_coords(g, tile, tx, ty, tz);
  return tx > 0 && ty > 0 && tz > 0 && tx < g.nt[0] - 1 && ty < g.nt[1] - 1 && tz < g.nt[2] - 1;
}

// Thread 0: bulk tensor copy of the box around the tile of item `slot`.
// Only interior tiles: x start 8 tx - 4 >= 0 is a multiple of 4 floats (16
// bytes) and the box lies inside the grid.  A map in global memory (packed
// plans; written by a copy before the launch) is first acquired by the
// tensor-map proxy.
__device__ __forceinline__ void issue_box(const CUtensorMap* tmap, bool global_map,
                                          const TileGeo& g, int tile, uint32_t dense,
                                          uint32_t bar) {
  if (global_map)
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;\n" ::"l"(
                     reinterpret_cast<uint64_t>(tmap))
                 : "memory");
  int tx, ty, tz;
  tile_coords(g, tile, tx, ty, tz);
  const int x = tx * kTile - 4, y = ty * kTile - 2, z = tz * kTile - 2, c = 0;
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
               "r"(kDenseBytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(dense),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(c), "r"(bar)
      : "memory");
}

// dense box (faces x -4..11) -> padded block (faces x -2..9), one x-row per thread
__device__ __forceinline__ void relayout(const float* __restrict__ dense, float* __restrict__ ub,
                                         int tid) {
  for (int row = tid; row < 3 * kB * kB; row += kThreads) {
    const int c = row / (kB * kB), zy = row % (kB * kB), z = zy / kB, y = zy % kB;
    const float4* src = reinterpret_cast<const float4*>(dense + row * kDX);
    const float4 a = src[0], b = src[1], d = src[2], e = src[3];
    float* dst = ub + c * kComp + z * kSZ + y * kSY;
    dst[0] = a.z;  dst[1] = a.w;
    dst[2] = b.x;  dst[3] = b.y;  dst[4] = b.z;  dst[5] = b.w;
    dst[6] = d.x;  dst[7] = d.y;  dst[8] = d.z;  dst[9] = d.w;
    dst[10] = e.x; dst[11] = e.y;
  }
}


// Binned points arrive in no particular order inside a tile; threads of a
// warp then often gather the same bank.  The item's points are ordered by
// cell of the tile (a counting sort over the 512 cells; points of one cell in
// any order, which changes no result), so a warp covers a run of neighbouring
// cells, as sorted points would.  Their data are read once, coalesced, in
// binned order and stored in that cell order in shared memory, so the
// evaluation reads them with plain shared loads.
template <int MODE>
struct PtStage {
  float off[3][kChunk];
  float val[MODE != 0 ? 3 : 1][MODE != 0 ? kChunk : 1];
  int idx[kChunk];
  short lc[kChunk];  // local cell: x + 8 y + 64 z
};

template <int MODE, bool kPacked>
__device__ __forceinline__ int local_cell_stage(const InterpArgs<float>& A, int slot, int* cnt,
                                                PtStage<MODE>& P, int* tmp, int tid) {
  const int tile = A.tile_list[slot];
  const int s = A.tile_start[tile] + (slot - A.tile_slot[tile]) * A.chunk;
  const int e = min(A.tile_end[tile], s + A.chunk);
  int tx, ty, tz;
  tile_coords(tile_geo<kPacked>(A.g, A.inst, A.tile_inst, tile), tile, tx, ty, tz);
  const int x0 = tx * kTile, y0 = ty * kTile, z0 = tz * kTile;
  cnt[tid] = 0;
  cnt[tid + kThreads] = 0;
  __syncthreads();
  // every global load of the item's points is issued here, before the
  // counting sort's barriers; only the stores wait for the sorted positions
  constexpr int kPer = kChunk / kThreads;
  int cell[kPer], rank[kPer], idx[kPer];
  float off[kPer][3], val[MODE != 0 ? kPer : 1][3];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int i = s + tid + k * kThreads;
    if (i < e) {
      const int32_t pc = __ldg(A.p_cell + i);
#pragma unroll
      for (int d = 0; d < 3; ++d) off[k][d] = __ldg(A.p_off + d * A.Q + i);
      if (MODE != 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) val[k][c] = __ldg(A.p_val + c * A.Q + i);
      }
      idx[k] = __ldg(A.p_idx + i);
      int cx, cy, cz;
      unpack_cell(pc, cx, cy, cz);
      cell[k] = ((cz - z0) * kTile + (cy - y0)) * kTile + (cx - x0);
      rank[k] = atomicAdd(cnt + cell[k], 1);
    }
  }
  __syncthreads();
  const int c0 = cnt[2 * tid], c1 = cnt[2 * tid + 1];
  int tot;
  const int pre = block_exclusive_scan(c0 + c1, tmp, tot);
  cnt[2 * tid] = pre;
  cnt[2 * tid + 1] = pre + c0;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int i = s + tid + k * kThreads;
    if (i < e) {
      const int q = cnt[cell[k]] + rank[k];
#pragma unroll
      for (int d = 0; d < 3; ++d) P.off[d][q] = off[k][d];
      if (MODE != 0) {
#pragma unroll
        for (int c = 0; c < 3; ++c) P.val[c][q] = val[k][c];
      }
      P.idx[q] = idx[k];
      P.lc[q] = (short)cell[k];
    }
  }
  return e - s;
}

// Per item: wait for its box (or stage it with cp.async), rewrite it into the
// padded block, issue the next item's box, evaluate the points
// (shared memory holds 3 CTAs per SM in mode 0 and 2 in the gradient modes;
// the register bounds follow)
template <int MODE, bool kPacked>
__global__ void __launch_bounds__(kThreads, MODE == 0 ? 3 : 2)
    k_interp_tma(const __grid_constant__ CUtensorMap tmap, InterpArgs<float> A) {
  extern __shared__ unsigned char smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(smem_raw) + kTmaAlign - 1) &
                         ~static_cast<uintptr_t>(kTmaAlign - 1);
  float* const dense = reinterpret_cast<float*>(base);
  float* const ub = dense + kDenseFloats;
  __shared__ __align__(8) uint64_t bar_store;
  __shared__ int next, abort_flag;
  __shared__ int cnt[2 * kThreads], tmp[32];
  PtStage<MODE>& pts = *reinterpret_cast<PtStage<MODE>*>(ub + 3 * kComp);
  const int tid = threadIdx.x;
  const int count = A.counters[0];
  const uint32_t bar = smem_u32(&bar_store), dense_s = smem_u32(dense);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag = 0;
    next = atomicAdd(work_counter<MODE>(A), 1);
  }
  __syncthreads();
  int cur = next;
  // the tile of an item, its structure's grid and tensor map
  auto geo_of = [&](int item) {
    return tile_geo<kPacked>(A.g, A.inst, A.tile_inst, A.tile_list[item]);
  };
  auto map_of = [&](const TileGeo& g) { return kPacked ? A.tmaps + g.inst : &tmap; };
  // only the instance of the current item is carried across iterations
  int cinst = 0;
  bool cur_tma = false;
  if (cur < count) {
    const TileGeo g = geo_of(cur);
    cinst = g.inst;
    cur_tma = tile_interior(g, A.tile_list[cur]);
    if (tid == 0 && cur_tma)
      issue_box(map_of(g), kPacked, g, A.tile_list[cur], dense_s, bar);
  }
  uint32_t parity = 0;
  while (cur < count) {
    const int np = local_cell_stage<MODE, kPacked>(A, cur, cnt, pts, tmp, tid);  // box in flight
    // thread 0 alone waits (bounded) for the box; the barrier below hands
    // the landed data and the outcome to the CTA
    if (cur_tma) {
      if (tid == 0 && !mbar_wait(bar, parity)) abort_flag = 1;
    } else {
      stage_block<kPacked>(A, cur, ub, tid);
      cp_async_commit();
      cp_async_wait_group<0>();
    }
    if (tid == 0) next = atomicAdd(work_counter<MODE>(A), 1);
    __syncthreads();  // box landed everywhere; next item known
    if (abort_flag) break;
    if (cur_tma) {
      parity ^= 1;
      relayout(dense, ub, tid);
      __syncthreads();  // dense free, padded block complete
    }
    const int nxt = next;
    int ninst = cinst;
    bool nxt_tma = false;
    if (nxt < count) {
      const TileGeo g = geo_of(nxt);
      ninst = g.inst;
      nxt_tma = tile_interior(g, A.tile_list[nxt]);
      if (tid == 0 && nxt_tma)
        issue_box(map_of(g), kPacked, g, A.tile_list[nxt], dense_s, bar);
    }
    float vs, gs;
    call_scales<kPacked>(A, cinst, vs, gs);
    // the points in cell order, from the staged copy
    for (int j = tid; j < np; j += kThreads) {
      const int c = pts.lc[j];
      const int lc[3] = {c & (kTile - 1), (c >> kTileShift) & (kTile - 1), c >> (2 * kTileShift)};
      const float off[3] = {pts.off[0][j], pts.off[1][j], pts.off[2][j]};
      float val[3] = {0.f, 0.f, 0.f};
      if (MODE != 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) val[k] = pts.val[k][j];
      }
      interp_one<float, MODE>(A, ub, lc, off, pts.idx[j], val, vs, gs);
    }
    __syncthreads();  // padded block free; `next` consumed
    cur = nxt;
    cinst = ninst;
    cur_tma = nxt_tma;
  }
  if (abort_flag && tid == 0) {
    atomicOr(A.status, kStatTimeout);
    mbar_wait(bar, parity);  // let a late box land before the CTA exits (bounded)
  }
}

// One point: the three stencil sums at local cell lc with offsets off, and
// (MODE != 0) their position derivatives weighted by val; results written at
// the point's original index gq.
template <typename Real, int MODE>
__device__ __forceinline__ void interp_one(const InterpArgs<Real>& A, const Real* ub,
                                           const int lc[3], const Real off[3], int gq,
                                           const Real val[3], Real vs, Real gs) {
  // weights for both staggerings per axis: [d][0] = s 0, [d][1] = s 1/2
  Real w[3][2][4], dw[3][2][4];
  int b[3][2];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      Real th;
      b[d][hf] = lc[d] + stencil_axis(off[d], hf == 1, th) + 2;
      if (MODE == 0)
        delta_weights(th, w[d][hf]);
      else
        delta_weights_d(th, w[d][hf], dw[d][hf]);
    }
  Real S[3];
  Real grad[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int hx = c != 0, hy = c != 1, hz = c != 2;
    const Real* uc = ub + c * kComp + b[2][hz] * kSZ + b[1][hy] * kSY + b[0][hx];
    Real tot = Real(0), gx = Real(0), gy = Real(0), gz = Real(0);
#pragma unroll
    for (int kz = 0; kz < 4; ++kz) {
      Real py = Real(0), pdy = Real(0), pdx = Real(0);
#pragma unroll
      for (int ky = 0; ky < 4; ++ky) {
        const Real* row = uc + kz * kSZ + ky * kSY;
        Real rx = Real(0), rdx = Real(0);
#pragma unroll
        for (int kx = 0; kx < 4; ++kx) {
          const Real v = row[kx];
          rx += w[0][hx][kx] * v;
          if (MODE != 0) rdx += dw[0][hx][kx] * v;
        }
        py += w[1][hy][ky] * rx;
        if (MODE != 0) {
          pdy += dw[1][hy][ky] * rx;
          pdx += w[1][hy][ky] * rdx;
        }
      }
      tot += w[2][hz][kz] * py;
      if (MODE != 0) {
        gz += dw[2][hz][kz] * py;
        gy += w[2][hz][kz] * pdy;
        gx += w[2][hz][kz] * pdx;
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
#pragma unroll
    for (int c = 0; c < 3; ++c) A.out_a[c * A.Q + gq] = vs * S[c];
  }
  if (MODE != 0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) A.out_b[d * A.Q + gq] = gs * grad[d];
  }
}

// The points of work item `slot`, read from global memory in binned order.
template <typename Real, int MODE, bool kPacked>
__device__ __forceinline__ void interp_points(const InterpArgs<Real>& A, int slot, const Real* ub,
                                              int tid) {
  const int tile = A.tile_list[slot];
  const int s = A.tile_start[tile] + (slot - A.tile_slot[tile]) * A.chunk;
  const int e = min(A.tile_end[tile], s + A.chunk);
  const TileGeo geo = tile_geo<kPacked>(A.g, A.inst, A.tile_inst, tile);
  int tx, ty, tz;
  tile_coords(geo, tile, tx, ty, tz);
  const int x0 = tx * kTile, y0 = ty * kTile, z0 = tz * kTile;
  Real vs, gs;
  call_scales<kPacked>(A, geo.inst, vs, gs);
  for (int i = s + tid; i < e; i += kThreads) {
    int cx, cy, cz;
    unpack_cell(__ldg(A.p_cell + i), cx, cy, cz);
    const int lc[3] = {cx - x0, cy - y0, cz - z0};
    const Real off[3] = {__ldg(A.p_off + i), __ldg(A.p_off + A.Q + i),
                         __ldg(A.p_off + 2 * A.Q + i)};
    Real val[3] = {Real(0), Real(0), Real(0)};
    if (MODE != 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) val[c] = __ldg(A.p_val + c * A.Q + i);
    }
    interp_one<Real, MODE>(A, ub, lc, off, __ldg(A.p_idx + i), val, vs, gs);
  }
}

template <typename Real>
size_t smem_bytes() {
  return sizeof(Real) * 2 * 3 * kComp;
}

template <int MODE>
constexpr size_t tma_smem() {
  return kTmaAlign + kDenseBytes + sizeof(float) * 3 * kComp + sizeof(PtStage<MODE>);
}

// cuTensorMapEncodeTiled from the driver, looked up once.
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(f);
  });
  return fn;
}

// Tensor map of the velocity field u [3][n2][n1][n0] (float), box 16 x 12 x 12 x 3.
// False when the driver function is missing or u is not 16-byte aligned.
bool make_velocity_map(const int n[3], const void* u, CUtensorMap* m) {
  const EncodeTiled enc = encode_tiled();
  if (!enc || (reinterpret_cast<uintptr_t>(u) & 15) != 0) return false;
  const cuuint64_t n0 = n[0], n1 = n[1], n2 = n[2];
  const cuuint64_t dims[4] = {n0, n1, n2, 3};
  const cuuint64_t strides[3] = {n0 * 4, n0 * n1 * 4, n0 * n1 * n2 * 4};
  const cuuint32_t box[4] = {kDX, kB, kB, 3};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(u), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename Real>
ib_status interp_t(ib_plan* p, const void* u, int mode, double vscale, double gscale,
                   cudaStream_t s, const GridCall* calls, const CUtensorMap* tmaps,
                   const InterpIO* io) {
  if (p->Q == 0) return IB_OK;
  // work-counter slots free for the interpolation (0, 1, 3 and 6 are the
  // work count, the push's counter, the near count and the force's counter)
  if (io && (mode == 0 || (io->counter != 2 && io->counter != 4 && io->counter != 5 &&
                           io->counter != 7)))
    return IB_ERR_INVALID_ARG;
  if ((p->n_inst > 1) != (calls != nullptr)) return IB_ERR_INVALID_ARG;
  InterpArgs<Real> A;
  A.g = p->grid;
  A.inst = p->n_inst > 1 ? p->inst : nullptr;
  A.tile_inst = p->n_inst > 1 ? p->tile_inst : nullptr;
  A.calls = calls;
  A.tmaps = tmaps;
  A.Q = p->Q;
  A.tile_start = p->tile_start;
  A.tile_end = p->tile_end;
  A.tile_slot = p->tile_slot;
  A.tile_list = p->tile_list;
  A.counters = p->tile_counters;
  A.work = p->tile_counters + (io ? io->counter : 2);
  A.p_cell = p->p_cell;
  A.p_off = (const Real*)p->p_off;
  A.p_val = (const Real*)(io && io->vals ? io->vals : p->p_val);
  A.p_idx = p->p_idx;
  A.chunk = p->chunk;
  // the projection weight w_q j0 of a Gauss point; none for the nodal rule
  A.u = (const Real*)u;
  A.vscale = (Real)vscale;
  A.gscale = (Real)gscale;
  A.out_a = (Real*)(io && io->out_a ? io->out_a : p->gq_a);
  A.out_b = (Real*)(io && io->out_b ? io->out_b : p->gq_b);
  A.status = p->dstatus;
  A.use_tma = 0;
  // persistent grid: the occupancy maximum, capped by the plan's tuning
  const int cap_ctas = p->interp_per_sm * p->sm_count;
  auto cap = [cap_ctas](int ctas) { return ctas < cap_ctas ? ctas : cap_ctas; };
  const size_t smem = smem_bytes<Real>();
  cudaMemsetAsync(A.work, 0, sizeof(int32_t), s);
  const bool packed = p->n_inst > 1;
  if constexpr (sizeof(Real) == 4) {
    // packed plans: the instances' maps in device memory (this one unused)
    CUtensorMap tmap = {};
    if (p->interp_tma && (packed ? tmaps != nullptr : make_velocity_map(p->grid.n, u, &tmap))) {
      A.use_tma = 1;
      auto run = [&](auto kernel, int ctas, size_t smem_b) {
        kernel<<<cap(ctas), kThreads, smem_b, s>>>(tmap, A);
      };
      if (mode == 0)
        run(packed ? k_interp_tma<0, true> : k_interp_tma<0, false>, p->interp_ctas_tma[0],
            tma_smem<0>());
      else if (mode == 1)
        run(packed ? k_interp_tma<1, true> : k_interp_tma<1, false>, p->interp_ctas_tma[1],
            tma_smem<1>());
      else
        run(packed ? k_interp_tma<2, true> : k_interp_tma<2, false>, p->interp_ctas_tma[2],
            tma_smem<2>());
      return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
    }
  }
  auto run = [&](auto kernel, int ctas) { kernel<<<cap(ctas), kThreads, smem, s>>>(A); };
  if (mode == 0)
    run(packed ? k_interp_tile<Real, 0, true> : k_interp_tile<Real, 0, false>, p->interp_ctas[0]);
  else if (mode == 1)
    run(packed ? k_interp_tile<Real, 1, true> : k_interp_tile<Real, 1, false>, p->interp_ctas[1]);
  else
    run(packed ? k_interp_tile<Real, 2, true> : k_interp_tile<Real, 2, false>, p->interp_ctas[2]);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

// Dynamic shared memory opt-in of a kernel and its CTAs per SM (0 on error).
template <typename K>
int opt_in(K kernel, size_t smem) {
  int n = 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kThreads, smem) != cudaSuccess)
    return 0;
  return n;
}

template <typename Real>
ib_status prepare_t(ib_plan* p) {
  // both variants of each kernel (one structure, packed); the persistent
  // grids take the smaller occupancy of the two
  const size_t smem = smem_bytes<Real>();
  const int per_sm[3] = {
      std::min(opt_in(k_interp_tile<Real, 0, false>, smem), opt_in(k_interp_tile<Real, 0, true>, smem)),
      std::min(opt_in(k_interp_tile<Real, 1, false>, smem), opt_in(k_interp_tile<Real, 1, true>, smem)),
      std::min(opt_in(k_interp_tile<Real, 2, false>, smem), opt_in(k_interp_tile<Real, 2, true>, smem))};
  for (int m = 0; m < 3; ++m) {
    if (per_sm[m] < 1) return IB_ERR_CUDA;
    p->interp_ctas[m] = p->sm_count * per_sm[m];
  }
  p->interp_tma = 0;
  if constexpr (sizeof(Real) == 4) {
    if (encode_tiled()) {
      const int tma_sm[3] = {
          std::min(opt_in(k_interp_tma<0, false>, tma_smem<0>()), opt_in(k_interp_tma<0, true>, tma_smem<0>())),
          std::min(opt_in(k_interp_tma<1, false>, tma_smem<1>()), opt_in(k_interp_tma<1, true>, tma_smem<1>())),
          std::min(opt_in(k_interp_tma<2, false>, tma_smem<2>()), opt_in(k_interp_tma<2, true>, tma_smem<2>()))};
      if (tma_sm[0] > 0 && tma_sm[1] > 0 && tma_sm[2] > 0) {
        for (int m = 0; m < 3; ++m) p->interp_ctas_tma[m] = p->sm_count * tma_sm[m];
        p->interp_tma = 1;
      }
    }
  }
  cudaGetLastError();
  return IB_OK;
}

}  // namespace

// Diagnostic of the failure path of the bounded wait: one thread arms an
// mbarrier for 16 bytes of transaction that no copy will deliver, so the wait
// gives up after `budget` cycles and the kernel latches the timeout bit, as the
// interpolation does when a TMA box never lands.  No copy is in flight, so
// nothing is left to wait for on exit.
__global__ void k_wait_probe(int* status, long long budget) {
  __shared__ __align__(8) uint64_t bar_s;
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bar_s);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(16)
                 : "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(bar, 0, budget)) set_status(status, kStatTimeout);
}

ib_status launch_wait_probe(int* status, double ms, cudaStream_t s) {
  int dev = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess)
    return IB_ERR_CUDA;
  k_wait_probe<<<1, 32, 0, s>>>(status, (long long)(ms * khz));
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

ib_status interp_prepare(ib_plan* p) {
  return p->precision == IB_FP64 ? prepare_t<double>(p) : prepare_t<float>(p);
}

ib_status launch_interp_points(ib_plan* p, const void* u, int mode, double vscale,
                               double gscale, cudaStream_t s, const GridCall* calls,
                               const void* tmaps, const InterpIO* io) {
  const CUtensorMap* m = static_cast<const CUtensorMap*>(tmaps);
  return p->precision == IB_FP64
             ? interp_t<double>(p, u, mode, vscale, gscale, s, calls, m, io)
             : interp_t<float>(p, u, mode, vscale, gscale, s, calls, m, io);
}

bool encode_velocity_map(const int n[3], const void* u, void* map) {
  static_assert(sizeof(CUtensorMap) == kTensorMapBytes, "tensor map size");
  return make_velocity_map(n, u, static_cast<CUtensorMap*>(map));
}

}  // namespace ibfe
