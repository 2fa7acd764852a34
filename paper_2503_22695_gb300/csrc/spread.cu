// Spreading of Gauss-point values onto the periodic MAC grid (Section 4.4):
//   f^c(face) = scale * sum_q V_q^c prod_d phi(r_d),   r_d = (chi_q,d - x_face,d)/h,
// with scale = h^-3 for forces (delta_h carries h^-3) and 1 for the adjoint
// of interpolation.
//
// Kernels over 8^3-cell Eulerian tiles, no floating-point atomics, bitwise
// reproducible:
//
// k_spread_zero (side stream, concurrent with the push) -- one warp per
//   "far" tile (no points in its 3x3x3 neighbourhood) writes its zeros with
//   16-byte stores: the bulk of the field's HBM traffic overlaps the
//   accumulation work.
// k_spread_push_fx (FP32 plans) / k_spread_push (FP64 plans) -- persistent
//   CTAs pulling work items from a counter (a work item is at most 1024
//   consecutive points of one tile, so densely populated tiles are shared by
//   several CTAs) accumulate the item's points into a halo'd 12^3 block per
//   component (they reach two cells beyond the tile; indices stay
//   unwrapped).  FP32: exact fixed-point words with 32-bit shared atomics
//   (see below); FP64: half-warp private copies in double, steps ordered by
//   __syncwarp, summed in copy order.
// k_spread_merge_fx / k_spread_merge -- for every "near" tile, each face
//   sums the blocks of its own tile and of the neighbours whose halo covers
//   it (at most two per axis), in ascending (z, y, x) source order and,
//   within a source tile, in work-item order, and is written once: exact
//   integer sums rounded once (FP32), doubles in that fixed order (FP64).
//   Periodic wrap happens only here, through the neighbour-tile index.
#include <algorithm>

#include "ib_device.cuh"

namespace ibfe {
namespace {

constexpr int kB = 12;                  // halo'd block edge: tile 8 + 2 + 2
constexpr int kBlk = kB * kB * kB;      // 1728 faces per component
constexpr int kItemBlk = 3 * kBlk;      // scratch block of one work item
constexpr int kSY = kB;                 // shared y stride
constexpr int kSZ = kB * kB + 1;        // shared z stride (145: the 16 (dz,dy) rows hit 16 banks)
constexpr int kAcc = kB * kSZ;          // 1740 per private copy (multiple of 4)
constexpr int kPW = 4;                  // warps per push CTA
constexpr int kPT = kPW * 32;           // push threads
constexpr int kCopies = 2 * kPW;        // one private copy per half-warp
constexpr int kBatch = kPT;             // points staged per batch
constexpr int kMT = 256;                // merge / zero threads
constexpr int kMW = kMT / 32;

template <typename Real>
struct SpreadArgs {
  GridDev g;
  int ntiles;
  const InstDev* inst;         // packed plans: instance table, else null
  const int32_t* tile_inst;    // packed plans: instance of each tile
  const GridCall* calls;       // packed plans: each instance's f and scale, else null
  int64_t Q;
  const int32_t* tile_start;
  const int32_t* tile_end;
  const int32_t* tile_slot;    // first work item of each tile
  const int32_t* tile_nitems;  // work items of each tile
  const int32_t* tile_near;
  const int32_t* tile_list;    // tile of each work item
  const int32_t* tile_list_near;
  int32_t* counters;           // [0] work items, [1] work counter, [3] near tiles
  const int32_t* p_cell;
  const Real* p_off;
  const Real* p_val;
  int chunk;                   // points per work item
  Real scale;
  Real* scratch;               // [items][3][12^3]
  Real* f;
  const uint32_t* tile_vmax;   // FP32: bits of max |value| over each tile's points
  int32_t* tile_done;          // FP32: work items of each tile written in this call
  int4* tile_sk;               // FP32: (first block slot or -1, exponent k + 11, item bound, items)
};

// cp.async of 4 bytes global -> shared (completion awaited with cp_async_wait)
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// staged point: x/y/z weights, value, row origin in the halo'd block
template <typename Real>
struct alignas(16) Staged {
  Real wx[4];
  Real wy[4];
  Real wz[4];
  Real val;
  int org;
};

// Tile index of tile coordinates within one tile of the grid's range
// ([-1, nt]): the periodic wrap is one compare per axis, no division.
__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
__device__ __forceinline__ int tile_of(int tx, int ty, int tz, const TileGeo& t) {
  return t.base + wrap1(tx, t.nt[0]) + t.nt[0] * (wrap1(ty, t.nt[1]) + t.nt[1] * wrap1(tz, t.nt[2]));
}

// The call's scale and output field for the structure `inst` (packed plans:
// its row of the call table; a plan of one structure: the arguments).
template <bool kPacked, typename Real>
__device__ __forceinline__ Real call_scale(const SpreadArgs<Real>& A, int inst) {
  if constexpr (kPacked) return (Real)__ldg(&A.calls[inst].s0);
  return A.scale;
}
template <bool kPacked, typename Real>
__device__ __forceinline__ Real* call_field(const SpreadArgs<Real>& A, int inst) {
  if constexpr (kPacked) return static_cast<Real*>(A.calls[inst].field);
  return A.f;
}

// One lane adds into one face per step and steps are ordered by __syncwarp,
// so every face receives its contributions in point order.
template <typename Real>
__device__ __forceinline__ void add_shared(Real* p, Real v) {
  *p += v;
}

template <typename Real>
__device__ __forceinline__ void zero_shared(Real* p, int n, int tid, int nthreads) {
  float4* v = reinterpret_cast<float4*>(p);
  const int n4 = n * (int)sizeof(Real) / 16;
  for (int i = tid; i < n4; i += nthreads) v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Work item `slot`: points [start + j kChunk, min(end, start + (j+1) kChunk))
// of its tile, j = slot - first item of the tile.
// Raw point data of one work item, copied to shared memory once.
template <typename Real>
struct RawItem {
  int32_t cell[kChunk];
  Real off[3][kChunk];
  Real val[3][kChunk];
};

template <typename Real>
__device__ __forceinline__ void push_item(const SpreadArgs<Real>& A, int slot, Staged<Real>* stage,
                                          Real* acc, RawItem<Real>* raw, int tid) {
  const int tile = A.tile_list[slot];
  const TileGeo geo = tile_geo<false>(A.g, nullptr, nullptr, tile);  // FP64: one structure
  int tx, ty, tz;
  tile_coords(geo, tile, tx, ty, tz);
  const Real scale = A.scale;
  const int s = A.tile_start[tile] + (slot - A.tile_slot[tile]) * A.chunk;
  const int e = min(A.tile_end[tile], s + A.chunk);
  const int x0 = tx * kTile, y0 = ty * kTile, z0 = tz * kTile;
  const int hw = tid >> 4, l16 = tid & 15, dz = l16 >> 2, dy = l16 & 3;
  const int warp = tid >> 5;
  Real* my = acc + hw * kAcc;
  const int lane_off = dz * kSZ + dy * kSY;
  const int n = e - s;
  // every load of the item in flight at once
  for (int i = tid; i < n; i += kPT) {
    cp_async4(&raw->cell[i], A.p_cell + s + i);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (sizeof(Real) == 4) {
        cp_async4(&raw->off[d][i], A.p_off + d * A.Q + s + i);
        cp_async4(&raw->val[d][i], A.p_val + d * A.Q + s + i);
      } else {
        raw->off[d][i] = A.p_off[d * A.Q + s + i];
        raw->val[d][i] = A.p_val[d * A.Q + s + i];
      }
    }
  }
  cp_async_wait();

  for (int c = 0; c < 3; ++c) {
    zero_shared(acc, kCopies * kAcc, tid, kPT);
    for (int b0 = s; b0 < e; b0 += kBatch) {
      const int nb = min(kBatch, e - b0);
      __syncthreads();  // previous batch consumed, accumulators zeroed
      if (tid < nb) {
        const int i = b0 - s + tid;
        int cx, cy, cz;
        unpack_cell(raw->cell[i], cx, cy, cz);
        Staged<Real> st;
        Real th;
        const int bx = cx - x0 + stencil_axis(raw->off[0][i], c != 0, th) + 2;
        delta_weights(th, st.wx);
        const int by = cy - y0 + stencil_axis(raw->off[1][i], c != 1, th) + 2;
        delta_weights(th, st.wy);
        const int bz = cz - z0 + stencil_axis(raw->off[2][i], c != 2, th) + 2;
        delta_weights(th, st.wz);
        st.val = raw->val[c][i] * scale;
        st.org = bz * kSZ + by * kSY + bx;
        stage[tid] = st;
      }
      __syncthreads();
      // The warp's two half-warps take points hw + 8k; the loop runs the
      // even half's trip count (never smaller) so __syncwarp sees the full
      // warp.  The next point's staged values are read before the current
      // point's read-modify-writes.
      const int steps = nb > 2 * warp ? (nb - 2 * warp + kCopies - 1) / kCopies : 0;
      int p = hw;
      Real w = Real(0), wx[4] = {Real(0), Real(0), Real(0), Real(0)};
      int o = 0;
      if (p < nb) {
        const Staged<Real>& st = stage[p];
        w = st.val * st.wz[dz] * st.wy[dy];
#pragma unroll
        for (int k = 0; k < 4; ++k) wx[k] = st.wx[k];
        o = st.org + lane_off;
      }
      for (int k = 0; k < steps; ++k, p += kCopies) {
        Real wn = Real(0), wxn[4] = {Real(0), Real(0), Real(0), Real(0)};
        int on = 0;
        if (p + kCopies < nb) {
          const Staged<Real>& st = stage[p + kCopies];
          wn = st.val * st.wz[dz] * st.wy[dy];
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) wxn[kk] = st.wx[kk];
          on = st.org + lane_off;
        }
        if (p < nb) {
          Real* q = my + o;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) add_shared(q + kk, w * wx[kk]);
        }
        __syncwarp();
        w = wn;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) wx[kk] = wxn[kk];
        o = on;
      }
    }
    __syncthreads();
    Real* out = A.scratch + ((int64_t)slot * 3 + c) * kBlk;
    for (int idx = tid; idx < kBlk; idx += kPT) {
      const int z = idx / (kB * kB), y = (idx / kB) % kB, x = idx % kB;
      const int o = z * kSZ + y * kSY + x;
      Real sum = Real(0);
#pragma unroll
      for (int w = 0; w < kCopies; ++w) sum += acc[w * kAcc + o];
      out[idx] = sum;
    }
    __syncthreads();
  }
}

template <typename Real>
__global__ void __launch_bounds__(kPT) k_spread_push(SpreadArgs<Real> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Staged<Real>* stage = reinterpret_cast<Staged<Real>*>(smem_raw);
  Real* acc = reinterpret_cast<Real*>(smem_raw + sizeof(Staged<Real>) * kBatch);
  RawItem<Real>* raw = reinterpret_cast<RawItem<Real>*>(
      smem_raw + sizeof(Staged<Real>) * kBatch + sizeof(Real) * kCopies * kAcc);
  __shared__ int next;
  const int tid = threadIdx.x;
  const int count = A.counters[0];
  for (;;) {
    __syncthreads();
    if (tid == 0) next = atomicAdd(A.counters + 1, 1);
    __syncthreads();
    const int k = next;
    if (k >= count) break;
    push_item(A, k, stage, acc, raw, tid);
  }
}

// ---------------------------------------------------------------------------
// FP32 plans: order-independent fixed-point accumulation.
//
// Every contribution C = V scale prod phi of a point of tile t, in units of
// 2^-k_t, is split into an integer part h = round(C) and a fraction
// l = round(2^11 (C - h)) (units of 2^-(k_t + 11)), and both are added with
// native 32-bit shared-memory atomics into the work item's two word blocks.
// Integer addition is exact and associative, so the blocks do not depend on
// the order of the additions, on the order of the points or on how a tile's
// points are cut into work items.
//
// Both parts come from the magic-number rounding t = x + 1.5 2^23, whose bit
// pattern is 0x4B400000 + round(x) for |x| < 2^22; three fmas per
// contribution give both patterns, which are added as they are:
//   t1 = C + M                 bits(t1) = Mb + h
//   z  = M - 2^11 (t1 - M)     (exact: a multiple of 2^11 below 2^33)
//   t2 = 2^11 C + z            bits(t2) = Mb + l,  |l| <= 2^10
// After n contributions the words are hi = n Mb + H and lo = n Mb + L (mod
// 2^32).  Mb = 301 2^22 has zero low 22 bits and |L| <= 2^20 (n <= 1024), so
// L is the sign-extended low 22 bits of lo and H = (hi - lo) + L; the item
// stores S = 2^11 H + L per face, exact.
//
// Exponent of a tile (fx_tile_exp): from the largest |V| over the tile's
// points (an integer maximum of float bit patterns, itself order-independent)
// and its point count n_t.  Every kernel weight product is at most 1/8, so
// with cm = max|V| |scale| / 8 < 2^e, n_eff = min(n_t, 1024) <= 2^L (1024:
// the largest work item any tuning may choose) and k = min(21, 30 - L) - e,
// each contribution is below 2^21 and |H| below 2^31 at every face of an
// item.  The resolution 2^-(k+11) is about 2^-31 of the tile's largest
// contribution times n_eff / 1024; tiles far from large values keep their
// own fine resolution.
//
// Merge (k_spread_merge_fx): each face sums the items' S of every source tile
// in 64-bit integers, aligns the source sums to one exponent per destination
// tile (left shifts that provably fit in 64 bits; finer sources beyond that
// headroom are shifted right, a loss below 2^-17 of the coarsest source's
// resolution), adds them and rounds once.
// ---------------------------------------------------------------------------
constexpr float kMagic = 12582912.0f;             // M = 1.5 * 2^23
constexpr float kMagicZ = 12582912.0f * 2049.0f;  // M (1 + 2^11), exact in float
constexpr int kFxThreads = 256;
constexpr int kFxWarps = kFxThreads / 32;
constexpr int kFxGroup = 16;  // points a warp stages at a time: 2 lanes per point
// Lane mapping: a warp takes one point at a time; lane (dz, dy, xh) adds the
// faces xh and xh + 2 of stencil row (dz, dy), one instruction per face,
// word and component.  With y stride 14 and z stride 168 the 16 row offsets
// 168 dz + 14 dy are the 16 even residues mod 32, so the 32 lanes of every
// atomic hit 32 distinct banks wherever the point lies.
constexpr int kFxSY = 14;
constexpr int kFxSZ = kB * kFxSY;       // 168
constexpr int kFxAcc = kB * kFxSZ;      // 2016 words per component
constexpr int kFxWords = 3 * kFxAcc;    // one word block (hi or lo) of a work item
constexpr int kFxBlk = 3 * kBlk;        // faces of an item's halo'd block: one int64 S each
// A staged point (9 float4, an odd stride so that the staging stores of the
// group's points to one slot spread over the banks): [0..3] the rows dz of
// (v0 w_z(1/2), v1 w_z(1/2), v2 w_z(0), 0) with v = 2^k V scale, [4..5] the
// pairs (w_y(0)[dy], w_y(1/2)[dy]), [6..7] the x weights of the two lane
// halves (xh = 0, 1: (s 0 [xh], s 0 [xh + 2], s 1/2 [xh], s 1/2 [xh + 2])),
// [8] the word offsets of the three components' stencil starts.  Each
// component takes its own staggering (0: x at 0, y and z at 1/2; 1: y at 0;
// 2: z at 0); a lane forms its row weight from the z and y parts.
constexpr int kFxRec = 9;
constexpr int kFxRecWy = 4;
constexpr int kFxRecWx = 6;
constexpr int kFxRecOrg = 8;

// adds the contribution C = w wx (in units of 2^-k) at word offset a
__device__ __forceinline__ void fx_add(unsigned* hi, unsigned* lo, float w, float w11, float wx) {
  const float t1 = fmaf(w, wx, kMagic);
  const float z = fmaf(t1, -2048.0f, kMagicZ);
  const float t2 = fmaf(w11, wx, z);
  atomicAdd(hi, __float_as_uint(t1));
  atomicAdd(lo, __float_as_uint(t2));
}

__device__ __forceinline__ int ceil_log2(int n) { return n > 1 ? 32 - __clz(n - 1) : 0; }

// Fixed-point exponent of a tile from the bits of its largest |V|, its point
// count and the call's scale (see above).  n_eff uses the largest work item
// any tuning may choose (kChunk), so the exponent, hence the result, does not
// depend on the plan's tuning.  Values of magnitude up to about 2^120 / |scale|
// are representable.
__device__ __forceinline__ int fx_tile_exp(uint32_t vmax_bits, int npts, float scale) {
  const float cm = 0.125f * __uint_as_float(vmax_bits) * fabsf(scale);
  if (!(cm > 0.f) || !(cm <= 3.0e38f)) return 0;  // no values, or not finite
  int e = 0;
  frexpf(cm, &e);  // cm < 2^e
  const int k = min(21, 30 - ceil_log2(min(npts, kChunk))) - e;
  return max(-100, min(k, 100));
}

// The 4-point weights of delta_weights with the hardware reciprocal square
// root and reciprocal (a few units in the last place instead of correctly
// rounded steps): q = (1 + p) rsqrt(1 + p), q - 1 = p / (1 + q).
__device__ __forceinline__ void fx_weights(float th, float w[4]) {
  const float om = 1.f - th;
  const float p = 4.f * th * om;
  const float s = 1.f + p;
  const float q = s * rsqrtf(s);
  const float qm1 = __fdividef(p, 1.f + q);
  w[0] = (2.f * om - qm1) * 0.125f;
  w[1] = (2.f * om + 2.f + qm1) * 0.125f;
  w[2] = (2.f * th + 2.f + qm1) * 0.125f;
  w[3] = (2.f * th - qm1) * 0.125f;
}

// Raw data of one point, loaded a group ahead so that the loads are in
// flight while the warp accumulates the current group.
struct FxRaw {
  int32_t cell;
  float off[3];
  float val[3];
};

__device__ __forceinline__ void fx_fetch(const SpreadArgs<float>& A, int i, FxRaw& r) {
  r.cell = __ldg(A.p_cell + i);
#pragma unroll
  for (int d = 0; d < 3; ++d) r.off[d] = __ldg(A.p_off + d * A.Q + i);
#pragma unroll
  for (int c = 0; c < 3; ++c) r.val[c] = __ldg(A.p_val + c * A.Q + i);
}

// Lanes pt and pt + kFxGroup stage point pt of the group.  Lane half `part`
// evaluates the 1-D weights of its staggering along all three axes (part 0:
// s = 0, part 1: s = 1/2), takes the other staggering's y weights and the z
// weights of its two rows from its partner lane, and writes the rows
// dz = 2 part, 2 part + 1.  Every lane of the warp runs this (the shuffles
// need the whole warp); `store` is false for lanes past the group's end.
__device__ __forceinline__ void fx_stage(float4* rec, int part, bool store, const FxRaw& r,
                                         const int lc0[3], float vscale) {
  int cc[3];
  unpack_cell(r.cell, cc[0], cc[1], cc[2]);
  int b[3][2];
  float th[3][2];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf)
      b[d][hf] = cc[d] - lc0[d] + stencil_axis(r.off[d], hf == 1, th[d][hf]) + 2;
  float w[3][4];  // this half's staggering
#pragma unroll
  for (int d = 0; d < 3; ++d) fx_weights(part ? th[d][1] : th[d][0], w[d]);
  const unsigned full = 0xffffffffu;
  float wyo[4];  // the partner's y weights (the other staggering)
#pragma unroll
  for (int j = 0; j < 4; ++j) wyo[j] = __shfl_xor_sync(full, w[1][j], kFxGroup);
  // the partner's z weights of this half's rows
  const float zo0 = __shfl_xor_sync(full, part ? w[2][0] : w[2][2], kFxGroup);
  const float zo1 = __shfl_xor_sync(full, part ? w[2][1] : w[2][3], kFxGroup);
  if (!store) return;
  float wy0[4], wyh[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    wy0[j] = part ? wyo[j] : w[1][j];
    wyh[j] = part ? w[1][j] : wyo[j];
  }
  const float v0 = r.val[0] * vscale, v1 = r.val[1] * vscale, v2 = r.val[2] * vscale;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float own = part ? w[2][2 + j] : w[2][j];
    const float oth = j ? zo1 : zo0;
    const float wz0 = part ? oth : own, wzh = part ? own : oth;
    // component 0: z, y at s = 1/2; component 1: z at 1/2, y at 0; component 2: z at 0, y at 1/2
    const float a0 = v0 * wzh, a1 = v1 * wzh, a2 = v2 * wz0;
    rec[2 * part + j] = make_float4(a0, a1, a2, 0.f);
  }
  rec[kFxRecWy + part] = part ? make_float4(wy0[2], wyh[2], wy0[3], wyh[3])
                              : make_float4(wy0[0], wyh[0], wy0[1], wyh[1]);
  reinterpret_cast<float2*>(rec + kFxRecWx)[part] = make_float2(w[0][0], w[0][2]);
  reinterpret_cast<float2*>(rec + kFxRecWx + 1)[part] = make_float2(w[0][1], w[0][3]);
  if (part == 0)
    reinterpret_cast<int4*>(rec)[kFxRecOrg] =
        make_int4(b[2][1] * kFxSZ + b[1][1] * kFxSY + b[0][0],
                  kFxAcc + b[2][1] * kFxSZ + b[1][0] * kFxSY + b[0][1],
                  2 * kFxAcc + b[2][0] * kFxSZ + b[1][1] * kFxSY + b[0][1], 0);
}

// Merge of the near tiles (FP32 plans): every face adds the S of the covering
// source tiles (each tile's blocks summed into its first block by the
// accumulation kernel) in the fixed order (oz, oy, ox), aligned to the
// destination tile's exponent k_ref (in units of 2^-(k+11)), and is rounded
// once.  With k'_s = k_s + 11 and m_s = ceil(n_s / 512) for source s (n_s
// points: m_s bounds its work items under any tuning, whose items hold 512
// to 1024 points),
//   k_ref = min(max_s k'_s, min_s (k'_s + 17 - ceil_log2(m_s))),
// so a source sum (below m_s 2^42) shifted left by k_ref - k'_s stays below
// 2^59 and eight of them below 2^62; a source with k'_s > k_ref is shifted
// right (floor).  k_ref, like k_s, does not depend on the tuning.  The conversion splits |S| into two 32-bit halves,
// each converted exactly rounded, joined by one fma: within one unit in the
// last place, the same bits for the same integers.
__device__ __forceinline__ float fx_to_float(long long S, float out_scale) {
  const unsigned long long m = S < 0 ? 0ull - (unsigned long long)S : (unsigned long long)S;
  const float f = fmaf((float)(unsigned)(m >> 32), 4294967296.0f, (float)(unsigned)m);
  return (S < 0 ? -f : f) * out_scale;
}

// v 2^sh, floor for sh < 0 (left shifts never exceed the headroom above; a
// right shift of 63 or more leaves the sign: floor of |v| < 2^63 over 2^63)
__device__ __forceinline__ long long fx_align(long long v, int sh) {
  return sh >= 0 ? (long long)((unsigned long long)v << sh) : (v >> min(-sh, 63));
}

template <bool kPacked>
__global__ void __launch_bounds__(kFxThreads) k_spread_push_fx(SpreadArgs<float> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* groups = reinterpret_cast<float4*>(smem_raw);
  unsigned* acc_hi = reinterpret_cast<unsigned*>(smem_raw + sizeof(float4) * kFxWarps * kFxGroup *
                                                                kFxRec);
  unsigned* acc_lo = acc_hi + kFxWords;
  __shared__ int next, last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int count = A.counters[0];
  // this lane's (dz, dy, xh) and its offset within a stencil
  const int ldz = lane >> 3, ldy = (lane >> 1) & 3, lxh = lane & 1;
  const int loff = ldz * kFxSZ + ldy * kFxSY + lxh;
  // this lane's staging role: point pt of the group, lane half `part`
  const int pt = lane & (kFxGroup - 1), part = (lane / kFxGroup) & 1;
  const bool stager = lane < 2 * kFxGroup;
  float4* G = groups + warp * kFxGroup * kFxRec;
  for (;;) {
    __syncthreads();  // previous item written out
    if (tid == 0) next = atomicAdd(A.counters + 1, 1);
    __syncthreads();
    const int slot = next;
    if (slot >= count) break;
    const int tile = A.tile_list[slot];
    const TileGeo geo = tile_geo<kPacked>(A.g, A.inst, A.tile_inst, tile);
    int tx, ty, tz;
    tile_coords(geo, tile, tx, ty, tz);
    const int t0 = A.tile_start[tile], t1 = A.tile_end[tile];
    const int s = t0 + (slot - A.tile_slot[tile]) * A.chunk;
    const int e = min(t1, s + A.chunk);
    const int lc0[3] = {tx * kTile, ty * kTile, tz * kTile};
    const int4 tsk = A.tile_sk[tile];
    const float vscale = call_scale<kPacked>(A, geo.inst) * ldexpf(1.f, tsk.y - 11);
    // warp w takes the groups starting at s + kFxGroup (w + 8 j)
    FxRaw raw = {0, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    int g0 = s + warp * kFxGroup;
    if (stager && g0 + pt < e) fx_fetch(A, g0 + pt, raw);
    for (int i = tid; i < 2 * kFxWords / 4; i += kFxThreads)
      reinterpret_cast<uint4*>(acc_hi)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();  // accumulators zeroed
    for (; g0 < e; g0 += kFxWarps * kFxGroup) {
      const int ng = min(kFxGroup, e - g0);
      fx_stage(G + pt * kFxRec, part, stager && pt < ng, raw, lc0, vscale);
      __syncwarp();
      const int gn = g0 + kFxWarps * kFxGroup;
      if (stager && gn + pt < e) fx_fetch(A, gn + pt, raw);
      // one point per warp step: lane (dz, dy, xh) adds faces xh and xh + 2
      // of its (dz, dy) row, for each component
#pragma unroll 2
      for (int q = 0; q < ng; ++q) {
        const float4* rq = G + q * kFxRec;
        const float4 vz = rq[ldz];
        const float2 wy = reinterpret_cast<const float2*>(rq + kFxRecWy)[ldy];
        const float4 wr = make_float4(vz.x * wy.y, vz.y * wy.x, vz.z * wy.y, 0.f);
        const float4 wx = rq[kFxRecWx + lxh];
        const int4 og = reinterpret_cast<const int4*>(rq)[kFxRecOrg];
        int a = og.x + loff;
        float w11 = wr.x * 2048.0f;
        fx_add(acc_hi + a, acc_lo + a, wr.x, w11, wx.x);
        fx_add(acc_hi + a + 2, acc_lo + a + 2, wr.x, w11, wx.y);
        a = og.y + loff;
        w11 = wr.y * 2048.0f;
        fx_add(acc_hi + a, acc_lo + a, wr.y, w11, wx.z);
        fx_add(acc_hi + a + 2, acc_lo + a + 2, wr.y, w11, wx.w);
        a = og.z + loff;
        w11 = wr.z * 2048.0f;
        fx_add(acc_hi + a, acc_lo + a, wr.z, w11, wx.z);
        fx_add(acc_hi + a + 2, acc_lo + a + 2, wr.z, w11, wx.w);
      }
      __syncwarp();  // group consumed before it is restaged
    }
    __syncthreads();
    // S = 2^11 H + L of every face, exact, in the 12-face rows of the scratch
    // block; consecutive threads take consecutive face pairs (16-byte stores)
    longlong2* out = reinterpret_cast<longlong2*>(A.scratch) + (int64_t)slot * (kFxBlk / 2);
    for (int u = tid; u < kFxBlk / 2; u += kFxThreads) {
      const int row = u / (kB / 2), x = 2 * (u % (kB / 2));
      const int c = row / (kB * kB), zy = row % (kB * kB);
      const int o = c * kFxAcc + (zy / kB) * kFxSZ + (zy % kB) * kFxSY + x;  // even: 8-byte aligned
      const uint2 hw = *reinterpret_cast<const uint2*>(acc_hi + o);
      const uint2 lw = *reinterpret_cast<const uint2*>(acc_lo + o);
      const int L0 = (int)(lw.x << 10) >> 10, L1 = (int)(lw.y << 10) >> 10;
      const int H0 = (int)(hw.x - lw.x) + L0, H1 = (int)(hw.y - lw.y) + L1;
      out[u] = make_longlong2((long long)H0 * 2048 + L0, (long long)H1 * 2048 + L1);
    }
    // Tiles cut into several work items: the item whose block completes the
    // tile's count adds all of the tile's item blocks, in item order and in
    // exact 64-bit integers, into the tile's first block, while they are
    // fresh in L2; the merge then reads one block per tile.  Every thread
    // fences its own block stores before the barrier that precedes the count;
    // the summing CTA fences after reading it.
    const int nit = A.tile_nitems[tile];
    if (nit > 1) {
      __threadfence();
      __syncthreads();
      if (tid == 0) last = atomicAdd(A.tile_done + tile, 1) + 1 == nit;
      __syncthreads();
      if (last) {
        __threadfence();
        longlong2* first = reinterpret_cast<longlong2*>(A.scratch) +
                           (int64_t)A.tile_slot[tile] * (kFxBlk / 2);
        for (int u = tid; u < kFxBlk / 2; u += kFxThreads) {
          long long a0 = 0, a1 = 0;
          for (int j = 0; j < nit; ++j) {
            const longlong2 v = __ldcg(first + (int64_t)j * (kFxBlk / 2) + u);
            a0 += v.x;
            a1 += v.y;
          }
          first[u] = make_longlong2(a0, a1);
        }
      }
    }
  }
}

// Per tile (FP32 plans), one thread each: the exponent k of its fixed-point
// words, its first block slot, the bound m = ceil(n / 512) on its work items
// under any tuning, and its work items; read by every push item of the tile
// and by the merge of each of its 27 neighbours.  Also zeroes the
// accumulation's counters (its work counter and the tiles' written items),
// which saves two memsets ahead of the push.
template <bool kPacked>
__global__ void __launch_bounds__(256) k_tile_info(SpreadArgs<float> A, int ntiles) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) A.counters[1] = 0;  // the accumulation's work counter
  if (t >= ntiles) return;
  A.tile_done[t] = 0;             // items of the tile written in this call
  const int ns = A.tile_nitems[t];
  const int npts = A.tile_end[t] - A.tile_start[t];
  const float scale = call_scale<kPacked>(A, kPacked ? __ldg(A.tile_inst + t) : 0);
  A.tile_sk[t] = make_int4(ns > 0 ? A.tile_slot[t] : -1,
                           ns > 0 ? fx_tile_exp(__ldg(A.tile_vmax + t), npts, scale) + 11 : 0,
                           (npts + kMinChunk - 1) / kMinChunk, ns);
}

// One CTA per near tile, one thread per face pair of each component, no
// barrier: lanes 0..26 of each warp load the records of the 27 tiles whose
// blocks cover the tile, the warp reduces the merge exponent
//   k_ref = min(max_s k'_s, min_s (k'_s + 17 - ceil_log2(m_s))),
// and each thread takes its up to eight sources' records by shuffle once,
// then, component by component, loads their blocks together and sums them.
template <bool kPacked>
__global__ void __launch_bounds__(kMT, 4) k_spread_merge_fx(SpreadArgs<float> A) {
  static_assert(kMT == 8 * 8 * 4, "one thread per face pair of a tile component");
  const unsigned full = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31;
  const int count = A.counters[3];
  const longlong2* scratch = reinterpret_cast<const longlong2*>(A.scratch);  // 2 faces each
  // this thread's faces: x = 2 xq and 2 xq + 1 of row (z, y)
  const int z = tid >> 5, y = (tid >> 2) & 7, xq = tid & 3;
  // covering sources along each axis: the tile itself, and the lower (upper)
  // neighbour for the faces 0, 1 (6, 7)
  const int lz = z <= 1 ? -1 : 0, ly = y <= 1 ? -1 : 0, lx = xq == 0 ? -1 : 0;
  const int nz = (z <= 1 || z >= 6) ? 2 : 1, ny = (y <= 1 || y >= 6) ? 2 : 1,
            nx = (xq == 0 || xq == 3) ? 2 : 1;
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    const int tile = A.tile_list_near[k];
    const TileGeo geo = tile_geo<kPacked>(A.g, A.inst, A.tile_inst, tile);
    int tx, ty, tz;
    tile_coords(geo, tile, tx, ty, tz);
    int4 r = make_int4(-1, 0, 0, 0);
    if (lane < 27)
      r = __ldg(A.tile_sk + tile_of(tx + lane % 3 - 1, ty + (lane / 3) % 3 - 1,
                                    tz + lane / 9 - 1, geo));
    const int kmax = __reduce_max_sync(full, r.w > 0 ? r.y : -1000);
    const int kcap = __reduce_min_sync(full, r.w > 0 ? r.y + 17 - ceil_log2(r.z) : 1000);
    const int kref = min(kmax, kcap);
    int2 sk[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int iz = i >> 2, iy = (i >> 1) & 1, ix = i & 1;
      const bool use = iz < nz && iy < ny && ix < nx;
      const int src = (lz + iz + 1) * 9 + (ly + iy + 1) * 3 + lx + ix + 1;
      const int slot = __shfl_sync(full, r.x, use ? src : 0);
      const int kx = __shfl_sync(full, r.y, use ? src : 0);
      sk[i] = make_int2(use ? slot : -1, use ? kx : kref);  // unused: value 0, shift 0
    }
    // The upper z sources (i >= 4) cover only the warps of z rows 0, 1, 6, 7
    // (nz is uniform in a warp: z = tid / 32).  Unless a covering source is
    // finer than k_ref (a right shift, rare), the warp aligns by left shifts
    // alone (exact); otherwise it takes the general alignment.
    bool finer = false;
#pragma unroll
    for (int i = 0; i < 8; ++i) finer |= sk[i].y > kref;
    const bool exact_left = !__any_sync(full, finer);
    const float osc = ldexpf(1.f, -kref);
    const int n0 = geo.n[0], n1 = geo.n[1];
    const int64_t cells = (int64_t)n0 * n1 * geo.n[2];
    float* const row0 = call_field<kPacked>(A, geo.inst) +
                        ((int64_t)(tz * kTile + z) * n1 + (ty * kTile + y)) * n0 + tx * kTile;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
      longlong2 v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        v[i] = make_longlong2(0, 0);
        if (sk[i].x >= 0) {
          // this face pair in the source tile's halo'd block (face-pair units)
          const int oz = lz + (i >> 2), oy = ly + ((i >> 1) & 1), ox = lx + (i & 1);
          const int q = ((z - oz * kTile + 2) * kB + (y - oy * kTile + 2)) * (kB / 2) + xq + 1 -
                        (kTile / 2) * ox;
          v[i] = __ldcg(scratch + (int64_t)sk[i].x * (kFxBlk / 2) + c * (kBlk / 2) + q);
        }
      }
      long long t0 = 0, t1 = 0;
      if (exact_left) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (i >= 4 && nz == 1) break;
          const int sh = kref - sk[i].y;  // 0 .. 17
          t0 += (long long)((unsigned long long)v[i].x << sh);
          t1 += (long long)((unsigned long long)v[i].y << sh);
        }
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          t0 += fx_align(v[i].x, kref - sk[i].y);
          t1 += fx_align(v[i].y, kref - sk[i].y);
        }
      }
      reinterpret_cast<float2*>(row0 + c * cells)[xq] =
          make_float2(fx_to_float(t0, osc), fx_to_float(t1, osc));
    }
  }
}

// Far tiles: one warp per tile, 3 components x 64 rows x 16-byte zeros.
template <typename Real, bool kPacked>
__global__ void __launch_bounds__(kMT) k_spread_zero(SpreadArgs<Real> A) {
  const int lane = threadIdx.x & 31;
  const int tile = blockIdx.x * kMW + (threadIdx.x >> 5);
  if (tile >= A.ntiles || A.tile_near[tile]) return;
  const TileGeo geo = tile_geo<kPacked>(A.g, A.inst, A.tile_inst, tile);
  int tx, ty, tz;
  tile_coords(geo, tile, tx, ty, tz);
  const int n0 = geo.n[0], n1 = geo.n[1];
  const int64_t cells = (int64_t)n0 * n1 * geo.n[2];
  Real* const f = call_field<kPacked>(A, geo.inst);
  const int x0 = tx * kTile, y0 = ty * kTile, z0 = tz * kTile;
  constexpr int kVec = 16 / sizeof(Real);          // reals per 16-byte store
  constexpr int kPerRow = kTile / kVec;
  for (int idx = lane; idx < 3 * 64 * kPerRow; idx += 32) {
    const int c = idx / (64 * kPerRow), r = (idx / kPerRow) % 64, v = idx % kPerRow;
    const int z = r >> 3, y = r & 7;
    Real* row = f + c * cells + ((int64_t)(z0 + z) * n1 + (y0 + y)) * n0 + x0;
    reinterpret_cast<float4*>(row)[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Near tiles: fixed-order sum of the halo'd blocks that cover each face.
// Source (ox, oy, oz) covers local face (x, y, z) when each offset is 0, or
// -1 with the coordinate <= 1, or +1 with it >= 6; the face is then at block
// index (x - 8 ox + 2, y - 8 oy + 2, z - 8 oz + 2).  One thread per x-row of 8
// faces (component, z, y): for each (oz, oy) source pair in order it reads
// the row's own-tile part (block x 2..9) and, for faces 0,1 and 6,7, the
// x-neighbours' halo pairs (block x 10,11 of ox = -1 and 0,1 of ox = +1),
// and adds them face by face in the order (oz, oy, ox).
template <typename Real>
__global__ void __launch_bounds__(kMT) k_spread_merge(SpreadArgs<Real> A) {
  __shared__ int src_slot[27], src_n[27];
  const int tid = threadIdx.x;
  const int count = A.counters[3];
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    const int tile = A.tile_list_near[k];
    const TileGeo geo = tile_geo<false>(A.g, nullptr, nullptr, tile);  // FP64: one structure
    int tx, ty, tz;
    tile_coords(geo, tile, tx, ty, tz);
    const int n0 = geo.n[0], n1 = geo.n[1];
    const int64_t cells = (int64_t)n0 * n1 * geo.n[2];
    const int x0 = tx * kTile, y0 = ty * kTile, z0 = tz * kTile;
    __syncthreads();
    if (tid < 27) {
      const int a = tid / 9 - 1, b = (tid / 3) % 3 - 1, c = tid % 3 - 1;
      const int nb = tile_of(tx + c, ty + b, tz + a, geo);
      src_slot[tid] = A.tile_slot[nb];
      src_n[tid] = A.tile_nitems[nb];
    }
    __syncthreads();
    if (tid < 3 * 64) {
      const int c = tid >> 6, z = (tid >> 3) & 7, y = tid & 7;
      const int ly = y <= 1 ? -1 : 0, lz = z <= 1 ? -1 : 0;
      const int hy = y >= 6 ? 1 : 0, hz = z >= 6 ? 1 : 0;
      Real sum[8];
#pragma unroll
      for (int x = 0; x < 8; ++x) sum[x] = Real(0);
      for (int oz = lz; oz <= hz; ++oz)
        for (int oy = ly; oy <= hy; ++oy) {
          const int rowoff = c * kBlk + ((z - oz * kTile + 2) * kB + (y - oy * kTile + 2)) * kB;
          const int s0 = (oz + 1) * 9 + (oy + 1) * 3;
          for (int ox = -1; ox <= 1; ++ox) {
            const int sl = src_slot[s0 + ox + 1], ns = src_n[s0 + ox + 1];
            for (int j = 0; j < ns; ++j) {
              const Real* r = A.scratch + (int64_t)(sl + j) * kItemBlk + rowoff;
              if (ox < 0) {          // faces 0,1 from the left neighbour's block x 10,11
                sum[0] += r[10];
                sum[1] += r[11];
              } else if (ox > 0) {   // faces 6,7 from the right neighbour's block x 0,1
                sum[6] += r[0];
                sum[7] += r[1];
              } else {
                Real v[8];
#pragma unroll
                for (int x = 0; x < 8; ++x) v[x] = r[2 + x];
#pragma unroll
                for (int x = 0; x < 8; ++x) sum[x] += v[x];
              }
            }
          }
        }
      Real* out = A.f + c * cells + ((int64_t)(z0 + z) * n1 + (y0 + y)) * n0 + x0;
#pragma unroll
      for (int x = 0; x < 8; ++x) out[x] = sum[x];
    }
  }
}

template <typename Real>
size_t push_smem() {
  return sizeof(Staged<Real>) * kBatch + sizeof(Real) * kCopies * kAcc + sizeof(RawItem<Real>);
}

constexpr size_t kFxSmem =
    sizeof(float4) * kFxWarps * kFxGroup * kFxRec + sizeof(unsigned) * 2 * kFxWords;

template <bool kPacked>
void launch_push(ib_plan* p, const SpreadArgs<float>& A, cudaStream_t s) {
  k_tile_info<kPacked><<<(p->ntiles + 255) / 256, 256, 0, s>>>(A, p->ntiles);
  p->prof_calls[IB_STAGE_SPREAD_PUSH] += 1;
  const int ev = prof_begin(p, IB_STAGE_SPREAD_PUSH, s);
  k_spread_push_fx<kPacked><<<std::min(p->push_ctas, p->push_per_sm * p->sm_count), kFxThreads,
                              kFxSmem, s>>>(A);
  prof_end(p, ev, s);
}

template <bool kPacked>
void launch_push(ib_plan* p, const SpreadArgs<double>& A, cudaStream_t s) {
  static_assert(!kPacked, "packed plans are FP32");
  k_spread_push<double><<<std::min(p->push_ctas, p->push_per_sm * p->sm_count), kPT,
                          push_smem<double>(), s>>>(A);
}

template <typename Real>
SpreadArgs<Real> spread_args(ib_plan* p, double scale, void* f, const GridCall* calls,
                             const void* vals = nullptr) {
  SpreadArgs<Real> A;
  A.g = p->grid;
  A.ntiles = p->ntiles;
  A.inst = p->n_inst > 1 ? p->inst : nullptr;
  A.tile_inst = p->n_inst > 1 ? p->tile_inst : nullptr;
  A.calls = calls;
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
  A.p_val = (const Real*)(vals ? vals : p->p_val);
  A.chunk = p->chunk;
  A.scale = (Real)scale;
  A.scratch = (Real*)p->spread_scratch;
  A.f = (Real*)f;
  A.tile_vmax = p->tile_vmax;
  A.tile_done = p->tile_done;
  A.tile_sk = reinterpret_cast<int4*>(p->tile_sk);
  return A;
}

template <typename Real, bool kPacked>
ib_status spread_t(ib_plan* p, double scale, void* f, bool zero_fill, cudaStream_t s,
                   const GridCall* calls, const void* vals) {
  SpreadArgs<Real> A = spread_args<Real>(p, scale, f, calls, vals);
  // the FP32 accumulation's counter is reset by k_tile_info
  if constexpr (sizeof(Real) == 8) cudaMemsetAsync(p->tile_counters + 1, 0, sizeof(int32_t), s);
  // far-tile zeros on the side stream, concurrent with the push (unless the
  // caller has already issued them)
  if (zero_fill) {
    cudaEventRecord(p->ev_fork, s);
    cudaStreamWaitEvent(p->zside, p->ev_fork, 0);
    k_spread_zero<Real, kPacked><<<(p->ntiles + kMW - 1) / kMW, kMT, 0, p->zside>>>(A);
    cudaEventRecord(p->ev_join, p->zside);
  }
  launch_push<kPacked>(p, A, s);
  if constexpr (sizeof(Real) == 4)
    k_spread_merge_fx<kPacked><<<p->merge_ctas, kMT, 0, s>>>(A);
  else
    k_spread_merge<Real><<<p->merge_ctas, kMT, 0, s>>>(A);
  if (zero_fill) cudaStreamWaitEvent(s, p->ev_join, 0);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

template <typename Real>
ib_status prepare_t(ib_plan* p) {
  int dev = 0, sms = 0, per_sm = 0, per_sm_merge = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return IB_ERR_CUDA;
  cudaError_t e;
  if (sizeof(Real) == 4) {
    // both variants (one structure, packed): the grid takes the smaller
    // occupancy of the two
    int per_sm_packed = 0;
    e = cudaFuncSetAttribute(k_spread_push_fx<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kFxSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_spread_push_fx<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kFxSmem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread_push_fx<false>,
                                                        kFxThreads, kFxSmem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_packed, k_spread_push_fx<true>,
                                                        kFxThreads, kFxSmem);
    per_sm = std::min(per_sm, per_sm_packed);
  } else {
    const int smem = (int)push_smem<Real>();
    e = cudaFuncSetAttribute(k_spread_push<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread_push<Real>, kPT, smem);
  }
  if (e == cudaSuccess) {
    if constexpr (sizeof(Real) == 4)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_merge, k_spread_merge_fx<false>,
                                                        kMT, 0);
    else
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_merge, k_spread_merge<Real>, kMT,
                                                        0);
  }
  if (e != cudaSuccess || per_sm < 1 || per_sm_merge < 1) return IB_ERR_CUDA;
  p->sm_count = sms;
  p->push_ctas = sms * per_sm;
  p->merge_ctas = sms * per_sm_merge;
  return IB_OK;
}

}  // namespace

size_t spread_scratch_bytes(int precision, int64_t slots) {
  // FP64: one double per face; FP32: the exact integer S per face
  return precision == IB_FP64 ? (size_t)slots * kItemBlk * sizeof(double)
                              : (size_t)slots * kFxBlk * sizeof(long long);
}

ib_status spread_prepare(ib_plan* p) {
  return p->precision == IB_FP64 ? prepare_t<double>(p) : prepare_t<float>(p);
}

// zeros, accumulation, merge (FP32: and the merge exponents)
int spread_launches(int precision) { return precision == IB_FP64 ? 3 : 4; }

ib_status launch_spread(ib_plan* p, double scale, void* f, cudaStream_t s, bool zero_fill,
                        const GridCall* calls, const void* vals) {
  if ((p->n_inst > 1) != (calls != nullptr)) return IB_ERR_INVALID_ARG;
  if (p->precision == IB_FP64)
    return p->n_inst > 1 ? IB_ERR_INVALID_ARG
                         : spread_t<double, false>(p, scale, f, zero_fill, s, calls, vals);
  return p->n_inst > 1 ? spread_t<float, true>(p, scale, f, zero_fill, s, calls, vals)
                       : spread_t<float, false>(p, scale, f, zero_fill, s, calls, vals);
}

ib_status launch_spread_zero(ib_plan* p, void* f, cudaStream_t s, const GridCall* calls) {
  if ((p->n_inst > 1) != (calls != nullptr)) return IB_ERR_INVALID_ARG;
  if (p->precision == IB_FP64) {
    SpreadArgs<double> A = spread_args<double>(p, 1.0, f, calls);
    k_spread_zero<double, false><<<(p->ntiles + kMW - 1) / kMW, kMT, 0, s>>>(A);
  } else {
    SpreadArgs<float> A = spread_args<float>(p, 1.0, f, calls);
    if (p->n_inst > 1)
      k_spread_zero<float, true><<<(p->ntiles + kMW - 1) / kMW, kMT, 0, s>>>(A);
    else
      k_spread_zero<float, false><<<(p->ntiles + kMW - 1) / kMW, kMT, 0, s>>>(A);
  }
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

}  // namespace ibfe
