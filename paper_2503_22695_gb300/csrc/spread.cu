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
  uint32_t* absmax;            // bits of max |value| over all points (fixed-point scale)
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

__device__ __forceinline__ int tile_of(int tx, int ty, int tz, const GridDev& g) {
  return wrap_idx(tx, g.nt[0]) + g.nt[0] * (wrap_idx(ty, g.nt[1]) + g.nt[1] * wrap_idx(tz, g.nt[2]));
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
  const int nt0 = A.g.nt[0], nt1 = A.g.nt[1];
  const int tile = A.tile_list[slot];
  const int tx = tile % nt0, ty = (tile / nt0) % nt1, tz = tile / (nt0 * nt1);
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
        st.val = raw->val[c][i] * A.scale;
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
// Every contribution C = V prod phi of an item, in units of 2^-k, is split into
// an integer part h = round(C) and a fraction l = round(2^11 (C - h)) (in
// units of 2^-(k+11)), and both are added with native 32-bit shared-memory
// atomics into one block per CTA.  Integer addition is exact and associative,
// so the block is the same whatever the order of the additions.
//
// Both parts come from the magic-number rounding t = x + 1.5 2^23, whose bit
// pattern is 0x4B400000 + round(x) for |x| < 2^22; three fmas per
// contribution give both patterns, which are added as they are:
//   t1 = C + M                 bits(t1) = Mb + h
//   z  = M - 2^11 (t1 - M)     (exact: a multiple of 2^11 below 2^32)
//   t2 = 2^11 C + z            bits(t2) = Mb + l,  |l| <= 2^10
// After n contributions the words are hi = n Mb + H and lo = n Mb + L (mod
// 2^32).  Mb = 301 2^22 has zero low 22 bits and |L| <= 2^20 (n <= 1024), so
// L is the sign-extended low 22 bits of lo, and H = (hi - lo) + L.  k comes
// from the largest |V| of the call (one integer atomicMax over the float bit
// patterns) so that |C| < 2^19, since every kernel weight product is at most
// 1/8; hence |H| < 2^29.  The resolution is 2^-(k+12), about 2^-31 of the
// largest contribution; each block value H 2^11 + L is rounded to float by
// one fma of the two parts converted to float (exact conversions while
// |H| < 2^24); the same integers always give the same float.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_absmax(const float* __restrict__ v, int64_t n,
                                               uint32_t* __restrict__ out) {
  float m = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(v[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

constexpr float kMagic = 12582912.0f;            // M = 1.5 * 2^23
constexpr float kMagicZ = 12582912.0f * 2049.0f; // M (1 + 2^11), exact in float
constexpr int kFxThreads = 256;
constexpr int kFxWarps = kFxThreads / 32;
constexpr int kFxGroup = 16;  // points a warp stages at a time
// Lane mapping: a warp takes one point at a time; lane (dz, dy, xh) adds the
// faces xh and xh + 2 of stencil row (dz, dy), one instruction per face pair
// and component.  With y stride 14 and z stride 168 the 16 row offsets
// 168 dz + 14 dy are the 16 even residues mod 32, so the 32 lanes of every
// atomic hit 32 distinct banks wherever the point lies.
constexpr int kFxSY = 14;
constexpr int kFxSZ = kB * kFxSY;       // 168
constexpr int kFxAcc = kB * kFxSZ;      // 2016 words per component

// The points a warp has staged, one array per field.  Each warp owns one
// group: staging needs no CTA barrier, only the warp's own __syncwarp.  The
// weight arrays are stencil-index major with rows padded by one record, so
// the staging stores of 16 consecutive points are contiguous and the per-point
// reads of the 2 or 4 distinct rows fall in distinct banks (one wavefront).
constexpr int kFxRow = kFxGroup + 1;
struct FxGroup {
  float4 val[kFxGroup];     // 2^k V^c * scale, c = 0..2; w: the packed stencil origin (fx_pack_origin)
  float2 wz[4][kFxRow];     // [dz][pt] = (w_z at s = 0, w_z at s = 1/2)
  float2 wy[4][kFxRow];     // [dy][pt] likewise
  float4 wx[2][kFxRow];     // [xh][pt] = (w_x(s 0)[xh], w_x(s 0)[xh + 2], w_x(s 1/2)[xh], w_x(s 1/2)[xh + 2])
};

// adds the contribution C = w wx (in units of 2^-k) at word offset a
__device__ __forceinline__ void fx_add(unsigned* hi, unsigned* lo, float w, float w11, float wx) {
  const float t1 = fmaf(w, wx, kMagic);
  const float z = fmaf(t1, -2048.0f, kMagicZ);
  const float t2 = fmaf(w11, wx, z);
  atomicAdd(hi, __float_as_uint(t1));
  atomicAdd(lo, __float_as_uint(t2));
}

// Fixed-point exponent k of the call: |C| = |V scale| prod phi < 2^19 in
// units of 2^-k, since every kernel weight product is at most 1/8.
__device__ __forceinline__ int fx_exponent(const SpreadArgs<float>& A) {
  const float cmax = 0.125f * __uint_as_float(*A.absmax) * fabsf(A.scale);
  int ex = 0;
  if (cmax > 0.f) frexpf(cmax, &ex);  // cmax < 2^ex
  return min(19 - ex, 100);           // keep 2^(k+11) a normal float
}

// The accumulator offsets of a stencil's first face, one per component, in
// 14 bits: with b_d the half-shifted (s = 1/2) start along axis d and g_d = 1
// when the unshifted (s = 0) start is one face further (0 otherwise),
// B = 168 b_z + 14 b_y + b_x < 2^11 and
//   o_0 = B + g_x,   o_1 = A + B + 14 g_y,   o_2 = 2 A + B + 168 g_z   (A = kFxAcc).
__device__ __forceinline__ int fx_pack_origin(const int b[3][2]) {
  const int B = b[2][1] * kFxSZ + b[1][1] * kFxSY + b[0][1];
  return B | (b[0][0] - b[0][1]) << 11 | (b[1][0] - b[1][1]) << 12 | (b[2][0] - b[2][1]) << 13;
}

// Raw data of one point, loaded a group ahead so that the loads are in
// flight while the warp accumulates the current group.
struct FxRaw {
  int32_t cell;
  float off[3];
  float val[3];
};

__device__ __forceinline__ void fx_fetch(const SpreadArgs<float>& A, int i, bool want_val,
                                         FxRaw& r) {
  r.cell = __ldg(A.p_cell + i);
#pragma unroll
  for (int d = 0; d < 3; ++d) r.off[d] = __ldg(A.p_off + d * A.Q + i);
  if (want_val) {
#pragma unroll
    for (int c = 0; c < 3; ++c) r.val[c] = __ldg(A.p_val + c * A.Q + i);
  }
}

// Lanes pt and pt + 16 stage point pt of the group: each evaluates three of
// the six 1-D weight sets (lane half 0: x at s = 0 and 1/2, y at s = 0;
// lane half 1: y at s = 1/2, z at s = 0 and 1/2), so both halves run the
// same instructions.
__device__ __forceinline__ void fx_stage(FxGroup& G, int pt, int part, const FxRaw& r,
                                         const int lc0[3], float vscale) {
  int cc[3];
  unpack_cell(r.cell, cc[0], cc[1], cc[2]);
  int b[3][2];
  float th[3][2];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) b[d][hf] = cc[d] - lc0[d] + stencil_axis(r.off[d], hf == 1, th[d][hf]) + 2;
  float wa[4], wb[4], wc[4];
  delta_weights(part ? th[1][1] : th[0][0], wa);
  delta_weights(part ? th[2][0] : th[0][1], wb);
  delta_weights(part ? th[2][1] : th[1][0], wc);
  if (part == 0) {
    G.wx[0][pt] = make_float4(wa[0], wa[2], wb[0], wb[2]);
    G.wx[1][pt] = make_float4(wa[1], wa[3], wb[1], wb[3]);
#pragma unroll
    for (int j = 0; j < 4; ++j) G.wy[j][pt].x = wc[j];
    G.val[pt] = make_float4(r.val[0] * vscale, r.val[1] * vscale, r.val[2] * vscale,
                            __int_as_float(fx_pack_origin(b)));
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      G.wy[j][pt].y = wa[j];
      G.wz[j][pt] = make_float2(wb[j], wc[j]);
    }
  }
}

__global__ void __launch_bounds__(kFxThreads) k_spread_push_fx(SpreadArgs<float> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FxGroup* groups = reinterpret_cast<FxGroup*>(smem_raw);
  unsigned* acc_hi = reinterpret_cast<unsigned*>(smem_raw + kFxWarps * sizeof(FxGroup));
  unsigned* acc_lo = acc_hi + 3 * kFxAcc;
  __shared__ int next;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int count = A.counters[0];
  const int nt0 = A.g.nt[0], nt1 = A.g.nt[1];
  // this lane's (dz, dy, xh) and its offset within a stencil
  const int ldz = lane >> 3, ldy = (lane >> 1) & 3, lxh = lane & 1;
  const int loff = ldz * kFxSZ + ldy * kFxSY + lxh;
  // this lane's staging role: point pt of the group, lane half `part`
  const int pt = lane & (kFxGroup - 1), part = lane >> 4;
  FxGroup& G = groups[warp];
  const int k = fx_exponent(A);
  const float vscale = A.scale * ldexpf(1.f, k);
  for (;;) {
    __syncthreads();  // previous item decoded
    if (tid == 0) next = atomicAdd(A.counters + 1, 1);
    __syncthreads();
    const int slot = next;
    if (slot >= count) break;
    const int tile = A.tile_list[slot];
    const int tx = tile % nt0, ty = (tile / nt0) % nt1, tz = tile / (nt0 * nt1);
    const int s = A.tile_start[tile] + (slot - A.tile_slot[tile]) * A.chunk;
    const int e = min(A.tile_end[tile], s + A.chunk);
    const int lc0[3] = {tx * kTile, ty * kTile, tz * kTile};
    // warp w takes the groups starting at s + 16 (w + 8 j)
    FxRaw raw;
    int g0 = s + warp * kFxGroup;
    if (g0 + pt < e) fx_fetch(A, g0 + pt, part == 0, raw);
    for (int i = tid; i < 3 * kFxAcc * 2 / 4; i += kFxThreads)
      reinterpret_cast<uint4*>(acc_hi)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();  // accumulators zeroed
    for (; g0 < e; g0 += kFxWarps * kFxGroup) {
      const int ng = min(kFxGroup, e - g0);
      if (pt < ng) fx_stage(G, pt, part, raw, lc0, vscale);
      __syncwarp();
      const int gn = g0 + kFxWarps * kFxGroup;
      if (gn + pt < e) fx_fetch(A, gn + pt, part == 0, raw);
      // one point per warp step: lane (dz, dy, xh) adds faces xh and xh + 2 of
      // its (dz, dy) row, for each component
      for (int q = 0; q < ng; ++q) {
        const float4 v = G.val[q];
        const int pk = __float_as_int(v.w);
        const int B = (pk & 0x7FF) + loff;
        const int4 org = make_int4(B + ((pk >> 11) & 1), kFxAcc + B + kFxSY * ((pk >> 12) & 1),
                                   2 * kFxAcc + B + kFxSZ * ((pk >> 13) & 1), 0);
        const float2 wz = G.wz[ldz][q], wy = G.wy[ldy][q];
        const float4 wx = G.wx[lxh][q];
        // component 0: z, y at s = 1/2, x at s = 0
        float wr = v.x * wz.y * wy.y;
        int a = org.x;
        fx_add(acc_hi + a, acc_lo + a, wr, wr * 2048.0f, wx.x);
        fx_add(acc_hi + a + 2, acc_lo + a + 2, wr, wr * 2048.0f, wx.y);
        // component 1: z at s = 1/2, y at s = 0, x at s = 1/2
        wr = v.y * wz.y * wy.x;
        a = org.y;
        fx_add(acc_hi + a, acc_lo + a, wr, wr * 2048.0f, wx.z);
        fx_add(acc_hi + a + 2, acc_lo + a + 2, wr, wr * 2048.0f, wx.w);
        // component 2: z at s = 0, y, x at s = 1/2
        wr = v.z * wz.x * wy.y;
        a = org.z;
        fx_add(acc_hi + a, acc_lo + a, wr, wr * 2048.0f, wx.z);
        fx_add(acc_hi + a + 2, acc_lo + a + 2, wr, wr * 2048.0f, wx.w);
      }
      __syncwarp();  // group consumed before it is restaged
    }
    __syncthreads();
    // decoded words (H, L) of every face, exact; consecutive threads take
    // consecutive face pairs of the 12-face x-rows (conflict-free reads,
    // contiguous 16-byte stores)
    int4* out = reinterpret_cast<int4*>(A.scratch) + (int64_t)slot * (kItemBlk / 2);
    for (int u = tid; u < 3 * kB * kB * (kB / 2); u += kFxThreads) {
      const int row = u / (kB / 2), x = 2 * (u % (kB / 2));
      const int c = row / (kB * kB), zy = row % (kB * kB);
      const int o = c * kFxAcc + (zy / kB) * kFxSZ + (zy % kB) * kFxSY + x;  // even: 8-byte aligned
      const uint2 hw = *reinterpret_cast<const uint2*>(acc_hi + o);
      const uint2 lw = *reinterpret_cast<const uint2*>(acc_lo + o);
      const int L0 = (int)(lw.x << 10) >> 10, L1 = (int)(lw.y << 10) >> 10;
      out[u] = make_int4((int)(hw.x - lw.x) + L0, L0, (int)(hw.y - lw.y) + L1, L1);
    }
  }
}

// Far tiles: one warp per tile, 3 components x 64 rows x 16-byte zeros.
template <typename Real>
__global__ void __launch_bounds__(kMT) k_spread_zero(SpreadArgs<Real> A) {
  const int lane = threadIdx.x & 31;
  const int tile = blockIdx.x * kMW + (threadIdx.x >> 5);
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

// FP32 plans: the same fixed-order walk over the covering blocks, summing the
// exact words of every face in integers (H in 64 bits, L in 32) and rounding
// once: S = 2^11 sum H + sum L is below 2^47, split as 2^24 hi + lo with both
// parts exact in float, so one fma gives the correctly rounded S, then scaled
// by 2^-(k+11).  The result does not depend on how a tile's points were cut
// into work items.
__global__ void __launch_bounds__(kMT) k_spread_merge_fx(SpreadArgs<float> A) {
  static_assert(kMT == 8 * 8 * 4, "one thread per face pair of a tile component");
  __shared__ int src_slot[27], src_n[27];
  const int tid = threadIdx.x;
  const int nt0 = A.g.nt[0], nt1 = A.g.nt[1];
  const int n0 = A.g.n[0], n1 = A.g.n[1];
  const int64_t cells = (int64_t)n0 * n1 * A.g.n[2];
  const int count = A.counters[3];
  const float out_scale = ldexpf(1.f, -(fx_exponent(A) + 11));
  const int4* scratch = reinterpret_cast<const int4*>(A.scratch);  // 2 faces per int4
  // this thread's faces: x = 2 xq and 2 xq + 1 of row (z, y), all three components
  const int z = tid >> 5, y = (tid >> 2) & 7, xq = tid & 3;
  const int ly = y <= 1 ? -1 : 0, lz = z <= 1 ? -1 : 0;
  const int hy = y >= 6 ? 1 : 0, hz = z >= 6 ? 1 : 0;
  // x neighbours: the left tile's block reaches faces 0, 1, the right one's 6, 7
  const int lx = xq == 0 ? -1 : 0, hx = xq == 3 ? 1 : 0;
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
    long long sh[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    int sl[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    for (int oz = lz; oz <= hz; ++oz)
      for (int oy = ly; oy <= hy; ++oy)
        for (int ox = lx; ox <= hx; ++ox) {
          // this face pair in the source tile's halo'd block (int4 units)
          const int q = ((z - oz * kTile + 2) * kB + (y - oy * kTile + 2)) * (kB / 2) + xq + 1 -
                        (kTile / 2) * ox;
          const int src = (oz + 1) * 9 + (oy + 1) * 3 + ox + 1;
          const int slt = src_slot[src], ns = src_n[src];
          const int4* r = scratch + (int64_t)slt * (kItemBlk / 2) + q;
#pragma unroll 2
          for (int j = 0; j < ns; ++j, r += kItemBlk / 2) {
            int4 v[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) v[c] = __ldg(r + c * (kBlk / 2));
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              sh[c][0] += v[c].x; sl[c][0] += v[c].y;
              sh[c][1] += v[c].z; sl[c][1] += v[c].w;
            }
          }
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float o[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const long long S = sh[c][i] * 2048 + sl[c][i];
        const int hi = (int)(S >> 24);  // |S| < 2^47: |hi| < 2^23, exact in float
        const int lo = (int)(S & 0xFFFFFF);
        o[i] = fmaf((float)hi, 16777216.0f, (float)lo) * out_scale;
      }
      float* row = A.f + c * cells + ((int64_t)(z0 + z) * n1 + (y0 + y)) * n0 + x0;
      reinterpret_cast<float2*>(row)[xq] = make_float2(o[0], o[1]);
    }
  }
}

template <typename Real>
size_t push_smem() {
  return sizeof(Staged<Real>) * kBatch + sizeof(Real) * kCopies * kAcc + sizeof(RawItem<Real>);
}

constexpr size_t kFxSmem = kFxWarps * sizeof(FxGroup) + sizeof(unsigned) * 2 * 3 * kFxAcc;

void launch_push(ib_plan* p, const SpreadArgs<float>& A, cudaStream_t s) {
  cudaMemsetAsync(p->tile_counters + 5, 0, sizeof(int32_t), s);
  if (p->Q > 0)
    k_absmax<<<p->sm_count * 4, 256, 0, s>>>((const float*)p->p_val, 3 * p->Q, A.absmax);
  p->prof_calls[IB_STAGE_SPREAD_PUSH] += 1;
  const int ev = prof_begin(p, IB_STAGE_SPREAD_PUSH, s);
  k_spread_push_fx<<<std::min(p->push_ctas, p->push_per_sm * p->sm_count), kFxThreads, kFxSmem,
                     s>>>(A);
  prof_end(p, ev, s);
}

void launch_push(ib_plan* p, const SpreadArgs<double>& A, cudaStream_t s) {
  k_spread_push<double><<<std::min(p->push_ctas, p->push_per_sm * p->sm_count), kPT,
                          push_smem<double>(), s>>>(A);
}

template <typename Real>
SpreadArgs<Real> spread_args(ib_plan* p, double scale, void* f) {
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
  A.chunk = p->chunk;
  A.scale = (Real)scale;
  A.scratch = (Real*)p->spread_scratch;
  A.f = (Real*)f;
  A.absmax = reinterpret_cast<uint32_t*>(p->tile_counters + 5);
  return A;
}

template <typename Real>
ib_status spread_t(ib_plan* p, double scale, void* f, bool zero_fill, cudaStream_t s) {
  SpreadArgs<Real> A = spread_args<Real>(p, scale, f);
  cudaMemsetAsync(p->tile_counters + 1, 0, sizeof(int32_t), s);
  // far-tile zeros on the side stream, concurrent with the push (unless the
  // caller has already issued them)
  if (zero_fill) {
    cudaEventRecord(p->ev_fork, s);
    cudaStreamWaitEvent(p->zside, p->ev_fork, 0);
    k_spread_zero<Real><<<(p->ntiles + kMW - 1) / kMW, kMT, 0, p->zside>>>(A);
    cudaEventRecord(p->ev_join, p->zside);
  }
  launch_push(p, A, s);
  if constexpr (sizeof(Real) == 4)
    k_spread_merge_fx<<<p->merge_ctas, kMT, 0, s>>>(A);
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
    e = cudaFuncSetAttribute(k_spread_push_fx, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kFxSmem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread_push_fx, kFxThreads,
                                                        kFxSmem);
  } else {
    const int smem = (int)push_smem<Real>();
    e = cudaFuncSetAttribute(k_spread_push<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread_push<Real>, kPT, smem);
  }
  if (e == cudaSuccess) {
    if constexpr (sizeof(Real) == 4)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_merge, k_spread_merge_fx, kMT, 0);
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
  // FP64: one double per face; FP32: the exact word pair (H, L) per face
  return (size_t)slots * kItemBlk * (precision == IB_FP64 ? sizeof(double) : sizeof(int2));
}

ib_status spread_prepare(ib_plan* p) {
  return p->precision == IB_FP64 ? prepare_t<double>(p) : prepare_t<float>(p);
}

int spread_launches() { return 4; }

ib_status launch_spread(ib_plan* p, double scale, void* f, cudaStream_t s, bool zero_fill) {
  return p->precision == IB_FP64 ? spread_t<double>(p, scale, f, zero_fill, s)
                                 : spread_t<float>(p, scale, f, zero_fill, s);
}

ib_status launch_spread_zero(ib_plan* p, void* f, cudaStream_t s) {
  if (p->precision == IB_FP64) {
    SpreadArgs<double> A = spread_args<double>(p, 1.0, f);
    k_spread_zero<double><<<(p->ntiles + kMW - 1) / kMW, kMT, 0, s>>>(A);
  } else {
    SpreadArgs<float> A = spread_args<float>(p, 1.0, f);
    k_spread_zero<float><<<(p->ntiles + kMW - 1) / kMW, kMT, 0, s>>>(A);
  }
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

}  // namespace ibfe
