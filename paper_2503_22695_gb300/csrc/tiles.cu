// Classification of the 8^3-cell Eulerian tiles after the Gauss points have
// been sorted by tile (the tiles of a packed plan are those of all its
// structures, each with the neighbours on its own periodic grid):
//   non-empty  the tile holds points              -> spread push / interp work
//   near       a tile of its 3x3x3 neighbourhood holds points
//                                                   -> its faces are merged
//   far        otherwise                          -> its faces are zero
// A non-empty tile is cut into work items ("chunks") of at most `chunk`
// consecutive points, so that a densely populated tile (mesh singularities
// concentrate points) is shared by several CTAs.  Work items are numbered in
// ascending (tile, chunk) order; a tile's first item number is its slot, and
// item k owns scratch block k.  Two kernels: per-CTA counts, then every CTA
// finds its output offsets from the counts of the CTAs before it and writes
// its part of the work list and of the near-tile list.
#include "ib_device.cuh"

namespace ibfe {
namespace {

constexpr int kT = 256;  // tiles per CTA

// Block-wide exclusive scans of K integers at once (one pair of barriers for
// all of them); total[k] receives the block sum of v[k].  tmp: K * 32 ints.
template <int K>
__device__ __forceinline__ void block_scan_k(const int (&v)[K], int (&pre)[K], int (&total)[K],
                                             int* tmp) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    x[k] = v[k];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(full, x[k], o);
      if (lane >= o) x[k] += y;
    }
    if (lane == 31) tmp[k * 32 + warp] = x[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      int w = lane < nw ? tmp[k * 32 + lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(full, w, o);
        if (lane >= o) w += y;
      }
      tmp[k * 32 + lane] = w;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    total[k] = tmp[k * 32 + nw - 1];
    pre[k] = (warp > 0 ? tmp[k * 32 + warp - 1] : 0) + x[k] - v[k];
  }
  __syncthreads();
}

// i in [-1, n]: its periodic image in [0, n)
__device__ __forceinline__ int wrap_one(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <bool kPacked>
__global__ void __launch_bounds__(kT) k_classify(GridDev g, const InstDev* __restrict__ inst,
                                                 const int32_t* __restrict__ tile_inst,
                                                 const int32_t* __restrict__ start,
                                                 const int32_t* __restrict__ end, int ntiles,
                                                 int32_t* __restrict__ nonempty,
                                                 int32_t* __restrict__ near,
                                                 int32_t* __restrict__ bcount, int chunk) {
  __shared__ int tmp[32];
  const int t = blockIdx.x * kT + threadIdx.x;
  int ne = 0, nr = 0, nch = 0, npt = 0;
  if (t < ntiles) {
    const TileGeo geo = tile_geo<kPacked>(g, inst, tile_inst, t);
    const int nt0 = geo.nt[0], nt1 = geo.nt[1], nt2 = geo.nt[2];
    int tx, ty, tz;
    tile_coords(geo, t, tx, ty, tz);
    npt = end[t] - start[t];
    ne = npt > 0;
    nch = (npt + chunk - 1) / chunk;
    // all 27 neighbours' ranges loaded at once (most tiles are far from the
    // structure and would otherwise wait for 27 dependent round trips)
    nr = 0;
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
      for (int b = -1; b <= 1; ++b)
#pragma unroll
        for (int c = -1; c <= 1; ++c) {
          const int nb = geo.base + wrap_one(tx + c, nt0) +
                         nt0 * (wrap_one(ty + b, nt1) + nt1 * wrap_one(tz + a, nt2));
          nr |= __ldg(end + nb) > __ldg(start + nb);
        }
    nonempty[t] = nch;
    near[t] = nr;
  }
  int cne, cpt;
  block_exclusive_scan(nch, tmp, cne);
  block_exclusive_scan(npt, tmp, cpt);
  const int cnr = __syncthreads_count(nr);
  if (threadIdx.x == 0) {
    bcount[3 * blockIdx.x] = cne;
    bcount[3 * blockIdx.x + 1] = cnr;
    bcount[3 * blockIdx.x + 2] = cpt;
  }
}

// counters: [0] work items, [1] push / [2] interp work counters, [3] near tiles.
// Also rewrites the tile point ranges as start = points of the tiles before,
// end = start + points (the same ranges for sorted points; the ranges
// themselves for binned points, whose counts arrive as start 0, end n).
__global__ void __launch_bounds__(kT) k_compact(const int32_t* __restrict__ nonempty,
                                                const int32_t* __restrict__ near, int ntiles,
                                                const int32_t* __restrict__ bcount, int nblocks,
                                                int32_t* __restrict__ start,
                                                int32_t* __restrict__ end,
                                                int32_t* __restrict__ slot,
                                                int32_t* __restrict__ work,
                                                int32_t* __restrict__ list_near,
                                                int32_t* __restrict__ counters) {
  __shared__ int tmp[5 * 32];
  __shared__ int base[3];
  // offsets: sums of the counts of the CTAs before this one (and of all)
  int sums[5] = {0, 0, 0, 0, 0};  // ne, nr, np before this CTA; ne, nr of all
  for (int b = threadIdx.x; b < nblocks; b += kT) {
    const int a = bcount[3 * b], c = bcount[3 * b + 1], d = bcount[3 * b + 2];
    if (b < (int)blockIdx.x) {
      sums[0] += a;
      sums[1] += c;
      sums[2] += d;
    }
    sums[3] += a;
    sums[4] += c;
  }
  int spre[5], stot[5];
  block_scan_k<5>(sums, spre, stot, tmp);
  const int t2 = stot[3], t3 = stot[4];
  if (threadIdx.x == 0) {
    base[0] = stot[0];
    base[1] = stot[1];
    base[2] = stot[2];
  }
  __syncthreads();
  const int t = blockIdx.x * kT + threadIdx.x;
  const int cnt[3] = {t < ntiles ? nonempty[t] : 0, t < ntiles ? near[t] : 0,
                      t < ntiles ? end[t] - start[t] : 0};
  const int ne = cnt[0], nr = cnt[1], np = cnt[2];
  int cpre[3], ctot[3];
  block_scan_k<3>(cnt, cpre, ctot, tmp);
  const int pne = cpre[0], pnr = cpre[1], pnp = cpre[2];
  if (t < ntiles) {
    start[t] = base[2] + pnp;
    end[t] = base[2] + pnp + np;
    slot[t] = ne ? base[0] + pne : -1;
    for (int j = 0; j < ne; ++j) work[base[0] + pne + j] = t;
    if (nr) list_near[base[1] + pnr] = t;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    counters[0] = t2;
    counters[1] = 0;
    counters[2] = 0;
    counters[3] = t3;
  }
}

}  // namespace

int classify_blocks(int ntiles) { return (ntiles + kT - 1) / kT; }

int64_t max_work_items(int ntiles, int64_t Q) { return ntiles + Q / kMinChunk + 1; }

ib_status launch_classify_tiles(ib_plan* p, cudaStream_t s) {
  const int nt = p->ntiles, nb = classify_blocks(nt);
  auto classify = p->n_inst > 1 ? k_classify<true> : k_classify<false>;
  classify<<<nb, kT, 0, s>>>(p->grid, p->inst, p->tile_inst, p->tile_start, p->tile_end, nt,
                             p->tile_nonempty, p->tile_near, p->tile_bcount, p->chunk);
  k_compact<<<nb, kT, 0, s>>>(p->tile_nonempty, p->tile_near, nt, p->tile_bcount, nb,
                              p->tile_start, p->tile_end, p->tile_slot, p->tile_list,
                              p->tile_list_near, p->tile_counters);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

}  // namespace ibfe
