// Classification of the 8^3-cell Eulerian tiles after the Gauss points have
// been sorted by tile:
//   non-empty  the tile holds points              -> spread push / interp work
//   near       a tile of its 3x3x3 neighbourhood holds points
//                                                   -> its faces are merged
//   far        otherwise                          -> its faces are zero
// A non-empty tile is cut into work items ("chunks") of at most kChunk
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

__global__ void __launch_bounds__(kT) k_classify(GridDev g, const int32_t* __restrict__ start,
                                                 const int32_t* __restrict__ end, int ntiles,
                                                 int32_t* __restrict__ nonempty,
                                                 int32_t* __restrict__ near,
                                                 int32_t* __restrict__ bcount) {
  __shared__ int tmp[32];
  const int t = blockIdx.x * kT + threadIdx.x;
  int ne = 0, nr = 0, nch = 0;
  if (t < ntiles) {
    const int nt0 = g.nt[0], nt1 = g.nt[1], nt2 = g.nt[2];
    const int tx = t % nt0, ty = (t / nt0) % nt1, tz = t / (nt0 * nt1);
    ne = end[t] > start[t];
    nch = (end[t] - start[t] + kChunk - 1) / kChunk;
    nr = ne;
    for (int a = -1; a <= 1 && !nr; ++a)
      for (int b = -1; b <= 1 && !nr; ++b)
        for (int c = -1; c <= 1 && !nr; ++c) {
          const int nb =
              wrap_idx(tx + c, nt0) + nt0 * (wrap_idx(ty + b, nt1) + nt1 * wrap_idx(tz + a, nt2));
          nr = end[nb] > start[nb];
        }
    nonempty[t] = nch;
    near[t] = nr;
  }
  int cne;
  block_exclusive_scan(nch, tmp, cne);
  const int cnr = __syncthreads_count(nr);
  if (threadIdx.x == 0) {
    bcount[2 * blockIdx.x] = cne;
    bcount[2 * blockIdx.x + 1] = cnr;
  }
}

// counters: [0] work items, [1] push / [2] interp work counters, [3] near tiles.
__global__ void __launch_bounds__(kT) k_compact(const int32_t* __restrict__ nonempty,
                                                const int32_t* __restrict__ near, int ntiles,
                                                const int32_t* __restrict__ bcount, int nblocks,
                                                int32_t* __restrict__ slot,
                                                int32_t* __restrict__ work,
                                                int32_t* __restrict__ list_near,
                                                int32_t* __restrict__ counters) {
  __shared__ int tmp[32];
  __shared__ int base[2];
  // offsets: sums of the counts of the CTAs before this one
  int ne_before = 0, nr_before = 0, ne_all = 0, nr_all = 0;
  for (int b = threadIdx.x; b < nblocks; b += kT) {
    const int a = bcount[2 * b], c = bcount[2 * b + 1];
    if (b < (int)blockIdx.x) {
      ne_before += a;
      nr_before += c;
    }
    ne_all += a;
    nr_all += c;
  }
  int t0, t1, t2, t3;
  block_exclusive_scan(ne_before, tmp, t0);
  block_exclusive_scan(nr_before, tmp, t1);
  block_exclusive_scan(ne_all, tmp, t2);
  block_exclusive_scan(nr_all, tmp, t3);
  if (threadIdx.x == 0) {
    base[0] = t0;
    base[1] = t1;
  }
  __syncthreads();
  const int t = blockIdx.x * kT + threadIdx.x;
  const int ne = t < ntiles ? nonempty[t] : 0;
  const int nr = t < ntiles ? near[t] : 0;
  int tot;
  const int pne = block_exclusive_scan(ne, tmp, tot);
  const int pnr = block_exclusive_scan(nr, tmp, tot);
  if (t < ntiles) {
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

int64_t max_work_items(int ntiles, int64_t Q) { return ntiles + Q / kChunk + 1; }

ib_status launch_classify_tiles(ib_plan* p, cudaStream_t s) {
  const int nt = p->ntiles, nb = classify_blocks(nt);
  k_classify<<<nb, kT, 0, s>>>(p->grid, p->tile_start, p->tile_end, nt, p->tile_nonempty,
                               p->tile_near, p->tile_bcount);
  k_compact<<<nb, kT, 0, s>>>(p->tile_nonempty, p->tile_near, nt, p->tile_bcount, nb,
                              p->tile_slot, p->tile_list, p->tile_list_near, p->tile_counters);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

}  // namespace ibfe
