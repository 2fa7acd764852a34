// Spreading of Gauss-point values onto the periodic MAC grid (Section 4.4):
//   f^c(face) = scale * sum_q V_q^c prod_d phi(r_d),   r_d = (chi_q,d - x_face,d)/h,
// with scale = h^-3 for forces (delta_h carries h^-3) and 1 for the adjoint
// of interpolation.
//
// Design: every 8x8x8-cell Eulerian tile is owned by one CTA, which computes
// all three components of its 3*512 faces and writes each exactly once, so
// the whole field (including the zero-fill outside the structure) is written
// in one pass with no global atomics.  The CTA pulls the points binned in its
// tile and in the neighbouring tiles (a point's stencil reaches two cells
// beyond its own cell) in a fixed order: neighbour tiles in (z, y, x) order,
// points in sorted order within a tile.  Point k of that sequence goes to
// warp k mod W; each warp accumulates into its own shared-memory copy of the
// tile, one point at a time, its 32 lanes covering the 48 (component, dz, dy)
// rows of the 4x4x4 stencil (the four dx entries of a row by one lane), so no
// two lanes touch the same face in one step.  The W copies are then summed in
// warp order.  Every face therefore sees its contributions in a fixed order,
// and the result is bitwise reproducible.
#include "ib_device.cuh"

namespace ibfe {
namespace {

constexpr int W = kSpreadWarps;
constexpr int kZS = 66;                    // z stride (bank spread across (z,y))
constexpr int kCS = kTile * kZS + 1;       // component stride
constexpr int kWS = 3 * kCS + 1;           // warp stride

template <typename Real>
struct SpreadArgs {
  GridDev g;
  int64_t Q;
  const int32_t* tile_start;
  const int32_t* tile_end;
  const int32_t* p_cell;
  const Real* p_off;
  const Real* p_val;
  Real scale;
  Real* f;
};

template <typename Real>
__device__ __forceinline__ Real pick4(const Real w[4], int i) {
  return i == 0 ? w[0] : (i == 1 ? w[1] : (i == 2 ? w[2] : w[3]));
}

template <typename Real>
__global__ void __launch_bounds__(W * 32) k_spread(SpreadArgs<Real> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* acc = reinterpret_cast<Real*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n0 = A.g.n[0], n1 = A.g.n[1], n2 = A.g.n[2];
  const int nt0 = A.g.nt[0], nt1 = A.g.nt[1], nt2 = A.g.nt[2];
  const int tile = blockIdx.x;
  const int tx = tile % nt0, ty = (tile / nt0) % nt1, tz = tile / (nt0 * nt1);
  const int64_t cells = (int64_t)n0 * n1 * n2;

  // neighbour tiles, deduplicated when a dimension has fewer than 3 tiles
  int offs[3][3], cnt[3];
  const int ntd[3] = {nt0, nt1, nt2};
  for (int d = 0; d < 3; ++d) {
    if (ntd[d] >= 3) {
      cnt[d] = 3;
      offs[d][0] = -1; offs[d][1] = 0; offs[d][2] = 1;
    } else if (ntd[d] == 2) {
      cnt[d] = 2;
      offs[d][0] = 0; offs[d][1] = 1;
    } else {
      cnt[d] = 1;
      offs[d][0] = 0;
    }
  }
  int total = 0;
  for (int a = 0; a < cnt[2]; ++a)
    for (int b = 0; b < cnt[1]; ++b)
      for (int c = 0; c < cnt[0]; ++c) {
        const int nb = wrap_idx(tx + offs[0][c], nt0) +
                       nt0 * (wrap_idx(ty + offs[1][b], nt1) + nt1 * wrap_idx(tz + offs[2][a], nt2));
        total += A.tile_end[nb] - A.tile_start[nb];
      }

  const int x0 = tx * kTile, y0 = ty * kTile, z0 = tz * kTile;
  if (total == 0) {  // nothing reaches this tile: zero-fill
    for (int idx = tid; idx < 3 * 512; idx += W * 32) {
      const int c = idx >> 9, r = idx & 511;
      const int z = r >> 6, y = (r >> 3) & 7, x = r & 7;
      A.f[c * cells + ((int64_t)(z0 + z) * n1 + (y0 + y)) * n0 + (x0 + x)] = Real(0);
    }
    return;
  }

  for (int i = tid; i < W * kWS; i += W * 32) acc[i] = Real(0);
  __syncthreads();
  Real* my = acc + warp * kWS;

  int k0 = 0;
  for (int a = 0; a < cnt[2]; ++a)
    for (int b = 0; b < cnt[1]; ++b)
      for (int c = 0; c < cnt[0]; ++c) {
        const int nb = wrap_idx(tx + offs[0][c], nt0) +
                       nt0 * (wrap_idx(ty + offs[1][b], nt1) + nt1 * wrap_idx(tz + offs[2][a], nt2));
        const int s = A.tile_start[nb], e = A.tile_end[nb];
        const int first = ((warp - k0) % W + W) % W;
        for (int i = s + first; i < e; i += W) {
          const int32_t pc = __ldg(A.p_cell + i);
          int cx, cy, cz;
          unpack_cell(pc, cx, cy, cz);
          const Real ox = __ldg(A.p_off + i), oy = __ldg(A.p_off + A.Q + i),
                     oz = __ldg(A.p_off + 2 * A.Q + i);
          const Real v0 = __ldg(A.p_val + i), v1 = __ldg(A.p_val + A.Q + i),
                     v2 = __ldg(A.p_val + 2 * A.Q + i);
#pragma unroll
          for (int rr = 0; rr < 2; ++rr) {
            const int row = lane + 32 * rr;
            if (row >= 48) break;
            const int comp = row >> 4, dz = (row >> 2) & 3, dy = row & 3;
            Real th;
            const int sz = stencil_axis(oz, comp != 2, th);
            const int rz = wrap_idx(cz + sz + dz, n2) - z0;
            if ((unsigned)rz >= (unsigned)kTile) continue;
            Real wz4[4];
            delta_weights(th, wz4);
            const int sy = stencil_axis(oy, comp != 1, th);
            const int ry = wrap_idx(cy + sy + dy, n1) - y0;
            if ((unsigned)ry >= (unsigned)kTile) continue;
            Real wy4[4];
            delta_weights(th, wy4);
            const int sx = stencil_axis(ox, comp != 0, th);
            Real wx4[4];
            delta_weights(th, wx4);
            const Real v = comp == 0 ? v0 : (comp == 1 ? v1 : v2);
            const Real base = v * A.scale * pick4(wz4, dz) * pick4(wy4, dy);
            Real* rowp = my + comp * kCS + rz * kZS + ry * kTile;
#pragma unroll
            for (int dx = 0; dx < 4; ++dx) {
              const int rx = wrap_idx(cx + sx + dx, n0) - x0;
              if ((unsigned)rx < (unsigned)kTile) rowp[rx] += base * wx4[dx];
            }
          }
        }
        k0 += e - s;
      }
  __syncthreads();
  for (int idx = tid; idx < 3 * 512; idx += W * 32) {
    const int c = idx >> 9, r = idx & 511;
    const int z = r >> 6, y = (r >> 3) & 7, x = r & 7;
    const int o = c * kCS + z * kZS + y * kTile + x;
    Real sum = Real(0);
#pragma unroll
    for (int w = 0; w < W; ++w) sum += acc[w * kWS + o];
    A.f[c * cells + ((int64_t)(z0 + z) * n1 + (y0 + y)) * n0 + (x0 + x)] = sum;
  }
}

template <typename Real>
ib_status spread_t(ib_plan* p, double scale, void* f, cudaStream_t s) {
  SpreadArgs<Real> A;
  A.g = p->grid;
  A.Q = p->Q;
  A.tile_start = p->tile_start;
  A.tile_end = p->tile_end;
  A.p_cell = p->p_cell;
  A.p_off = (const Real*)p->p_off;
  A.p_val = (const Real*)p->p_val;
  A.scale = (Real)scale;
  A.f = (Real*)f;
  const size_t smem = sizeof(Real) * W * kWS;
  static bool attr_set[2] = {false, false};
  const int which = sizeof(Real) == 8;
  if (!attr_set[which]) {
    if (cudaFuncSetAttribute(k_spread<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return IB_ERR_CUDA;
    attr_set[which] = true;
  }
  k_spread<Real><<<p->ntiles, W * 32, smem, s>>>(A);
  return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ERR_CUDA;
}

}  // namespace

ib_status launch_spread(ib_plan* p, double scale, void* f, cudaStream_t s) {
  return p->precision == IB_FP64 ? spread_t<double>(p, scale, f, s)
                                 : spread_t<float>(p, scale, f, s);
}

}  // namespace ibfe
