// Batched form (a parameter sweep over independent structures): hexahedral
// meshes of uneven sizes, each on its own periodic grid with its own
// materials, run as ONE packed plan.
//
// At creation the instances' meshes are laid end to end (node, element and
// material ids offset by the instances before), their grids' 8^3-cell tiles
// are numbered consecutively, and device tables give every tile and element
// its instance (grid sizes, first tile, h), every material id its row and
// its element range.  Each stage of the coupling is then one launch over the
// whole batch: one force launch over all elements, one binning of all Gauss
// points into all instances' tiles, one persistent accumulation kernel whose
// work counter hands out the (tile, chunk) items of every instance, one
// merge over every near tile, one persistent interpolation, one gather per
// nodal result.  What differs per instance inside a stage -- the output or
// input grid array, the h-dependent scale, the tensor map of the staged
// field -- is read from per-call tables indexed by the tile's instance.  The
// instances' positions and nodal inputs are gathered into packed arrays by
// one kernel and the nodal outputs scattered back by another; the forward
// and the backward sequences (those of ib_forward and ib_backward) are each
// captured once in a CUDA graph and replayed with one launch.
//
// Each instance's arithmetic is the one a plan of that structure alone
// performs: the same element computations; per-tile fixed-point exponents,
// exact sums and merge alignment that depend on the tile's own points only
// (not on how the tuning cuts them into work items); per-point
// interpolation; node gathers over the same incident elements in the same
// order; reduction trees over each material's own element range.  So every
// instance's results are bitwise those of ib_forward / ib_backward on it.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ib_device.cuh"

namespace ibfe {
namespace {

// One instance's nodal arrays (the caller's) and its range of packed nodes.
struct NodeSeg {
  int base, count;
  const int32_t* cell;  // positions [3][count]
  const float* off;
  float* G;             // forward outputs [3][count]
  float* U;
  const float* Gin;     // backward inputs [3][count] (gG may be null: zero)
  const float* gU;
  const float* gG;
  float* gx;            // backward output
};

enum : int { kPackPos = 0, kUnpackFwd = 1, kPackAdj = 2, kUnpackAdj = 3 };

// Packed nodal arrays <-> the instances' own: blockIdx.y is the instance,
// one thread per node and three components.
template <int kMode>
__global__ void __launch_bounds__(256) k_nodes(const NodeSeg* __restrict__ segs, int64_t N,
                                               int32_t* __restrict__ cell, float* __restrict__ a,
                                               float* __restrict__ b, float* __restrict__ c) {
  const NodeSeg sg = segs[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sg.count) return;
  const int64_t n = sg.count, j = (int64_t)sg.base + i;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (kMode == kPackPos) {
      cell[d * N + j] = sg.cell[d * n + i];
      a[d * N + j] = sg.off[d * n + i];
    } else if (kMode == kUnpackFwd) {
      sg.G[d * n + i] = a[d * N + j];
      sg.U[d * n + i] = b[d * N + j];
    } else if (kMode == kPackAdj) {
      a[d * N + j] = sg.Gin[d * n + i];
      b[d * N + j] = sg.gU[d * n + i];
      if (c) c[d * N + j] = sg.gG ? sg.gG[d * n + i] : 0.f;
    } else {
      sg.gx[d * n + i] = a[d * N + j];
    }
  }
}

// Parameter gradients of the packed material rows to [n][IB_MAX_MATERIALS]
// rows per instance (zero past an instance's materials).
__global__ void k_gparams(const double* __restrict__ ered, const int2* __restrict__ mats,
                          double* __restrict__ out) {
  const int i = blockIdx.x;
  const int2 m = mats[i];  // (first packed row, rows)
  for (int k = threadIdx.x; k < IB_MAX_MATERIALS * kParamRow; k += blockDim.x) {
    const int r = k / kParamRow;
    out[(int64_t)i * IB_MAX_MATERIALS * kParamRow + k] =
        r < m.y ? ered[(int64_t)(m.x + r) * kParamRow + k % kParamRow] : 0.0;
  }
}

bool ok(cudaError_t e) { return e == cudaSuccess; }

template <typename T>
bool dalloc(T** p, size_t bytes) {
  *p = nullptr;
  return ok(cudaMalloc((void**)p, bytes ? bytes : 16));
}

}  // namespace
}  // namespace ibfe

using namespace ibfe;

struct ib_batch {
  int n = 0;
  std::vector<ib_instance> inst;
  ib_plan* P = nullptr;
  int64_t N = 0, E = 0;
  int max_nodes = 0;
  double gunit = 1.0;
  // packed mesh (owned; the plan refers to it)
  int32_t* conn = nullptr;
  float* X = nullptr;
  float* fib = nullptr;
  int32_t* mat_id = nullptr;
  // packed nodal arrays
  int32_t* cell = nullptr;
  float* off = nullptr;
  float *G = nullptr, *U = nullptr, *Gin = nullptr, *gU = nullptr, *gG = nullptr, *gx = nullptr;
  bool any_gG = false;
  NodeSeg* segs = nullptr;
  int2* gp_rows = nullptr;    // per instance: first packed material row, rows
  double* gparams = nullptr;  // [n][IB_MAX_MATERIALS][kParamRow]
  GridCall* calls = nullptr;  // 5 tables of n rows
  void* tmaps = nullptr;      // 2 tables of n tensor maps (u, gf), or null
  PackedCalls pc = {};
  cudaStream_t cap = nullptr;
  cudaGraphExec_t fwd = nullptr, adj = nullptr;
  bool has_adj = false;
};

namespace {

void destroy(ib_batch* b) {
  if (!b) return;
  if (b->fwd) cudaGraphExecDestroy(b->fwd);
  if (b->adj) cudaGraphExecDestroy(b->adj);
  if (b->P) plan_free(b->P);
  void* ptrs[] = {b->conn, b->X, b->fib, b->mat_id, b->cell, b->off, b->G, b->U, b->Gin,
                  b->gU, b->gG, b->gx, b->segs, b->gp_rows, b->gparams, b->calls, b->tmaps};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

ib_pos packed_pos(const ib_batch* b) {
  ib_pos x;
  x.cell = b->cell;
  x.off = b->off;
  x.x64 = nullptr;
  x.grad_unit = b->gunit;
  return x;
}

dim3 node_grid(const ib_batch* b) { return dim3((b->max_nodes + 255) / 256, b->n); }

ib_status run_forward(ib_batch* b, cudaStream_t s) {
  const ib_pos x = packed_pos(b);
  MatTable none;
  std::memset(&none, 0, sizeof(none));
  k_nodes<kPackPos><<<node_grid(b), 256, 0, s>>>(b->segs, b->N, b->cell, b->off, nullptr, nullptr);
  ib_status st = forward_body(b->P, none, &x, b->inst[0].u, b->G, b->inst[0].f, b->U, s, &b->pc);
  if (st == IB_OK)
    k_nodes<kUnpackFwd><<<node_grid(b), 256, 0, s>>>(b->segs, b->N, nullptr, b->G, b->U, nullptr);
  return st == IB_OK && ok(cudaGetLastError()) ? IB_OK : (st == IB_OK ? IB_ERR_CUDA : st);
}

ib_status run_adjoint(ib_batch* b, cudaStream_t s) {
  const ib_pos x = packed_pos(b);
  MatTable none;
  std::memset(&none, 0, sizeof(none));
  k_nodes<kPackPos><<<node_grid(b), 256, 0, s>>>(b->segs, b->N, b->cell, b->off, nullptr, nullptr);
  k_nodes<kPackAdj><<<node_grid(b), 256, 0, s>>>(b->segs, b->N, nullptr, b->Gin, b->gU,
                                                 b->any_gG ? b->gG : nullptr);
  // the instances' own fields come from the call tables; the pointers passed
  // here only mark which adjoint terms are wanted
  const ib_instance& i0 = b->inst[0];
  ib_status st = backward_body(b->P, none, b->P->n_mats_dev, &x, i0.u, b->Gin,
                               b->any_gG ? b->gG : nullptr, i0.gf, b->gU, b->gx, i0.gu,
                               /*params=*/true, nullptr, s, &b->pc);
  if (st == IB_OK) {
    k_gparams<<<b->n, 128, 0, s>>>(b->P->ered, b->gp_rows, b->gparams);
    k_nodes<kUnpackAdj><<<node_grid(b), 256, 0, s>>>(b->segs, b->N, nullptr, b->gx, nullptr,
                                                     nullptr);
  }
  return st == IB_OK && ok(cudaGetLastError()) ? IB_OK : (st == IB_OK ? IB_ERR_CUDA : st);
}

ib_status capture(ib_batch* b, ib_status (*fn)(ib_batch*, cudaStream_t), cudaGraphExec_t* out) {
  if (!ok(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal))) return IB_ERR_CUDA;
  ib_status st = fn(b, b->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(b->cap, &g);
  if (st == IB_OK && ec != cudaSuccess) st = IB_ERR_CUDA;
  if (st == IB_OK && !ok(cudaGraphInstantiate(out, g, 0))) st = IB_ERR_CUDA;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  return st;
}

// Host validation of one instance.
ib_status check_instance(const ib_instance& in) {
  const ib_mesh& m = in.mesh;
  if (m.elem_type != IB_ELEM_HEX8 || m.n_nodes <= 0 || m.n_elems <= 0 || !m.conn || !m.X)
    return IB_ERR_INVALID_ARG;
  const ib_status gs = check_grid(&in.grid);
  if (gs != IB_OK) return gs;
  if (in.n_mats <= 0 || in.n_mats > IB_MAX_MATERIALS) return IB_ERR_INVALID_ARG;
  for (int k = 0; k < in.n_mats; ++k)
    if (!material_valid(in.mats[k])) return IB_ERR_INVALID_ARG;
  if (!in.x.cell || !in.x.off || !std::isfinite(in.x.grad_unit) || in.x.grad_unit < 0.0)
    return IB_ERR_INVALID_ARG;
  if (!in.u || !in.G || !in.f || !in.U) return IB_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(in.f) & 15) || (reinterpret_cast<uintptr_t>(in.u) & 15))
    return IB_ERR_INVALID_ARG;
  return IB_OK;
}

// The packed mesh, plan, tables and buffers of a batch.
ib_status build(ib_batch* b, cudaStream_t s) {
  const int n = b->n;
  std::vector<int> nb(n + 1, 0), eb(n + 1, 0), tb(n + 1, 0), mb(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const ib_instance& in = b->inst[i];
    nb[i + 1] = nb[i] + in.mesh.n_nodes;
    eb[i + 1] = eb[i] + in.mesh.n_elems;
    tb[i + 1] = tb[i] + (in.grid.n[0] / kTile) * (in.grid.n[1] / kTile) * (in.grid.n[2] / kTile);
    mb[i + 1] = mb[i] + in.n_mats;
    b->max_nodes = std::max(b->max_nodes, in.mesh.n_nodes);
  }
  const int64_t N = nb[n], E = eb[n];
  if (N >= (1LL << 31) || E >= (1LL << 31) / 8) return IB_ERR_CAPACITY;
  b->N = N;
  b->E = E;
  // connectivity and material ids offset on the host
  std::vector<int32_t> conn(8 * E), mid(E), einst(E), tinst(tb[n]);
  bool any_fib = false;
  for (int i = 0; i < n; ++i) {
    const ib_instance& in = b->inst[i];
    const int Ei = in.mesh.n_elems;
    std::vector<int32_t> ci(8 * (size_t)Ei), mi(Ei, 0);
    if (!ok(cudaMemcpyAsync(ci.data(), in.mesh.conn, 4 * ci.size(), cudaMemcpyDeviceToHost, s)) ||
        (in.mesh.mat_id && !ok(cudaMemcpyAsync(mi.data(), in.mesh.mat_id, 4 * (size_t)Ei,
                                               cudaMemcpyDeviceToHost, s))) ||
        !ok(cudaStreamSynchronize(s)))
      return IB_ERR_CUDA;
    for (int a = 0; a < 8; ++a)
      for (int e = 0; e < Ei; ++e) {
        const int32_t v = ci[(size_t)a * Ei + e];
        if (v < 0 || v >= in.mesh.n_nodes) return IB_ERR_INVALID_ARG;
        conn[(size_t)a * E + eb[i] + e] = v + nb[i];
      }
    for (int e = 0; e < Ei; ++e) {
      if (mi[e] < 0 || mi[e] >= in.n_mats) return IB_ERR_INVALID_ARG;
      mid[eb[i] + e] = mi[e] + mb[i];
      einst[eb[i] + e] = i;
    }
    for (int t = tb[i]; t < tb[i + 1]; ++t) tinst[t] = i;
    any_fib = any_fib || in.mesh.fibres;
  }
  // the instance table, material rows and ranges, call tables
  std::vector<InstDev> idev(n);
  std::vector<MatRow> rows(mb[n]);
  std::vector<int2> ranges(mb[n]), gp_rows(n);
  std::vector<GridCall> calls(5 * (size_t)n);
  std::vector<NodeSeg> segs(n);
  int need = 0;
  for (int i = 0; i < n; ++i) {
    const ib_instance& in = b->inst[i];
    InstDev& r = idev[i];
    for (int d = 0; d < 3; ++d) {
      r.n[d] = in.grid.n[d];
      r.nt[d] = in.grid.n[d] / kTile;
    }
    r.tile_base = tb[i];
    r.pad = 0;
    r.h = in.grid.h;
    for (int m = 0; m < in.n_mats; ++m) {
      MatRow& w = rows[mb[i] + m];
      std::memset(&w, 0, sizeof(w));
      w.model = in.mats[m].model;
      for (int k = 0; k < in.mats[m].n_params; ++k) w.p[k] = in.mats[m].params[k];
      w.p[kTa] = in.mats[m].Ta;
      mat_entry_finish(w.p, w.pf, w.act);
      need |= 1 << w.model;
      if (w.p[kTa] != 0.0) need |= kLawAct;
      ranges[mb[i] + m] = make_int2(eb[i], eb[i + 1]);
    }
    gp_rows[i] = make_int2(mb[i], in.n_mats);
    // the scalars the single-structure sequences compute from h
    const double h = in.grid.h, ih3 = 1.0 / (h * h * h), gxu = b->gunit;
    calls[0 * n + i] = GridCall{in.f, ih3, 0.0};                        // spread_f
    calls[1 * n + i] = GridCall{const_cast<void*>(in.u), 1.0, 0.0};     // interp_u
    calls[2 * n + i] = GridCall{const_cast<void*>(in.gf), ih3, ih3 / h * gxu};  // interp_gf
    calls[3 * n + i] = GridCall{in.gu, 1.0, 0.0};                       // spread_gu
    calls[4 * n + i] = GridCall{const_cast<void*>(in.u), 0.0, gxu / h}; // interp_ug
    NodeSeg& g = segs[i];
    g.base = nb[i];
    g.count = in.mesh.n_nodes;
    g.cell = in.x.cell;
    g.off = in.x.off;
    g.G = static_cast<float*>(in.G);
    g.U = static_cast<float*>(in.U);
    g.Gin = static_cast<const float*>(in.G);
    g.gU = static_cast<const float*>(in.gU);
    g.gG = static_cast<const float*>(in.gG);
    g.gx = static_cast<float*>(in.gx);
  }
  // tensor maps of every instance's u and gf (TMA staging), if all encode
  std::vector<unsigned char> maps(2 * (size_t)n * kTensorMapBytes);
  bool tma = true;
  for (int i = 0; i < n && tma; ++i) {
    const ib_instance& in = b->inst[i];
    tma = encode_velocity_map(in.grid.n, in.u, &maps[(size_t)i * kTensorMapBytes]) &&
          (!b->has_adj ||
           encode_velocity_map(in.grid.n, in.gf, &maps[(size_t)(n + i) * kTensorMapBytes]));
  }
  // device copies
  const size_t n3 = 3 * (size_t)N;
  bool good = dalloc(&b->conn, 4 * 8 * (size_t)E) && dalloc(&b->X, 4 * n3) &&
              (!any_fib || dalloc(&b->fib, 4 * 6 * (size_t)E)) && dalloc(&b->mat_id, 4 * E) &&
              dalloc(&b->cell, 4 * n3) && dalloc(&b->off, 4 * n3) && dalloc(&b->G, 4 * n3) &&
              dalloc(&b->U, 4 * n3) && dalloc(&b->Gin, 4 * n3) && dalloc(&b->gU, 4 * n3) &&
              dalloc(&b->gG, 4 * n3) && dalloc(&b->gx, 4 * n3) &&
              dalloc(&b->segs, sizeof(NodeSeg) * n) && dalloc(&b->gp_rows, sizeof(int2) * n) &&
              dalloc(&b->gparams, sizeof(double) * kParamRow * IB_MAX_MATERIALS * n) &&
              dalloc(&b->calls, sizeof(GridCall) * calls.size()) &&
              (!tma || dalloc(&b->tmaps, maps.size()));
  if (!good) return IB_ERR_CUDA;
  good = ok(cudaMemcpyAsync(b->conn, conn.data(), 4 * conn.size(), cudaMemcpyHostToDevice, s)) &&
         ok(cudaMemcpyAsync(b->mat_id, mid.data(), 4 * mid.size(), cudaMemcpyHostToDevice, s)) &&
         ok(cudaMemcpyAsync(b->segs, segs.data(), sizeof(NodeSeg) * n, cudaMemcpyHostToDevice, s)) &&
         ok(cudaMemcpyAsync(b->gp_rows, gp_rows.data(), sizeof(int2) * n, cudaMemcpyHostToDevice,
                            s)) &&
         ok(cudaMemsetAsync(b->gparams, 0, sizeof(double) * kParamRow * IB_MAX_MATERIALS * n, s)) &&
         ok(cudaMemcpyAsync(b->calls, calls.data(), sizeof(GridCall) * calls.size(),
                            cudaMemcpyHostToDevice, s)) &&
         (!tma || ok(cudaMemcpyAsync(b->tmaps, maps.data(), maps.size(), cudaMemcpyHostToDevice, s)));
  // reference coordinates and fibres, one strided copy per instance (the
  // default fibre pair e_x, e_y for instances without fibres)
  std::vector<float> defib;
  for (int i = 0; i < n && good; ++i) {
    const ib_instance& in = b->inst[i];
    const size_t Ni = in.mesh.n_nodes, Ei = in.mesh.n_elems;
    good = ok(cudaMemcpy2DAsync(b->X + nb[i], 4 * N, in.mesh.X, 4 * Ni, 4 * Ni, 3,
                                cudaMemcpyDeviceToDevice, s));
    if (good && any_fib) {
      const void* src = in.mesh.fibres;
      if (!src) {
        defib.assign(6 * Ei, 0.f);
        std::fill(defib.begin(), defib.begin() + Ei, 1.f);
        std::fill(defib.begin() + 4 * Ei, defib.begin() + 5 * Ei, 1.f);
        src = defib.data();
      }
      good = ok(cudaMemcpy2DAsync(b->fib + eb[i], 4 * E, src, 4 * Ei, 4 * Ei, 6,
                                  in.mesh.fibres ? cudaMemcpyDeviceToDevice
                                                 : cudaMemcpyHostToDevice, s)) &&
             ok(cudaStreamSynchronize(s));
    }
  }
  if (!good || !ok(cudaStreamSynchronize(s))) return IB_ERR_CUDA;
  // the packed plan over the packed mesh
  ib_mesh pm;
  pm.n_nodes = (int32_t)N;
  pm.n_elems = (int32_t)E;
  pm.conn = b->conn;
  pm.X = b->X;
  pm.fibres = b->fib;
  pm.mat_id = b->mat_id;
  pm.elem_type = IB_ELEM_HEX8;
  const ib_instance& i0 = b->inst[0];
  GridDev g0;
  for (int d = 0; d < 3; ++d) {
    g0.n[d] = i0.grid.n[d];
    g0.nt[d] = i0.grid.n[d] / kTile;
    g0.origin[d] = i0.grid.origin[d];
  }
  g0.h = i0.grid.h;
  ib_status st =
      plan_build(&pm, g0, tb[n], IB_QUAD_GAUSS2, IB_FP32_SPLIT, mb[n], s, &b->P, /*packed=*/true);
  if (st != IB_OK) return st;
  ib_plan* P = b->P;
  P->n_inst = n;
  P->n_mats_dev = mb[n];
  P->mat_need = need;
  good = dalloc(&P->inst, sizeof(InstDev) * n) && dalloc(&P->tile_inst, 4 * (size_t)tb[n]) &&
         dalloc(&P->elem_inst, 4 * (size_t)E) && dalloc(&P->mat_dev, sizeof(MatRow) * mb[n]) &&
         ok(cudaMemcpyAsync(P->inst, idev.data(), sizeof(InstDev) * n, cudaMemcpyHostToDevice, s)) &&
         ok(cudaMemcpyAsync(P->tile_inst, tinst.data(), 4 * tinst.size(), cudaMemcpyHostToDevice,
                            s)) &&
         ok(cudaMemcpyAsync(P->elem_inst, einst.data(), 4 * einst.size(), cudaMemcpyHostToDevice,
                            s)) &&
         ok(cudaMemcpyAsync(P->mat_dev, rows.data(), sizeof(MatRow) * rows.size(),
                            cudaMemcpyHostToDevice, s)) &&
         ok(cudaMemcpyAsync(P->mat_range, ranges.data(), sizeof(int2) * ranges.size(),
                            cudaMemcpyHostToDevice, s)) &&
         ok(cudaStreamSynchronize(s));
  if (!good) return IB_ERR_CUDA;
  const unsigned char* tm = static_cast<const unsigned char*>(b->tmaps);
  b->pc.spread_f = b->calls;
  b->pc.interp_u = b->calls + n;
  b->pc.interp_gf = b->calls + 2 * n;
  b->pc.spread_gu = b->calls + 3 * n;
  b->pc.interp_ug = b->calls + 4 * n;
  b->pc.tmaps_u = tma ? tm : nullptr;
  b->pc.tmaps_gf = tma && b->has_adj ? tm + (size_t)n * kTensorMapBytes : nullptr;
  return IB_OK;
}

}  // namespace

extern "C" {

ib_status ib_batch_create(int32_t n, const ib_instance* inst, int32_t precision, void* stream,
                          ib_batch** out) {
  if (!out) return IB_ERR_INVALID_ARG;
  *out = nullptr;
  if (n <= 0 || !inst || precision != IB_FP32_SPLIT) return IB_ERR_INVALID_ARG;
  bool has_adj = true, any_gG = false;
  for (int i = 0; i < n; ++i) {
    const ib_status st = check_instance(inst[i]);
    if (st != IB_OK) return st;
    if (inst[i].x.grad_unit != inst[0].x.grad_unit) return IB_ERR_INVALID_ARG;
    const ib_instance& in = inst[i];
    if (!(in.gU && in.gf && in.gu && in.gx)) has_adj = false;
    if (in.gf && (reinterpret_cast<uintptr_t>(in.gf) & 15)) return IB_ERR_INVALID_ARG;
    if (in.gu && (reinterpret_cast<uintptr_t>(in.gu) & 15)) return IB_ERR_INVALID_ARG;
    any_gG = any_gG || in.gG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  ib_batch* b = new ib_batch();
  b->n = n;
  b->inst.assign(inst, inst + n);
  b->has_adj = has_adj;
  b->any_gG = any_gG;
  b->gunit = inst[0].x.grad_unit > 0.0 ? inst[0].x.grad_unit : 1.0;
  ib_status st = build(b, s);
  // one tuning for the packed plan, timed on the batch's own forward (timing
  // the backward separately chose other caps for it, at the same speed)
  if (st == IB_OK) st = autotune_with(b->P, [b](cudaStream_t t) { return run_forward(b, t); }, s);
  if (st == IB_OK && !ok(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)))
    st = IB_ERR_CUDA;
  if (st == IB_OK) st = capture(b, run_forward, &b->fwd);
  if (st == IB_OK && has_adj) st = capture(b, run_adjoint, &b->adj);
  if (st == IB_OK && !ok(cudaStreamSynchronize(s))) st = IB_ERR_CUDA;
  if (st != IB_OK) {
    destroy(b);
    return st;
  }
  *out = b;
  return IB_OK;
}

ib_status ib_batch_forward(ib_batch* b, void* stream) {
  if (!b || !b->fwd) return IB_ERR_INVALID_ARG;
  return ok(cudaGraphLaunch(b->fwd, reinterpret_cast<cudaStream_t>(stream))) ? IB_OK
                                                                             : IB_ERR_CUDA;
}

ib_status ib_batch_adjoint(ib_batch* b, void* stream) {
  if (!b || !b->adj) return IB_ERR_INVALID_ARG;
  return ok(cudaGraphLaunch(b->adj, reinterpret_cast<cudaStream_t>(stream))) ? IB_OK
                                                                             : IB_ERR_CUDA;
}

ib_status ib_batch_gparams(ib_batch* b, double* gparams, void* stream) {
  if (!b || !gparams) return IB_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!ok(cudaMemcpyAsync(gparams, b->gparams,
                          sizeof(double) * kParamRow * IB_MAX_MATERIALS * (size_t)b->n,
                          cudaMemcpyDeviceToHost, s)))
    return IB_ERR_CUDA;
  return ok(cudaStreamSynchronize(s)) ? IB_OK : IB_ERR_CUDA;
}

ib_status ib_batch_get_tuning(const ib_batch* b, int32_t tuning[4]) {
  if (!b || !b->P) return IB_ERR_INVALID_ARG;
  return ib_plan_get_tuning(b->P, tuning);
}

ib_status ib_batch_destroy(ib_batch* b) {
  if (!b) return IB_ERR_INVALID_ARG;
  destroy(b);
  return IB_OK;
}

}  // extern "C"
