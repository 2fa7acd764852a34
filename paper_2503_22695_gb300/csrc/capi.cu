// C ABI of libibfe: plan lifecycle, argument validation and the operator
// entry points declared in include/ibfe.h.  Every operator is a short,
// stream-ordered sequence of the kernels in this directory; nothing here
// allocates after ib_plan_create.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <vector>

#include "ib_internal.cuh"

namespace ibfe {
int sort_hist_blocks(int64_t Q);
}

using namespace ibfe;

namespace {

constexpr int kIncShift = 28;

bool ok(cudaError_t e) { return e == cudaSuccess; }

template <typename T>
bool dalloc(T** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  return ok(cudaMalloc((void**)p, bytes));
}

void free_plan(ib_plan* p) {
  if (!p) return;
  void* ptrs[] = {p->inc_off, p->inc_idx, p->mass, p->inv_mass, p->wj0, p->elem_scratch,
                  p->elem_scratch2, p->keys[0], p->keys[1], p->vals[0], p->vals[1], p->hist,
                  p->tile_start, p->tile_end, p->tile_slot, p->tile_nonempty, p->tile_near,
                  p->tile_list, p->tile_list_near, p->tile_vmax, p->tile_done, p->tile_sk, p->tile_bcount, p->tile_counters,
                  p->digit_tot, p->rpart, p->spread_scratch, p->q_cell, p->q_off, p->q_val, p->p_cell,
                  p->p_off, p->p_val, p->p_idx, p->vol_jm1, p->gq_a, p->gq_b, p->epart, p->ered,
                  p->dstatus, p->node_tmp, p->pen_part, p->mat_range, p->inst, p->tile_inst,
                  p->elem_inst, p->mat_dev};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->own_side_bufs)
    for (void* q : {p->q_val_b, p->p_val_b, p->gq_c, p->elem_scratch3})
      if (q) cudaFree(q);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->hi) cudaStreamDestroy(p->hi);
  if (p->zside) cudaStreamDestroy(p->zside);
  for (cudaEvent_t ev : {p->ev_fork, p->ev_join, p->ev_ffork, p->ev_fsorted, p->ev_fjoin,
                         p->ev_hjoin})
    if (ev) cudaEventDestroy(ev);
  if (p->ev) {
    for (int i = 0; i < p->ev_cap; ++i) cudaEventDestroy(p->ev[i]);
    delete[] p->ev;
    delete[] p->ev_stage;
  }
  delete p;
}

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Host-side fault injection for error-path tests: IBFE_FAULT="entry[:code]"
// makes that C entry point return `code` (default IB_ERR_CUDA) before doing
// anything.  Read on every call; no device is touched.
ib_status injected(const char* entry) {
  const char* spec = std::getenv("IBFE_FAULT");
  if (!spec) return IB_OK;
  const char* colon = std::strchr(spec, ':');
  const size_t n = colon ? (size_t)(colon - spec) : std::strlen(spec);
  if (n != std::strlen(entry) || std::strncmp(spec, entry, n) != 0) return IB_OK;
  const int code = colon ? std::atoi(colon + 1) : (int)IB_ERR_CUDA;
  return code > 0 ? (ib_status)code : IB_ERR_CUDA;
}

bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; }

ib_status check_launch(ib_status st) {
  if (st != IB_OK) return st;
  return ok(cudaGetLastError()) ? IB_OK : IB_ERR_CUDA;
}

ib_status check_pos(const ib_plan* p, const ib_pos* x) {
  if (!x || !std::isfinite(x->grad_unit) || x->grad_unit < 0.0) return IB_ERR_INVALID_ARG;
  if (p->precision == IB_FP64) return x->x64 ? IB_OK : IB_ERR_INVALID_ARG;
  return (x->cell && x->off) ? IB_OK : IB_ERR_INVALID_ARG;
}

// The length per which position derivatives are returned (ib_pos.grad_unit).
double gunit(const ib_pos* x) { return x->grad_unit > 0.0 ? x->grad_unit : 1.0; }

const void* pos_a(const ib_plan* p, const ib_pos* x) {
  return p->precision == IB_FP64 ? (const void*)x->x64 : (const void*)x->cell;
}

ib_status make_table(const ib_plan* p, const ib_material* mats, int32_t n_mats, MatTable& mt) {
  if (!mats || n_mats <= 0 || n_mats > IB_MAX_MATERIALS || n_mats <= p->max_mat_id)
    return IB_ERR_INVALID_ARG;
  std::memset(&mt, 0, sizeof(mt));
  mt.n = n_mats;
  for (int m = 0; m < n_mats; ++m) {
    // exponential laws divide by their rate constants in the energy
    if (!material_valid(mats[m])) return IB_ERR_INVALID_ARG;
    mt.model[m] = mats[m].model;
    for (int k = 0; k < mats[m].n_params; ++k) mt.p[m][k] = mats[m].params[k];
    mt.p[m][kTa] = mats[m].Ta;
    mat_entry_finish(mt.p[m], mt.pf[m], mt.act[m]);
  }
  return IB_OK;
}

// Fold recorded event pairs into the per-stage sums (waits for them).
void prof_flush(ib_plan* p) {
  if (!p->ev_used) return;
  cudaEventSynchronize(p->ev[p->ev_used - 1]);
  for (int i = 0; i + 1 < p->ev_used; i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->ev[i], p->ev[i + 1]) == cudaSuccess)
      p->prof_ms[p->ev_stage[i / 2]] += ms;
  }
  p->ev_used = 0;
}

}  // namespace

// Profiler intervals: a begin reserves an event pair and records its first
// event; the end records the second.  Intervals may nest (a kernel inside a
// stage); the ring is emptied only when none is open, and an interval that
// finds it full while another is open is not timed.
int ibfe::prof_begin(ib_plan* p, int stage, cudaStream_t s) {
  int idx = -1;
  if (p->prof_on && p->ev) {
    if (p->ev_used + 2 > p->ev_cap && p->prof_depth == 0) prof_flush(p);
    if (p->ev_used + 2 <= p->ev_cap) {
      idx = p->ev_used;
      p->ev_used += 2;
      p->ev_stage[idx / 2] = stage;
      cudaEventRecord(p->ev[idx], s);
    }
  }
  p->prof_depth++;
  return idx;
}

void ibfe::prof_end(ib_plan* p, int idx, cudaStream_t s) {
  p->prof_depth--;
  if (idx >= 0) cudaEventRecord(p->ev[idx + 1], s);
}

namespace {

// One stage of an operator: counts its kernel launches and, while profiling
// is enabled, brackets it with CUDA events on the operator's stream.
struct Stage {
  ib_plan* p;
  cudaStream_t s;
  int idx;
  Stage(ib_plan* p_, int stage, cudaStream_t s_, int launches) : p(p_), s(s_) {
    p->prof_launches[stage] += launches;
    p->prof_calls[stage] += 1;
    idx = prof_begin(p, stage, s);
  }
  ~Stage() { prof_end(p, idx, s); }
};

int sort_launches(const ib_plan* p) {
  // FP32 binning: classify, compact (ranges), scatter.  FP64: radix passes
  // (hist, digit scan, scatter), bounds, classify, compact, reorder
  if (p->precision != IB_FP64) return 3;
  return 3 * ((sort_key_bits(p->ntiles) + 7) / 8) + 4;
}

// forward pieces shared by the entry points
ib_status do_points_sorted(ib_plan* p, const ib_pos* x, const void* nodal, cudaStream_t s) {
  ib_status st;
  {
    Stage sc(p, IB_STAGE_POINTS, s, 1);
    st = launch_points(p, pos_a(p, x), x->off, nodal, nodal ? 1 : 0, s);
  }
  if (st != IB_OK) return st;
  Stage sc(p, IB_STAGE_SORT, s, sort_launches(p));
  return launch_sort_points(p, nodal != nullptr, s);
}

ib_status do_interp(ib_plan* p, const void* u, int mode, double vs, double gs, cudaStream_t s,
                    const GridCall* calls = nullptr, const void* tmaps = nullptr,
                    const InterpIO* io = nullptr) {
  Stage sc(p, IB_STAGE_INTERP, s, 1);
  return launch_interp_points(p, u, mode, vs, gs, s, calls, tmaps, io);
}

ib_status do_project(ib_plan* p, const void* vals, void* elem, cudaStream_t s) {
  Stage sc(p, IB_STAGE_PROJECT, s, 1);
  // the interpolated values (gq_a) carry no w_q j0 yet; the position
  // gradients (gq_b) already have it through the carried values
  return launch_elem_project(p, vals, vals == p->gq_a, elem, s);
}

ib_status do_gather(ib_plan* p, const void* elem, const void* scale, void* out, cudaStream_t s,
                    const void* add = nullptr, double mul = 1.0) {
  Stage sc(p, IB_STAGE_GATHER, s, 1);
  return launch_node_gather(p, elem, scale, out, s, add, mul);
}

// Coupling-point values gq [3][Q] to nodal values: Gauss rule, the lumped
// projection out = add + scale * gather(project(gq)) (scale: the inverse mass
// or none); nodal rule, the points are the nodes: out = add + gq.
ib_status to_nodes(ib_plan* p, const void* gq, void* elem, const void* scale, void* out,
                   cudaStream_t s, const void* add = nullptr) {
  if (p->quad == IB_QUAD_NODAL) {
    Stage sc(p, IB_STAGE_GATHER, s, 1);
    return launch_node_copy(p, gq, out, add, s);
  }
  ib_status st = do_project(p, gq, elem, s);
  if (st == IB_OK) st = do_gather(p, elem, scale, out, s, add);
  return st;
}

ib_status do_spread(ib_plan* p, double scale, void* f, cudaStream_t s, bool zero_fill = true,
                    const GridCall* calls = nullptr, const void* vals = nullptr) {
  Stage sc(p, IB_STAGE_SPREAD, s, spread_launches(p->precision) - (zero_fill ? 0 : 1));
  return launch_spread(p, scale, f, s, zero_fill, calls, vals);
}

ib_status do_reduce(ib_plan* p, int nvals, int n_mats, cudaStream_t s, bool real_parts) {
  Stage sc(p, IB_STAGE_REDUCE, s, 2);
  return launch_reduce_parts(p, nvals, n_mats, s, real_parts);
}

ib_status do_interp_tail(ib_plan* p, const void* u, void* U, cudaStream_t s,
                         void* elem = nullptr, const PackedCalls* pc = nullptr) {
  if (!elem) elem = p->elem_scratch;
  ib_status st = pc ? do_interp(p, u, 0, 1.0, 0.0, s, pc->interp_u, pc->tmaps_u)
                    : do_interp(p, u, 0, 1.0, 0.0, s);
  if (st == IB_OK) st = to_nodes(p, p->gq_a, elem, p->inv_mass, U, s);
  return st;
}

}  // namespace

extern "C" {

int32_t ib_version(void) { return 100; }

double ib_active_tension(double t) {
  const double period = 0.8, peak = 84260.0, width = 0.005;
  double tc = std::fmod(t, period);
  if (tc < 0.0) tc += period;
  if (tc < 0.5) return 0.0;
  const double r = tc < 0.65 ? tc - 0.5 : period - tc;  // rise, then mirrored fall
  return peak * (1.0 - std::exp(-r * r / width));
}

const char* ib_status_str(ib_status s) {
  switch (s) {
    case IB_OK: return "ok";
    case IB_ERR_INVALID_ARG: return "invalid argument";
    case IB_ERR_CUDA: return "CUDA error";
    case IB_ERR_NONFINITE: return "position offset outside [0,1) or not finite";
    case IB_ERR_CAPACITY: return "size exceeds a documented limit";
    case IB_ERR_TIMEOUT: return "bounded device wait gave up";
    case IB_ERR_UNSUPPORTED: return "unsupported configuration";
    case IB_ERR_INVERTED: return "element with non-positive reference Jacobian";
  }
  return "unknown status";
}

ib_status ib_plan_create(const ib_mesh* mesh, const ib_grid* grid, int32_t quad,
                         int32_t precision, void* stream, ib_plan** out) {
  if (const ib_status f = injected("ib_plan_create")) return f;
  if (!out) return IB_ERR_INVALID_ARG;
  *out = nullptr;
  if (!mesh || !grid) return IB_ERR_INVALID_ARG;
  if (precision != IB_FP32_SPLIT && precision != IB_FP64 && precision != IB_FP32_SPLIT_F32STAB &&
      precision != IB_FP32_SPLIT_DFVOL)
    return IB_ERR_INVALID_ARG;
  if (quad != IB_QUAD_GAUSS2 && quad != IB_QUAD_NODAL) return IB_ERR_INVALID_ARG;
  if (mesh->n_nodes <= 0 || mesh->n_elems < 0 || (mesh->n_elems > 0 && !mesh->conn) || !mesh->X)
    return IB_ERR_INVALID_ARG;
  if (mesh->elem_type != IB_ELEM_HEX8 && mesh->elem_type != IB_ELEM_TET4 &&
      mesh->elem_type != IB_ELEM_TET10)
    return IB_ERR_INVALID_ARG;
  const ib_status gs = check_grid(grid);
  if (gs != IB_OK) return gs;
  GridDev g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = grid->n[d];
    g.nt[d] = grid->n[d] / kTile;
    g.origin[d] = grid->origin[d];
  }
  g.h = grid->h;
  return plan_build(mesh, g, g.nt[0] * g.nt[1] * g.nt[2], quad, precision, IB_MAX_MATERIALS,
                    S(stream), out);
}

}  // extern "C"

namespace ibfe {

ib_status check_grid(const ib_grid* grid) {
  if (!(grid->h > 0.0) || !std::isfinite(grid->h)) return IB_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d) {
    if (!std::isfinite(grid->origin[d])) return IB_ERR_INVALID_ARG;
    if (grid->n[d] < kTile || grid->n[d] > (1 << kPackBits)) return IB_ERR_UNSUPPORTED;
    if (grid->n[d] % kTile) return IB_ERR_UNSUPPORTED;
  }
  return IB_OK;
}

ib_status plan_build(const ib_mesh* mesh, const GridDev& grid, int ntiles, int32_t quad,
                     int32_t precision, int mat_cap, cudaStream_t s, ib_plan** out,
                     bool packed) {
  // nodes and coupling points per element
  const int nc = mesh->elem_type == IB_ELEM_TET10 ? 10 : (mesh->elem_type == IB_ELEM_TET4 ? 4 : 8);
  const int nq = mesh->elem_type == IB_ELEM_HEX8 ? 8 : 4;
  if ((int64_t)mesh->n_elems >= (1LL << kIncShift) / 8) return IB_ERR_CAPACITY;
  // Q coupling points: the element rule's points (8 per hexahedron, 4 per
  // tetrahedron) or the nodes
  const int64_t E = mesh->n_elems, N = mesh->n_nodes;
  const int64_t Q = quad == IB_QUAD_NODAL ? N : nq * E;

  // connectivity and materials to the host for validation and incidence lists
  std::vector<int32_t> conn(nc * E), mid;
  if (E > 0 && !ok(cudaMemcpyAsync(conn.data(), mesh->conn, sizeof(int32_t) * nc * E,
                                   cudaMemcpyDeviceToHost, s)))
    return IB_ERR_CUDA;
  if (mesh->mat_id) {
    mid.resize(E);
    if (E > 0 && !ok(cudaMemcpyAsync(mid.data(), mesh->mat_id, sizeof(int32_t) * E,
                                     cudaMemcpyDeviceToHost, s)))
      return IB_ERR_CUDA;
  }
  if (!ok(cudaStreamSynchronize(s))) return IB_ERR_CUDA;
  for (int64_t k = 0; k < nc * E; ++k)
    if (conn[k] < 0 || conn[k] >= N) return IB_ERR_INVALID_ARG;
  int max_mid = 0;
  for (int32_t m : mid) {
    if (m < 0 || m >= mat_cap) return IB_ERR_INVALID_ARG;
    max_mid = m > max_mid ? m : max_mid;
  }

  // node -> (corner, element) incidence, ascending element then corner
  std::vector<int32_t> inc_off(N + 1, 0), inc_idx(nc * E);
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < nc; ++a) inc_off[conn[a * E + e] + 1]++;
  for (int64_t n = 0; n < N; ++n) inc_off[n + 1] += inc_off[n];
  {
    std::vector<int32_t> fill(inc_off.begin(), inc_off.end() - 1);
    for (int64_t e = 0; e < E; ++e)
      for (int a = 0; a < nc; ++a)
        inc_idx[fill[conn[a * E + e]]++] =
            static_cast<int32_t>((static_cast<uint32_t>(a) << kIncShift) | static_cast<uint32_t>(e));
  }

  ib_plan* p = new ib_plan;
  std::memset(p, 0, sizeof(ib_plan));
  p->precision = precision;
  p->quad = quad;
  p->elem = mesh->elem_type;
  p->nc = nc;
  p->nq = nq;
  p->chunk = kChunk;
  // the fastest tuning of the 256^3 shell forward in A/B runs
  p->fe_ctas = 4;
  p->push_per_sm = 8;
  p->interp_per_sm = 3;
  p->N = (int)N;
  p->E = (int)E;
  p->Q = Q;
  p->rsize = precision == IB_FP64 ? sizeof(double) : sizeof(float);
  p->grid = grid;
  p->ntiles = ntiles;
  p->n_inst = 1;
  p->mat_cap = mat_cap;
  p->conn = mesh->conn;
  p->X = mesh->X;
  p->fibres = mesh->fibres;
  p->mat_id = mesh->mat_id;
  p->max_mat_id = max_mid;
  p->hist_blocks = sort_hist_blocks(Q);
  const size_t rs = p->rsize;
  bool good = dalloc(&p->inc_off, 4 * (N + 1)) && dalloc(&p->inc_idx, 4 * nc * E) &&
              dalloc(&p->mass, rs * N) && dalloc(&p->inv_mass, rs * N) &&
              dalloc(&p->wj0, rs * nc * E) && dalloc(&p->elem_scratch, rs * 3 * nc * E) &&
              dalloc(&p->elem_scratch2, rs * 3 * nc * E) && dalloc(&p->keys[0], 4 * Q) &&
              dalloc(&p->keys[1], 4 * Q) && dalloc(&p->vals[0], 4 * Q) &&
              dalloc(&p->vals[1], 4 * Q) && dalloc(&p->hist, 4 * 256 * (size_t)p->hist_blocks) &&
              dalloc(&p->tile_start, 4 * (size_t)p->ntiles) &&
              dalloc(&p->tile_end, 4 * (size_t)p->ntiles) &&
              dalloc(&p->tile_slot, 4 * (size_t)p->ntiles) &&
              dalloc(&p->tile_nonempty, 4 * (size_t)p->ntiles) &&
              dalloc(&p->tile_near, 4 * (size_t)p->ntiles) &&
              dalloc(&p->tile_list, 4 * (size_t)max_work_items(p->ntiles, Q)) &&
              dalloc(&p->tile_list_near, 4 * (size_t)p->ntiles) &&
              dalloc(&p->tile_vmax, 4 * (size_t)p->ntiles) &&
              dalloc(&p->tile_done, 4 * (size_t)p->ntiles) &&
              dalloc(&p->tile_sk, 16 * (size_t)p->ntiles) &&
              dalloc(&p->tile_bcount, 12 * (size_t)classify_blocks(p->ntiles)) &&
              dalloc(&p->tile_counters, 32) && dalloc(&p->digit_tot, 4 * 256) &&
              dalloc(&p->rpart, 8 * kParamRow * (size_t)mat_cap * kReduceCTAs) &&
              dalloc(&p->mat_range, sizeof(int2) * (size_t)mat_cap) &&
              dalloc(&p->spread_scratch,
                     spread_scratch_bytes(precision, Q < p->ntiles ? (Q > 0 ? Q : 1)
                                                                   : max_work_items(p->ntiles, Q))) &&
              dalloc(&p->q_cell, 4 * Q) &&
              dalloc(&p->q_off, rs * 3 * Q) && dalloc(&p->q_val, rs * 3 * Q) &&
              dalloc(&p->p_cell, 4 * Q) && dalloc(&p->p_off, rs * 3 * Q) &&
              dalloc(&p->p_val, rs * 3 * Q) && dalloc(&p->p_idx, 4 * Q) &&
              dalloc(&p->node_tmp, rs * 6 * (size_t)N) &&
              dalloc(&p->gq_a, rs * 3 * Q) && dalloc(&p->gq_b, rs * 3 * Q) &&
              dalloc(&p->epart, 8 * kParamRow * (size_t)(E > 0 ? E : 1)) &&
              dalloc(&p->ered, 8 * kParamRow * (size_t)mat_cap) && dalloc(&p->dstatus, 16) &&
              dalloc(&p->pen_part, 8 * penalty_scratch_doubles()) &&
              (packed || ((precision != IB_FP64 || dalloc(&p->q_val_b, rs * 3 * Q)) &&
                          dalloc(&p->p_val_b, rs * 3 * Q) &&
                          dalloc(&p->gq_c, rs * 3 * Q) &&
                          dalloc(&p->elem_scratch3, rs * 3 * nc * E))) &&
              (precision != IB_FP32_SPLIT_DFVOL ||
               dalloc(&p->vol_jm1, sizeof(float) * 2 * (nc == 8 ? 8 : 4) * (size_t)(E > 0 ? E : 1)));
  p->own_side_bufs = !packed;
  if (!good) {
    free_plan(p);
    cudaGetLastError();
    return IB_ERR_CUDA;
  }
  if (packed) {
    // the backward's interpolation-adjoint branch of a packed plan forks
    // after the spreading adjoint is done with these
    p->q_val_b = p->q_val;
    p->p_val_b = p->p_val;
    p->gq_c = p->gq_b;
    p->elem_scratch3 = p->elem_scratch2;
  }
  // every material's elements: the whole mesh (packed plans narrow them)
  const std::vector<int2> ranges(mat_cap, make_int2(0, (int)E));
  good = ok(cudaMemcpyAsync(p->inc_off, inc_off.data(), 4 * (N + 1), cudaMemcpyHostToDevice, s)) &&
         ok(cudaMemcpyAsync(p->mat_range, ranges.data(), sizeof(int2) * mat_cap,
                            cudaMemcpyHostToDevice, s)) &&
         (E == 0 || ok(cudaMemcpyAsync(p->inc_idx, inc_idx.data(), 4 * nc * E,
                                       cudaMemcpyHostToDevice, s))) &&
         ok(cudaMemsetAsync(p->dstatus, 0, 16, s));
  int least = 0, greatest = 0;  // stream priorities (greatest: numerically lowest)
  if (good)
    good = ok(cudaDeviceGetStreamPriorityRange(&least, &greatest)) &&
           ok(cudaStreamCreateWithPriority(&p->hi, cudaStreamNonBlocking, greatest)) &&
           ok(cudaEventCreateWithFlags(&p->ev_hjoin, cudaEventDisableTiming)) &&
           ok(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking)) &&
           ok(cudaStreamCreateWithFlags(&p->zside, cudaStreamNonBlocking)) &&
           ok(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming)) &&
           ok(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming)) &&
           ok(cudaEventCreateWithFlags(&p->ev_ffork, cudaEventDisableTiming)) &&
           ok(cudaEventCreateWithFlags(&p->ev_fsorted, cudaEventDisableTiming)) &&
           ok(cudaEventCreateWithFlags(&p->ev_fjoin, cudaEventDisableTiming));
  if (good) good = spread_prepare(p) == IB_OK && interp_prepare(p) == IB_OK;
  if (!good || launch_plan_static(p, s) != IB_OK || !ok(cudaStreamSynchronize(s))) {
    free_plan(p);
    return IB_ERR_CUDA;
  }
  int st = 0;
  if (!ok(cudaMemcpy(&st, p->dstatus, sizeof(int), cudaMemcpyDeviceToHost))) {
    free_plan(p);
    return IB_ERR_CUDA;
  }
  if (st & kStatInverted) {
    free_plan(p);
    return IB_ERR_INVERTED;
  }
  *out = p;
  return IB_OK;
}

void plan_free(ib_plan* p) { free_plan(p); }

}  // namespace ibfe

extern "C" {

ib_status ib_plan_destroy(ib_plan* plan) {
  if (!plan) return IB_ERR_INVALID_ARG;
  free_plan(plan);
  return IB_OK;
}

ib_status ib_lumped_mass(ib_plan* p, void* mass, void* stream) {
  if (!p || !mass) return IB_ERR_INVALID_ARG;
  return ok(cudaMemcpyAsync(mass, p->mass, p->rsize * p->N, cudaMemcpyDeviceToDevice, S(stream)))
             ? IB_OK
             : IB_ERR_CUDA;
}

ib_status ib_fe_force(ib_plan* p, const ib_material* mats, int32_t n_mats, const ib_pos* x,
                      void* G, double* energy, void* stream) {
  if (const ib_status f = injected("ib_fe_force")) return f;
  if (!p || !G) return IB_ERR_INVALID_ARG;
  ib_status st = check_pos(p, x);
  if (st != IB_OK) return st;
  MatTable mt;
  if ((st = make_table(p, mats, n_mats, mt)) != IB_OK) return st;
  cudaStream_t s = S(stream);
  {
    Stage sc(p, IB_STAGE_FORCE, s, 1);
    st = launch_fe_force(p, mt, pos_a(p, x), x->off, p->elem_scratch, energy != nullptr, s);
  }
  if (st == IB_OK) st = do_gather(p, p->elem_scratch, nullptr, G, s);
  if (st == IB_OK) st = launch_penalty(p, x, G, energy != nullptr, s);
  if (st == IB_OK && energy) {
    st = do_reduce(p, 1, n_mats, s, false);
    double red[kParamRow * IB_MAX_MATERIALS];
    double pen = 0.0;
    if (st == IB_OK &&
        (!ok(cudaMemcpyAsync(red, p->ered, sizeof(red), cudaMemcpyDeviceToHost, s)) ||
         (penalty_on(p) && !ok(cudaMemcpyAsync(&pen, penalty_energy_dev(p), sizeof(double),
                                               cudaMemcpyDeviceToHost, s))) ||
         !ok(cudaStreamSynchronize(s))))
      st = IB_ERR_CUDA;
    if (st == IB_OK) {
      double en = pen;
      for (int m = 0; m < n_mats; ++m) en += red[m * kParamRow];
      *energy = en;
    }
  }
  return check_launch(st);
}

ib_status ib_spread(ib_plan* p, const ib_pos* x, const void* G, void* f, void* stream) {
  if (const ib_status f = injected("ib_spread")) return f;
  if (!p || !G || !f || !aligned16(f)) return IB_ERR_INVALID_ARG;
  ib_status st = check_pos(p, x);
  if (st != IB_OK) return st;
  cudaStream_t s = S(stream);
  st = do_points_sorted(p, x, G, s);
  if (st == IB_OK) st = do_spread(p, 1.0 / (p->grid.h * p->grid.h * p->grid.h), f, s);
  return check_launch(st);
}

ib_status ib_interp(ib_plan* p, const ib_pos* x, const void* u, void* U, void* stream) {
  if (const ib_status f = injected("ib_interp")) return f;
  if (!p || !u || !U) return IB_ERR_INVALID_ARG;
  ib_status st = check_pos(p, x);
  if (st != IB_OK) return st;
  cudaStream_t s = S(stream);
  st = do_points_sorted(p, x, nullptr, s);
  if (st == IB_OK) st = do_interp_tail(p, u, U, s);
  return check_launch(st);
}

}  // extern "C"

namespace ibfe {

ib_status forward_body(ib_plan* p, const MatTable& mt, const ib_pos* x, const void* u, void* G,
                       void* f, void* U, cudaStream_t s, const PackedCalls* pc) {
  // Two branches forked from the caller's stream s.  The critical one -- the
  // FE force, the nodal gather, the carried values and the spreading -- runs
  // on stream m; the Gauss-point binning, the far-tile zeros and the
  // interpolation depend only on x and u and run on the side stream b beside
  // it.  The spreading waits for the binning; s waits for both branches.  For
  // a plan of one structure m is the plan's high-priority stream, so that the
  // CTA scheduler prefers the critical kernels (0.417 -> 0.405 ms at 256^3);
  // a packed batch, whose merge and interpolation balance differently, was
  // slower that way (1.17 -> 1.28 ms) and keeps m = s.
  cudaStream_t b = p->side, m = p->n_inst > 1 ? s : p->hi;
  if (!ok(cudaEventRecord(p->ev_ffork, s)) || !ok(cudaStreamWaitEvent(b, p->ev_ffork, 0)) ||
      (m != s && !ok(cudaStreamWaitEvent(m, p->ev_ffork, 0))))
    return IB_ERR_CUDA;
  ib_status st = do_points_sorted(p, x, nullptr, b);
  // the spreading's per-tile maxima zeroed here, off the critical stream,
  // which takes them after waiting for the binning
  if (st == IB_OK && p->precision != IB_FP64 &&
      !ok(cudaMemsetAsync(p->tile_vmax, 0, sizeof(uint32_t) * p->ntiles, b)))
    st = IB_ERR_CUDA;
  if (st == IB_OK && !ok(cudaEventRecord(p->ev_fsorted, b))) st = IB_ERR_CUDA;
  // the far-tile zeros of f (HBM writes) on the side branch, beside the
  // force kernel and ahead of the interpolation
  if (st == IB_OK) {
    p->prof_launches[IB_STAGE_SPREAD] += 1;  // overlapped: not in the spread stage's time
    st = launch_spread_zero(p, f, b, pc ? pc->spread_f : nullptr);
  }
  if (st == IB_OK) st = do_interp_tail(p, u, U, b, p->elem_scratch2, pc);
  if (st == IB_OK && !ok(cudaEventRecord(p->ev_fjoin, b))) st = IB_ERR_CUDA;
  if (st == IB_OK) {
    Stage sc(p, IB_STAGE_FORCE, m, 1);
    st = launch_fe_force(p, mt, pos_a(p, x), x->off, p->elem_scratch, false, m);
  }
  if (st == IB_OK) st = do_gather(p, p->elem_scratch, nullptr, G, m);
  if (st == IB_OK) st = launch_penalty(p, x, G, false, m);
  if (st == IB_OK) {
    // the carried values before the binning is waited for, then their binned
    // copy: the values overlap the binning's end (computing them at the binned
    // positions in one pass after the wait, as the backward does, measured
    // 0.404 -> 0.418 ms here)
    Stage sc(p, IB_STAGE_POINTS, m, 2);
    st = launch_point_values(p, G, m);
    if (st == IB_OK && !ok(cudaStreamWaitEvent(m, p->ev_fsorted, 0))) st = IB_ERR_CUDA;
    if (st == IB_OK) st = launch_permute_values(p, m, true, nullptr, nullptr, false);
  }
  if (st == IB_OK)
    st = do_spread(p, 1.0 / (p->grid.h * p->grid.h * p->grid.h), f, m, /*zero_fill=*/false,
                   pc ? pc->spread_f : nullptr);
  if (st == IB_OK && m != s &&
      (!ok(cudaEventRecord(p->ev_hjoin, m)) || !ok(cudaStreamWaitEvent(s, p->ev_hjoin, 0))))
    st = IB_ERR_CUDA;
  if (st == IB_OK && !ok(cudaStreamWaitEvent(s, p->ev_fjoin, 0))) st = IB_ERR_CUDA;
  return check_launch(st);
}

}  // namespace ibfe

extern "C" {

ib_status ib_forward(ib_plan* p, const ib_material* mats, int32_t n_mats, const ib_pos* x,
                     const void* u, void* G, void* f, void* U, void* stream) {
  if (const ib_status f = injected("ib_forward")) return f;
  if (!p || !u || !G || !f || !U || !aligned16(f) || p->n_inst > 1) return IB_ERR_INVALID_ARG;
  ib_status st = check_pos(p, x);
  if (st != IB_OK) return st;
  MatTable mt;
  if ((st = make_table(p, mats, n_mats, mt)) != IB_OK) return st;
  return forward_body(p, mt, x, u, G, f, U, S(stream), nullptr);
}

ib_status ib_step(ib_plan* p, ib_fluid* fl, const ib_material* mats, int32_t n_mats,
                  const ib_pos* x, void* u, void* G, void* f, void* U, void* pr, void* stream) {
  if (const ib_status f = injected("ib_step")) return f;
  if (!p || !fl || !u || !G || !f || !U || !aligned16(f) || !aligned16(u) ||
      !fluid_matches(fl, p))
    return IB_ERR_INVALID_ARG;
  ib_status st = check_pos(p, x);
  if (st != IB_OK) return st;
  MatTable mt;
  if ((st = make_table(p, mats, n_mats, mt)) != IB_OK) return st;
  cudaStream_t s = S(stream);
  const double h = p->grid.h;
  // nodal force of x^n, spread at x^n
  {
    Stage sc(p, IB_STAGE_FORCE, s, 1);
    st = launch_fe_force(p, mt, pos_a(p, x), x->off, p->elem_scratch, false, s);
  }
  if (st == IB_OK) st = do_gather(p, p->elem_scratch, nullptr, G, s);
  if (st == IB_OK) st = launch_penalty(p, x, G, false, s);
  if (st == IB_OK) st = do_points_sorted(p, x, G, s);
  if (st == IB_OK) st = do_spread(p, 1.0 / (h * h * h), f, s);
  // u^n -> u^{n+1} in place
  if (st == IB_OK) st = fluid_step_async(fl, u, f, u, pr, nullptr, s);
  // U = interpolation of u^{n+1} at the same (binned) points, then x += dt U
  if (st == IB_OK) st = do_interp_tail(p, u, U, s);
  if (st == IB_OK) st = launch_advance_positions(p, x, U, fluid_dt(fl), s);
  return check_launch(st);
}

}  // extern "C"

namespace ibfe {

ib_status backward_body(ib_plan* p, const MatTable& mt, int n_mats, const ib_pos* x,
                        const void* u, const void* G, const void* gG, const void* gf,
                        const void* gU, void* gx, void* gu, bool params, double* gparams,
                        cudaStream_t s, const PackedCalls* pc) {
  cudaStream_t b = p->side;
  const double h = p->grid.h, ih3 = 1.0 / (h * h * h);
  const size_t nbytes = p->rsize * 3 * (size_t)p->N;
  void* gGt = p->node_tmp;  // the force cotangent gG + (df/dG)^T gf
  // the interpolation adjoint's position term, added into gx after the join
  void* gxi = static_cast<char*>(p->node_tmp) + nbytes;
  const bool force = gG || gf;
  const double gxu = gunit(x);
  // Gauss points built and binned once for both transfer adjoints
  ib_status st = do_points_sorted(p, x, nullptr, s);
  // The interpolation adjoint (a spreading of gU and the position term of
  // the interpolation of u) runs on the side stream with its own carried
  // values, gradient output, projection scratch, nodal result and work
  // counter (the per-tile maxima of the carried values are its spreading's),
  // beside the spreading adjoint (an interpolation of gf: values and position
  // weights) and the force adjoint on the caller's stream.  For a plan of one
  // structure it forks right after the binning (0.75 -> 0.67 ms at 256^3); a
  // packed batch, whose persistent transfer kernels each fill the GPU, forks
  // it after the spreading adjoint, beside the force adjoint alone (forking
  // at the binning took 2.3 -> 3.3 ms for the 48-instance sweep).
  const InterpIO io_u = {p->p_val_b, nullptr, p->gq_c, 4};
  auto side = [&]() {
    if (!gU) return;
    if (st == IB_OK && (!ok(cudaEventRecord(p->ev_ffork, s)) ||
                        !ok(cudaStreamWaitEvent(b, p->ev_ffork, 0))))
      st = IB_ERR_CUDA;
    if (st == IB_OK) {
      Stage sc(p, IB_STAGE_POINTS, b, binned_values_launches(p));
      st = launch_binned_values(p, gU, b, true, p->q_val_b, p->p_val_b);
    }
    if (st == IB_OK) st = do_spread(p, 1.0, gu, b, true, pc ? pc->spread_gu : nullptr, p->p_val_b);
    if (st == IB_OK)
      st = pc ? do_interp(p, nullptr, 2, 0.0, 0.0, b, pc->interp_ug, pc->tmaps_u, &io_u)
              : do_interp(p, u, 2, 0.0, gxu / h, b, nullptr, nullptr, &io_u);
    if (st == IB_OK) st = to_nodes(p, p->gq_c, p->elem_scratch3, nullptr, gxi, b);
    if (st == IB_OK && !ok(cudaEventRecord(p->ev_fjoin, b))) st = IB_ERR_CUDA;
  };
  if (!pc) side();
  if (st == IB_OK && gf) {
    Stage sc(p, IB_STAGE_POINTS, s, binned_values_launches(p));
    st = launch_binned_values(p, G, s, false);
  }
  if (st == IB_OK && gf)
    st = pc ? do_interp(p, nullptr, 1, 0.0, 0.0, s, pc->interp_gf, pc->tmaps_gf)
            : do_interp(p, gf, 1, ih3, ih3 / h * gxu, s);
  if (st == IB_OK && gf) st = to_nodes(p, p->gq_a, p->elem_scratch, p->inv_mass, gGt, s, gG);
  // the spreading adjoint's position term: a packed plan's side branch reuses
  // gq_b and elem_scratch2, so it is projected before that branch forks;
  // otherwise after the force adjoint, which needs only gGt (0.646 -> 0.626
  // ms at 256^3)
  if (pc && st == IB_OK && gf) st = to_nodes(p, p->gq_b, p->elem_scratch2, nullptr, gx, s);
  if (st == IB_OK && !gf) {
    if (!ok(cudaMemsetAsync(gx, 0, nbytes, s)) ||
        !ok(gG ? cudaMemcpyAsync(gGt, gG, nbytes, cudaMemcpyDeviceToDevice, s)
               : cudaMemsetAsync(gGt, 0, nbytes, s)))
      st = IB_ERR_CUDA;
  }
  if (pc) side();
  if (st == IB_OK && force) {
    Stage sc(p, IB_STAGE_FORCE, s, 1);
    st = launch_fe_force_adj(p, mt, pos_a(p, x), x->off, gGt, p->elem_scratch, params, s);
  }
  if (st == IB_OK && force && params) st = do_reduce(p, kParamRow, n_mats, s, true);
  if (!pc && st == IB_OK && gf) st = to_nodes(p, p->gq_b, p->elem_scratch2, nullptr, gx, s);
  // join: gx = (spreading adjoint's term + interpolation adjoint's term) +
  // the force adjoint's gather, in that order
  if (st == IB_OK && gU && !ok(cudaStreamWaitEvent(s, p->ev_fjoin, 0))) st = IB_ERR_CUDA;
  if (st == IB_OK && gU) {
    Stage sc(p, IB_STAGE_GATHER, s, 1);
    st = launch_node_copy(p, gxi, gx, gx, s);
  }
  if (st == IB_OK && force) st = do_gather(p, p->elem_scratch, nullptr, gx, s, gx, gxu);
  if (st == IB_OK && force) st = launch_penalty_adj(p, gGt, gx, s, gxu);
  if (st == IB_OK && params) {
    const size_t pb = sizeof(double) * kParamRow * (size_t)n_mats;
    if (!force && !ok(cudaMemsetAsync(p->ered, 0, pb, s))) st = IB_ERR_CUDA;
    if (st == IB_OK && gparams &&
        !ok(cudaMemcpyAsync(gparams, p->ered, pb, cudaMemcpyDeviceToDevice, s)))
      st = IB_ERR_CUDA;
  }
  return check_launch(st);
}

}  // namespace ibfe

extern "C" {

ib_status ib_backward(ib_plan* p, const ib_material* mats, int32_t n_mats, const ib_pos* x,
                      const void* u, const void* G, const void* gG, const void* gf,
                      const void* gU, void* gx, void* gu, double* gparams, void* stream) {
  if (const ib_status f = injected("ib_backward")) return f;
  if (!p || !gx || (gf && !G) || (gU && (!gu || !u)) || (gu && !aligned16(gu)) || p->n_inst > 1)
    return IB_ERR_INVALID_ARG;
  ib_status st = check_pos(p, x);
  if (st != IB_OK) return st;
  MatTable mt;
  if ((st = make_table(p, mats, n_mats, mt)) != IB_OK) return st;
  return backward_body(p, mt, n_mats, x, u, G, gG, gf, gU, gx, gu, gparams != nullptr, gparams,
                       S(stream), nullptr);
}

ib_status ib_spread_adj(ib_plan* p, const ib_pos* x, const void* G, const void* gf, void* gG,
                        void* gx, void* stream) {
  if (const ib_status f = injected("ib_spread_adj")) return f;
  if (!p || !G || !gf || !gG) return IB_ERR_INVALID_ARG;
  ib_status st = check_pos(p, x);
  if (st != IB_OK) return st;
  cudaStream_t s = S(stream);
  const double h = p->grid.h, ih3 = 1.0 / (h * h * h);
  st = do_points_sorted(p, x, G, s);
  if (st == IB_OK) st = do_interp(p, gf, gx ? 1 : 0, ih3, ih3 / h * gunit(x), s);
  if (st == IB_OK) st = to_nodes(p, p->gq_a, p->elem_scratch, p->inv_mass, gG, s);
  if (st == IB_OK && gx) st = to_nodes(p, p->gq_b, p->elem_scratch2, nullptr, gx, s);
  return check_launch(st);
}

ib_status ib_interp_adj(ib_plan* p, const ib_pos* x, const void* u, const void* gU, void* gu,
                        void* gx, void* stream) {
  if (const ib_status f = injected("ib_interp_adj")) return f;
  if (!p || !gU || !gu || (gx && !u) || !aligned16(gu)) return IB_ERR_INVALID_ARG;
  ib_status st = check_pos(p, x);
  if (st != IB_OK) return st;
  cudaStream_t s = S(stream);
  st = do_points_sorted(p, x, gU, s);
  if (st == IB_OK) st = do_spread(p, 1.0, gu, s);
  if (st == IB_OK && gx) {
    st = do_interp(p, u, 2, 0.0, gunit(x) / p->grid.h, s);
    if (st == IB_OK) st = to_nodes(p, p->gq_b, p->elem_scratch2, nullptr, gx, s);
  }
  return check_launch(st);
}

}  // extern "C"

namespace ibfe {
// Adjoint of the nodal force without host output: Hv on the device and, if
// `params`, the parameter gradients left in p->ered ([n_mats][kParamRow]).
ib_status fe_force_adj_async(ib_plan* p, const ib_material* mats, int32_t n_mats,
                             const ib_pos* x, const void* v, void* Hv, bool params,
                             cudaStream_t s) {
  if (!p || !v || !Hv) return IB_ERR_INVALID_ARG;
  ib_status st = check_pos(p, x);
  if (st != IB_OK) return st;
  MatTable mt;
  if ((st = make_table(p, mats, n_mats, mt)) != IB_OK) return st;
  {
    Stage sc(p, IB_STAGE_FORCE, s, 1);
    st = launch_fe_force_adj(p, mt, pos_a(p, x), x->off, v, p->elem_scratch, params, s);
  }
  if (st == IB_OK) st = do_gather(p, p->elem_scratch, nullptr, Hv, s, nullptr, gunit(x));
  if (st == IB_OK) st = launch_penalty_adj(p, v, Hv, s, gunit(x));
  if (st == IB_OK && params) st = do_reduce(p, kParamRow, n_mats, s, true);
  return check_launch(st);
}
}  // namespace ibfe

extern "C" {

ib_status ib_fe_force_adj(ib_plan* p, const ib_material* mats, int32_t n_mats, const ib_pos* x,
                          const void* v, void* Hv, double* gparams, void* stream) {
  if (const ib_status f = injected("ib_fe_force_adj")) return f;
  cudaStream_t s = S(stream);
  ib_status st = fe_force_adj_async(p, mats, n_mats, x, v, Hv, gparams != nullptr, s);
  if (st == IB_OK && gparams) {
    double red[kParamRow * IB_MAX_MATERIALS];
    if (!ok(cudaMemcpyAsync(red, p->ered, sizeof(red), cudaMemcpyDeviceToHost, s)) ||
        !ok(cudaStreamSynchronize(s)))
      return IB_ERR_CUDA;
    for (int m = 0; m < n_mats; ++m)
      for (int k = 0; k < kParamRow; ++k) gparams[m * kParamRow + k] = red[m * kParamRow + k];
  }
  return st;
}

ib_status ib_plan_get_tuning(const ib_plan* p, int32_t tuning[4]) {
  if (!p || !tuning) return IB_ERR_INVALID_ARG;
  tuning[0] = p->chunk;
  tuning[1] = p->fe_ctas;
  tuning[2] = p->push_per_sm;
  tuning[3] = p->interp_per_sm;
  return IB_OK;
}

ib_status ib_plan_set_tuning(ib_plan* p, const int32_t tuning[4]) {
  if (!p || !tuning) return IB_ERR_INVALID_ARG;
  if (tuning[0] < kMinChunk || tuning[0] > kChunk || tuning[1] < 1 || tuning[1] > 5 ||
      tuning[2] < 1 || tuning[2] > 8 || tuning[3] < 1 || tuning[3] > 8)
    return IB_ERR_INVALID_ARG;
  p->chunk = tuning[0];
  p->fe_ctas = tuning[1];
  p->push_per_sm = tuning[2];
  p->interp_per_sm = tuning[3];
  return IB_OK;
}

}  // extern "C"

namespace ibfe {

ib_status autotune_with(ib_plan* p, const std::function<ib_status(cudaStream_t)>& run,
                        cudaStream_t s) {
  ib_status st = IB_OK;
  constexpr int kTimed = 5;
  cudaEvent_t a[kTimed] = {}, b[kTimed] = {};
  for (int k = 0; k < kTimed; ++k)
    if (!ok(cudaEventCreate(&a[k])) || !ok(cudaEventCreate(&b[k]))) st = IB_ERR_CUDA;
  // A scratch twice the L2 size, written before every timed call, so that
  // each call starts from a cold cache as a time step streaming the grid
  // does (back-to-back calls on a warm L2 ranked the candidates differently
  // from the timed steps).  Without it (allocation refused) the calls run
  // back to back.
  int dev = 0, l2 = 0;
  void* flush = nullptr;
  size_t flush_bytes = 0;
  if (ok(cudaGetDevice(&dev)) && ok(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev)) &&
      l2 > 0) {
    flush_bytes = 2 * (size_t)l2;
    if (!ok(cudaMalloc(&flush, flush_bytes))) {
      flush = nullptr;
      cudaGetLastError();
    }
  }
  // one warm-up call, then the median of five timed calls, enqueued back to
  // back as time steps are (a host wait between the calls put the launch
  // latency of each call's start into its time, which favoured other tunings
  // than the steps do)
  auto time_run = [&](float& ms) -> ib_status {
    ib_status r = run(s);
    for (int k = 0; k < kTimed && r == IB_OK; ++k) {
      if (flush && !ok(cudaMemsetAsync(flush, k, flush_bytes, s))) return IB_ERR_CUDA;
      if (!ok(cudaEventRecord(a[k], s))) return IB_ERR_CUDA;
      r = run(s);
      if (r == IB_OK && !ok(cudaEventRecord(b[k], s))) r = IB_ERR_CUDA;
    }
    if (r != IB_OK) return r;
    float t[kTimed];
    if (!ok(cudaEventSynchronize(b[kTimed - 1]))) return IB_ERR_CUDA;
    for (int k = 0; k < kTimed; ++k)
      if (!ok(cudaEventElapsedTime(&t[k], a[k], b[k]))) return IB_ERR_CUDA;
    std::sort(t, t + kTimed);
    ms = t[kTimed / 2];
    return IB_OK;
  };
  int32_t cur[4];
  ib_plan_get_tuning(p, cur);
  const int32_t cand[4][5] = {
      {1024, 512, 0, 0, 0}, {4, 3, 5, 2, 1}, {8, 3, 2, 0, 0}, {3, 8, 2, 0, 0}};
  // Each entry keeps its current value unless a candidate is faster by more
  // than 2%: many tunings lie within the timing noise of each other, and a
  // choice among those by noise alone moved the forward by 5% between runs.
  constexpr float kMargin = 0.98f;
  for (int k = 0; k < 4 && st == IB_OK; ++k) {
    int32_t best = cur[k];
    float best_ms = 0.f;
    st = time_run(best_ms);
    for (int j = 0; j < 5 && cand[k][j] && st == IB_OK; ++j) {
      if (cand[k][j] == cur[k]) continue;
      int32_t trial[4] = {cur[0], cur[1], cur[2], cur[3]};
      trial[k] = cand[k][j];
      ib_plan_set_tuning(p, trial);
      float ms = 0.f;
      st = time_run(ms);
      if (st == IB_OK && ms < kMargin * best_ms) {
        best = cand[k][j];
        best_ms = ms;
      }
    }
    cur[k] = best;
    ib_plan_set_tuning(p, cur);
  }
  for (int k = 0; k < kTimed; ++k) {
    if (a[k]) cudaEventDestroy(a[k]);
    if (b[k]) cudaEventDestroy(b[k]);
  }
  if (flush) cudaFree(flush);
  return st;
}

}  // namespace ibfe

extern "C" {

ib_status ib_plan_autotune(ib_plan* p, const ib_material* mats, int32_t n_mats,
                           const ib_pos* x, const void* u, void* stream, int32_t tuning[4]) {
  if (!p || !u) return IB_ERR_INVALID_ARG;
  ib_status st = check_pos(p, x);
  if (st != IB_OK) return st;
  cudaStream_t s = S(stream);
  const size_t rs = p->rsize;
  const size_t field = rs * 3 * (size_t)p->grid.n[0] * p->grid.n[1] * p->grid.n[2];
  void *G = nullptr, *f = nullptr, *U = nullptr;
  if (!ok(cudaMalloc(&G, rs * 3 * (size_t)p->N)) || !ok(cudaMalloc(&f, field)) ||
      !ok(cudaMalloc(&U, rs * 3 * (size_t)p->N)))
    st = IB_ERR_CUDA;
  if (st == IB_OK)
    st = autotune_with(
        p, [&](cudaStream_t t) { return ib_forward(p, mats, n_mats, x, u, G, f, U, t); }, s);
  if (G) cudaFree(G);
  if (f) cudaFree(f);
  if (U) cudaFree(U);
  if (st == IB_OK && tuning) ib_plan_get_tuning(p, tuning);
  return st;
}

ib_status ib_plan_set_profiling(ib_plan* p, int32_t enable) {
  if (!p) return IB_ERR_INVALID_ARG;
  if (enable && !p->ev) {
    const int cap = 8192;
    p->ev = new cudaEvent_t[cap];
    p->ev_stage = new int[cap / 2];
    for (int i = 0; i < cap; ++i)
      if (!ok(cudaEventCreate(&p->ev[i]))) {
        for (int j = 0; j < i; ++j) cudaEventDestroy(p->ev[j]);
        delete[] p->ev;
        delete[] p->ev_stage;
        p->ev = nullptr;
        p->ev_stage = nullptr;
        return IB_ERR_CUDA;
      }
    p->ev_cap = cap;
    p->ev_used = 0;
  }
  p->prof_on = enable ? 1 : 0;
  return IB_OK;
}

ib_status ib_plan_profile(ib_plan* p, void* stream, double* ms, int64_t* calls,
                          int64_t* launches, int32_t reset) {
  if (!p) return IB_ERR_INVALID_ARG;
  if (!ok(cudaStreamSynchronize(S(stream)))) return IB_ERR_CUDA;
  prof_flush(p);
  for (int i = 0; i < IB_STAGE_COUNT; ++i) {
    if (ms) ms[i] = p->prof_ms[i];
    if (calls) calls[i] = p->prof_calls[i];
    if (launches) launches[i] = p->prof_launches[i];
    if (reset) {
      p->prof_ms[i] = 0.0;
      p->prof_calls[i] = 0;
      p->prof_launches[i] = 0;
    }
  }
  return IB_OK;
}

ib_status ib_diag_wait_timeout(double ms, void* stream) {
  if (!(ms > 0.0) || ms > 10000.0) return IB_ERR_INVALID_ARG;
  cudaStream_t s = S(stream);
  int* d = nullptr;
  int h = 0;
  if (!ok(cudaMalloc(&d, sizeof(int)))) return IB_ERR_CUDA;
  ib_status st = ok(cudaMemsetAsync(d, 0, sizeof(int), s)) ? launch_wait_probe(d, ms, s)
                                                            : IB_ERR_CUDA;
  if (st == IB_OK && (!ok(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
                      !ok(cudaStreamSynchronize(s))))
    st = IB_ERR_CUDA;
  cudaFree(d);
  if (st != IB_OK) return st;
  return (h & kStatTimeout) ? IB_ERR_TIMEOUT : IB_OK;
}

ib_status ib_plan_sync_status(ib_plan* p, void* stream) {
  if (!p) return IB_ERR_INVALID_ARG;
  cudaStream_t s = S(stream);
  int st = 0;
  if (!ok(cudaStreamSynchronize(s)) ||
      !ok(cudaMemcpy(&st, p->dstatus, sizeof(int), cudaMemcpyDeviceToHost)) ||
      !ok(cudaMemset(p->dstatus, 0, sizeof(int))))
    return IB_ERR_CUDA;
  if (st & kStatNonfinite) return IB_ERR_NONFINITE;
  if (st & kStatInverted) return IB_ERR_INVERTED;
  if (st & kStatTimeout) return IB_ERR_TIMEOUT;
  return IB_OK;
}

}  // extern "C"
