// Internal declarations shared by the CUDA translation units of libibfe.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <functional>
#include <type_traits>

#include "ibfe.h"

namespace ibfe {

// Calls f(std::integral_constant<int, kEl>) for the plan's element type.
template <typename F>
void with_elem(int elem, F&& f) {
  if (elem == IB_ELEM_TET4)
    f(std::integral_constant<int, IB_ELEM_TET4>{});
  else if (elem == IB_ELEM_TET10)
    f(std::integral_constant<int, IB_ELEM_TET10>{});
  else
    f(std::integral_constant<int, IB_ELEM_HEX8>{});
}

constexpr int kTile = 8;            // Eulerian tile edge (cells) of the spread kernel
constexpr int kTileShift = 3;
constexpr int kSpreadWarps = 8;     // warps (private accumulators) per spread CTA
constexpr int kPackBits = 10;       // packed wrapped cell: x | y << 10 | z << 20
constexpr int kChunk = 1024;        // maximum points per spread / interp work item
constexpr int kMinChunk = 512;      // smallest work item the tuning may choose

// Device-side status bits latched by kernels (read by ib_plan_sync_status).
constexpr int kStatNonfinite = 1;
constexpr int kStatInverted = 2;
constexpr int kStatTimeout = 4;

// Parameter row: the law's parameters from column 0, T_a in column kTa.
constexpr int kParamRow = IB_PARAM_ROW;
constexpr int kTa = IB_PARAM_ROW - 1;

// Law sets of the force kernel's instantiations: bit m for ib_model m, and
// kLawAct for the active fibre stress.  The host launches the smallest
// instantiated set that covers the material table.
constexpr int kLawAct = 1 << 5;
constexpr int kLawBase = (1 << IB_NEO_HOOKEAN) | (1 << IB_FIBRE1) | (1 << IB_HO);
constexpr int kLawBaseAct = kLawBase | kLawAct;
constexpr int kLawAll = kLawBase | (1 << IB_STD_REINF) | (1 << IB_FIBRE2) | kLawAct;
// Not a law: the exact volumetric invariant of IB_FP32_SPLIT_DFVOL plans.
constexpr int kLawVolX = 1 << 6;

// Material table passed by value to kernels: the parameters in double, their
// FP32 roundings (read by the FP32 force kernels, which thus convert none on
// the device: GB300 converts at the FP64 rate), and whether the active
// tension is nonzero.
struct MatTable {
  int n;
  int model[IB_MAX_MATERIALS];
  int act[IB_MAX_MATERIALS];
  double p[IB_MAX_MATERIALS][kParamRow];
  float pf[IB_MAX_MATERIALS][kParamRow];
};

// Grid description used on the device.
struct GridDev {
  int n[3];
  int nt[3];          // tiles per dimension
  double h;
  double origin[3];
};

// Packed batches (batch.cu): several structures ("instances"), each with its
// own mesh, periodic grid and materials, held by one plan whose tiles,
// elements, nodes and material ids are the instances' ranges laid end to
// end.  A tile or an element finds its instance through the plan's
// tile_inst / elem_inst tables and the instance's grid in InstDev; a plan
// of one structure has no tables and uses its GridDev.
struct InstDev {
  int n[3];
  int nt[3];          // tiles per dimension
  int tile_base;      // first tile of the instance in the plan's numbering
  int pad;
  double h;
};

// Per-instance operands of one call on a packed plan: the instance's grid
// array (the spreading's output or the interpolated field) and the call's
// scalars (spreading: s0 = scale; interpolation: s0 = vscale, s1 = gscale).
struct GridCall {
  void* field;
  double s0, s1;
};

// One row of a material table in device memory (packed plans; rows indexed
// by the packed material ids), with the fields of a MatTable entry.
struct MatRow {
  int model;
  int act;
  double p[kParamRow];
  float pf[kParamRow];
};

// The derived fields of a table entry from its double parameters p.
inline void mat_entry_finish(const double* p, float* pf, int& act) {
  for (int k = 0; k < kParamRow; ++k) pf[k] = static_cast<float>(p[k]);
  act = p[kTa] != 0.0;
}

template <typename Real>
struct PosDev {
  const int32_t* cell;  // FP32 split
  const float* off;
  const double* x64;    // FP64
};

struct ib_plan_impl;

// Parameters of each ib_model, -1 for an unknown model.
inline int model_n_params(int model) {
  switch (model) {
    case IB_NEO_HOOKEAN: return 2;
    case IB_FIBRE1: return 4;
    case IB_HO: return 9;
    case IB_STD_REINF: return 4;
    case IB_FIBRE2: return 5;
    default: return -1;
  }
}

// Host check of one material: known model, matching parameter count, finite
// parameters and nonzero rate constants where the energy divides by them.
inline bool material_valid(const ib_material& m) {
  const int np = model_n_params(m.model);
  if (np < 0 || m.n_params != np) return false;
  for (int k = 0; k < np; ++k)
    if (!std::isfinite(m.params[k])) return false;
  if (!std::isfinite(m.Ta)) return false;
  if (m.model == IB_FIBRE1 && m.params[2] == 0.0) return false;
  if (m.model == IB_FIBRE2 && m.params[3] == 0.0) return false;
  if (m.model == IB_HO)
    for (int k : {1, 3, 5, 7})
      if (m.params[k] == 0.0) return false;
  return true;
}

}  // namespace ibfe

// The opaque plan.
struct ib_plan {
  int precision;         // ib_precision
  int quad;              // ib_quad: coupling points are Gauss points or nodes
  int elem;              // ib_elem
  int nc, nq;            // nodes and coupling points per element (hex 8, 8; P1 4, 4; P2 10, 4)
  int N, E;
  int64_t Q;             // coupling points: 8 E Gauss points or N nodes
  ibfe::GridDev grid;
  int ntiles;
  const int32_t* conn;
  const void* X;
  const void* fibres;
  const int32_t* mat_id;
  int max_mat_id;        // largest material id used by the mesh
  size_t rsize;          // sizeof(Real)

  // static derived data
  int32_t* inc_off;      // [N+1]
  int32_t* inc_idx;      // [8E]: corner*E + e
  void* mass;            // Real [N]
  void* inv_mass;        // Real [N]
  void* wj0;             // Real [8E] (q-major: q*E + e)

  // workspace
  void* elem_scratch;    // Real [3 nc][E]
  void* elem_scratch2;   // Real [3 nc][E]
  uint32_t* keys[2];     // [Q]
  int32_t* vals[2];      // [Q]
  int32_t* hist;         // radix histogram / offsets
  int hist_blocks;
  int32_t* tile_start;   // [ntiles]
  int32_t* tile_end;     // [ntiles]
  int32_t* tile_slot;    // [ntiles] first work item of each tile holding points (-1: none)
  int32_t* tile_nonempty;// [ntiles] number of work items of the tile
  int32_t* tile_near;    // [ntiles] 1 if a tile of its 3x3x3 neighbourhood holds points
  int32_t* tile_list;    // [max work items] tile of each work item
  int32_t* tile_list_near;// [ntiles] near tiles, ascending
  uint32_t* tile_vmax;   // [ntiles] FP32: bits of the largest |carried value| of each tile
  int32_t* tile_done;    // [ntiles] work items of the tile written (FP32 spreading, per call)
  int32_t* tile_sk;      // [4 ntiles] FP32: first block slot, exponent, item bound, items
  int32_t* tile_bcount;  // [2 * classify CTAs] per-CTA counts
  int32_t* tile_counters;// [8] [0] work items, [1] push counter, [2] interpolation counter,
                         //     [3] near count, [4] second interpolation's counter,
                         //     [6] FE force block counter
  int32_t* digit_tot;    // [256] radix digit totals
  double* rpart;         // [reduce CTAs][IB_MAX_MATERIALS*kParamRow] reduction partials
  cudaStream_t side;     // interpolation branch of ib_forward
  cudaStream_t hi;       // ib_forward's critical branch (force -> spread), high priority
  cudaStream_t zside;    // far-tile zero-fill of the spread
  cudaEvent_t ev_fork, ev_join;      // spread zero-fill fork / join
  cudaEvent_t ev_ffork, ev_fsorted, ev_fjoin, ev_hjoin;  // ib_forward branch events
  int sm_count, push_ctas, merge_ctas, interp_ctas[3];
  int interp_tma, interp_ctas_tma[3];  // FP32: TMA-staged interpolation available
  // launch tuning (ib_plan_set_tuning / ib_plan_autotune): points per work
  // item, FE-force CTAs per SM in the forward, caps on the spreading and
  // interpolation CTAs per SM (the occupancy maxima above are per-SM * sm_count)
  int chunk, fe_ctas, push_per_sm, interp_per_sm;
  void* spread_scratch;  // Real [slots][3][12^3] halo'd per-tile blocks
  int32_t* q_cell;       // packed wrapped cell per Gauss point (unsorted, gq order)
  void* q_off;           // Real [3][Q]
  void* q_val;           // Real [3][Q]
  int32_t* p_cell;       // sorted copies
  void* p_off;           // Real [3][Q]
  void* p_val;           // Real [3][Q]
  int32_t* p_idx;        // [Q] original gq
  void* node_tmp;        // Real [2][3][N] nodal work vectors (fused backward)
  // the fused backward's interpolation-adjoint branch, beside the spreading
  // adjoint: its own carried values, gradient outputs and projection scratch
  // (owned by plans of one structure; a packed plan's alias q_val, p_val,
  // gq_b and elem_scratch2)
  void* q_val_b;         // Real [3][Q] (FP64 plans; FP32 plans bin the values in one pass)
  void* p_val_b;         // Real [3][Q]
  void* gq_c;            // Real [3][Q]
  void* elem_scratch3;   // Real [3 nc][E]
  bool own_side_bufs;
  // penalty tethers (ib_plan_set_penalty; caller-owned device arrays)
  const int32_t* pen_nodes;
  int pen_n;
  const void* pen_w;
  double pen_kappa;
  double* pen_part;      // energy partials and their sum
  void* vol_jm1;         // float2 [force points][E]: exact J - 1 (IB_FP32_SPLIT_DFVOL only)
  void* gq_a;            // Real [3][Q] per-Gauss-point outputs (gq order)
  void* gq_b;            // Real [3][Q]
  double* epart;         // per-element partial sums: energy [E] (double), parameter
                         // gradients [kParamRow][E] (Real)
  double* ered;          // [IB_MAX_MATERIALS*kParamRow] reduced sums
  int* dstatus;          // device status word
  // packed batch (batch.cu); n_inst = 1 and null tables for one structure
  int n_inst;
  ibfe::InstDev* inst;   // [n_inst]
  int32_t* tile_inst;    // [ntiles] instance of each tile
  int32_t* elem_inst;    // [E] instance of each element
  ibfe::MatRow* mat_dev; // [n_mats_dev] material table (packed plans)
  int n_mats_dev;
  int mat_need;          // packed plans: bit m for each ib_model used, kLawAct if a T_a != 0
  int2* mat_range;       // [mat_cap] element range of each material id (reductions)
  int mat_cap;           // material ids the reduction buffers hold

  // per-stage profiling (host side; events only while prof_on)
  int prof_on;
  cudaEvent_t* ev;       // [ev_cap] start/stop pairs
  int* ev_stage;         // [ev_cap / 2]
  int ev_cap, ev_used;
  int prof_depth;        // open profiler intervals
  double prof_ms[IB_STAGE_COUNT];
  int64_t prof_calls[IB_STAGE_COUNT];
  int64_t prof_launches[IB_STAGE_COUNT];
};

namespace ibfe {

// ----------------------------------------------------------------------------
// host-side launchers (each file implements its group)
// ----------------------------------------------------------------------------
// fe_force.cu
ib_status launch_fe_force(ib_plan* p, const MatTable& mt, const void* x_cell_or_x64,
                          const float* off, void* elem_out, bool energy, cudaStream_t s);
ib_status launch_fe_force_adj(ib_plan* p, const MatTable& mt, const void* x_cell_or_x64,
                              const float* off, const void* v, void* elem_out, bool params,
                              cudaStream_t s);
// real_parts: the partials are in the plan's Real (parameter gradients),
// else in double (energy); the sums are in double either way
ib_status launch_reduce_parts(ib_plan* p, int nvals, int n_mats, cudaStream_t s,
                              bool real_parts);
// one instantiation of the force kernel's launcher (fe_kernel.cuh; explicit
// instantiations in fe_force_f32.cu, fe_force_adj.cu, fe_force_var.cu)
template <typename Real, typename S, bool kEnergy, bool kAdj, bool kParams, int kLaws, int kEl>
ib_status fe_run(ib_plan* p, const MatTable& mt, const void* xa, const float* off, const void* v,
                 void* out, cudaStream_t s);

// assemble.cu
// out = add + src over 3 N values (add optional, may be out)
ib_status launch_node_copy(ib_plan* p, const void* src, void* out, const void* add,
                           cudaStream_t s);
// out = add + mul node_scale * (gather of elem); add optional (may be out)
ib_status launch_node_gather(ib_plan* p, const void* elem, const void* node_scale, void* out,
                             cudaStream_t s, const void* add = nullptr, double mul = 1.0);
// weighted: the values are multiplied by the points' w_q j0 first (the
// interpolated values gq_a; not the position gradients gq_b)
ib_status launch_elem_project(ib_plan* p, const void* gq_vals, bool weighted, void* elem_out,
                              cudaStream_t s);
ib_status launch_plan_static(ib_plan* p, cudaStream_t s);

// points.cu
// Build Gauss points (position + carried value) and sort them by tile.
// val_kind: 0 = no value, 1 = w j0 sum_a N_a V_a / m_a from nodal V.
ib_status launch_points(ib_plan* p, const void* x_cell_or_x64, const float* off,
                        const void* nodal, int val_kind, cudaStream_t s);
ib_status launch_sort_points(ib_plan* p, bool with_val, cudaStream_t s);
// Carried values of already-built points (unsorted, into q_out or q_val), and
// their binned copy (from q_in or q_val into p_out or p_val; vmax: also the
// per-tile maxima the FP32 spreading's exponents take).
ib_status launch_point_values(ib_plan* p, const void* nodal, cudaStream_t s,
                              void* q_out = nullptr);
// zero_vmax false: the maxima were zeroed by the caller, ahead on the stream
// (or one it waits for)
ib_status launch_permute_values(ib_plan* p, cudaStream_t s, bool vmax = true,
                                const void* q_in = nullptr, void* p_out = nullptr,
                                bool zero_vmax = true);
// The carried values of the nodal field `nodal` at the binned points, into
// p_out (or p_val), with the per-tile maxima when vmax: FP32 binning in one
// pass (needs the binning done); FP64 plans through q_tmp (q_val if null)
// and a permutation; the nodal rule by a permutation of `nodal` itself.
ib_status launch_binned_values(ib_plan* p, const void* nodal, cudaStream_t s, bool vmax,
                               void* q_tmp = nullptr, void* p_out = nullptr);
int binned_values_launches(const ib_plan* p);

// spread.cu
// zero_fill false: the far-tile zeros were issued by launch_spread_zero
// calls (packed plans): each instance's output field and scale, replacing
// f and scale (device array, one GridCall per instance)
// vals: the binned carried values (default p_val)
ib_status launch_spread(ib_plan* p, double scale, void* f, cudaStream_t s, bool zero_fill = true,
                        const GridCall* calls = nullptr, const void* vals = nullptr);
// zeros of the tiles no coupling point reaches (needs the points binned)
ib_status launch_spread_zero(ib_plan* p, void* f, cudaStream_t s,
                             const GridCall* calls = nullptr);
ib_status spread_prepare(ib_plan* p);
size_t spread_scratch_bytes(int precision, int64_t slots);
int spread_launches(int precision);

// interp.cu
// mode 0: out_a[gq] = vscale * sum u prod phi (U^IB; the projection to the
//         nodes applies w_q j0)
// mode 1: out_a[gq] = vscale * sum u prod phi,
//         out_b[gq] = gscale * sum_c val_c * grad_chi(sum u^c prod phi)
// mode 2: only out_b (gradient) as in mode 1.
// calls / tmaps (packed plans): each instance's field, vscale and gscale,
// and each instance's tensor map of its field (device arrays; tmaps null:
// no TMA staging)
// io (optional, modes 1 and 2 only): the binned carried values read, the
// outputs a and b and the work-counter slot, for two interpolations in
// flight at once (default p_val, gq_a, gq_b, slot 2)
struct InterpIO {
  const void* vals;
  void* out_a;
  void* out_b;
  int counter;
};
ib_status launch_interp_points(ib_plan* p, const void* u, int mode, double vscale,
                               double gscale, cudaStream_t s, const GridCall* calls = nullptr,
                               const void* tmaps = nullptr, const InterpIO* io = nullptr);
// the tensor map of a FP32 field [3][n2][n1][n0] for the interpolation's TMA
// staging, written to `map` (128 bytes, host); false if unavailable
bool encode_velocity_map(const int n[3], const void* u, void* map);
constexpr size_t kTensorMapBytes = 128;
ib_status interp_prepare(ib_plan* p);
// the bounded-wait diagnostic (latches kStatTimeout into *status after ms)
ib_status launch_wait_probe(int* status, double ms, cudaStream_t s);

// capi.cu
// grid validation of ib_plan_create, and the plan builder behind it (also
// used for packed plans: `grid` is then the first instance's, `ntiles` the
// instances' total and mat_cap their total material count)
ib_status check_grid(const ib_grid* grid);
// packed: the plan of a batch (the backward's side-branch buffers alias the
// spreading adjoint's, which that plan's backward is done with when it forks)
ib_status plan_build(const ib_mesh* mesh, const GridDev& grid, int ntiles, int32_t quad,
                     int32_t precision, int mat_cap, cudaStream_t s, ib_plan** out,
                     bool packed = false);
void plan_free(ib_plan* p);
// the autotuner's coordinate descent over the plan's tuning, timing `run`
// (one warm-up and the median of five cold-L2 calls per candidate)
ib_status autotune_with(ib_plan* p, const std::function<ib_status(cudaStream_t)>& run,
                        cudaStream_t s);
// Per-instance operands of the forward and backward of a packed plan
// (device arrays of one GridCall or tensor map per instance): spread_f
// (f_i, h_i^-3), interp_u (u_i, 1, 0), tmaps_u, interp_gf (gf_i, h_i^-3,
// h_i^-4 gunit), tmaps_gf, spread_gu (gu_i, 1), interp_ug (u_i, 0, gunit / h_i).
struct PackedCalls {
  const GridCall* spread_f;
  const GridCall* interp_u;
  const void* tmaps_u;
  const GridCall* interp_gf;
  const void* tmaps_gf;
  const GridCall* spread_gu;
  const GridCall* interp_ug;
};
// The sequences of ib_forward and ib_backward (pc null: one structure, the
// fields and scalars are the arguments; pc set: a packed plan, the fields and
// h-dependent scalars are pc's).  params: compute the parameter gradients
// into p->ered (copied to gparams when it is not null).
ib_status forward_body(ib_plan* p, const MatTable& mt, const ib_pos* x, const void* u, void* G,
                       void* f, void* U, cudaStream_t s, const PackedCalls* pc);
ib_status backward_body(ib_plan* p, const MatTable& mt, int n_mats, const ib_pos* x,
                        const void* u, const void* G, const void* gG, const void* gf,
                        const void* gU, void* gx, void* gu, bool params, double* gparams,
                        cudaStream_t s, const PackedCalls* pc);
// profiler interval around a kernel inside a stage (sub-stage timing; its
// launches are counted by the enclosing stage)
int prof_begin(ib_plan* p, int stage, cudaStream_t s);
void prof_end(ib_plan* p, int idx, cudaStream_t s);
ib_status fe_force_adj_async(ib_plan* p, const ib_material* mats, int32_t n_mats,
                             const ib_pos* x, const void* v, void* Hv, bool params,
                             cudaStream_t s);

// penalty.cu: tethers of the solid boundary, applied after the nodal gather
bool penalty_on(const ib_plan* p);
ib_status launch_penalty(ib_plan* p, const ib_pos* x, void* G, bool energy, cudaStream_t s);
const double* penalty_energy_dev(const ib_plan* p);
// Hv -= mul kappa w v at the tethered nodes
ib_status launch_penalty_adj(ib_plan* p, const void* v, void* Hv, cudaStream_t s,
                             double mul = 1.0);
size_t penalty_scratch_doubles();

// fluid.cu
ib_status fluid_step_async(ib_fluid* fl, const void* u, const void* f, void* u_next, void* p,
                           double* residuals, cudaStream_t s);
bool fluid_matches(const ib_fluid* fl, const ib_plan* p);
double fluid_dt(const ib_fluid* fl);
// x += dt U on the plan's position storage (split cells carry whole cells)
ib_status launch_advance_positions(ib_plan* p, const ib_pos* x, const void* U, double dt,
                                   cudaStream_t s);

// tiles.cu
ib_status launch_classify_tiles(ib_plan* p, cudaStream_t s);
int classify_blocks(int ntiles);
int64_t max_work_items(int ntiles, int64_t Q);
int sort_key_bits(int ntiles);
constexpr int kReduceCTAs = 128;

}  // namespace ibfe
