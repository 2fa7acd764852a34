/*
 * ibfe -- immersed-boundary coupling operators on one GB300 (sm_103a).
 *
 * C ABI of the CUDA library libibfe.so.  It implements the Lagrangian-Eulerian
 * coupling step of the matrix-free immersed-boundary method of arXiv
 * 2503.22695 (Ma, Cai, Wang, Luo, Gao, "Fully GPU-Accelerated Immersed
 * Boundary Method for Fluid-Structure Interaction in Complex Cardiac Models"):
 *
 *   ib_fe_force  nodal force of the hyperelastic structure, Section 4.4
 *                F_i = -sum_{q in H_q} P(X_q) : grad_X phi_i(X_q) w_q with P from
 *                the strain energies of Section 3 / Section 6.3
 *   ib_spread    spreading f = E(X, F), Section 2 Eq. (1), discrete form of
 *                Section 4.4 (quadrature by the element Gauss rule)
 *   ib_interp    interpolation U = I(X, u), Section 2 Eq. (2), discrete form of
 *                Section 4.4 (U^IB at Gauss points, then the lumped L2
 *                projection onto the finite-element space)
 *   and their adjoints (vector-Jacobian products).  The adjointness of
 *   spreading and interpolation under one quadrature (Section 4.4) is the
 *   identity  h^3 sum_faces f . u = sum_nodes G . U.
 *
 *   The coupling points are chosen per plan (ib_quad): the Gauss points of
 *   the elements (IB_QUAD_GAUSS2, above) or the nodes themselves
 *   (IB_QUAD_NODAL, the nodal quadrature rule N_q of Section 4.4: U_a is
 *   U^IB at the node's displaced position, and f spreads the nodal forces
 *   G_a from the nodes).  The nodal force is the Gauss-rule one in both.
 *
 * Conventions
 *   Grid    periodic box [origin, origin + n h); fields are [3][n2][n1][n0]
 *           (x fastest).  Component c lives on the lower c-faces: face
 *           (i0,i1,i2) of component c sits at origin_d + (i_d + s_cd) h with
 *           s_cd = 0 if d == c and 1/2 otherwise (the MAC staggering of
 *           Section 4.3).  Requires 8 <= n_d <= 1024 and n_d % 8 == 0.
 *   Kernel  4-point Peskin delta, delta_h(x) = h^-3 prod_d phi(x_d / h).
 *   Mesh    trilinear hexahedra (VTK corner order), conn [8][E] int32,
 *           reference coordinates X [3][N]; 2x2x2 Gauss rule, unit weights.
 *   Positions (ib_pos)
 *           IB_FP32_SPLIT: cell int32 [3][N] + off float [3][N] in [0,1); the
 *           node sits at origin + (cell + off) h.  Cells are NOT wrapped (a
 *           structure may straddle the periodic seam).
 *           IB_FP64: x64 double [3][N] absolute coordinates.
 *   Mass    lumped: m_a = sum_{e,q} N_a(xi_q) w_q j0.
 *   Units   G is the integrated nodal force; f is a force density (delta_h
 *           carries h^-3); u, U are velocities.
 *   Floating type of every array argument named "Real" below: float for
 *   IB_FP32_SPLIT plans, double for IB_FP64 plans.
 *
 * Ownership, streams and errors
 *   All array pointers are caller-owned DEVICE memory unless marked host.  The
 *   plan keeps the mesh pointers given at creation (the caller keeps them
 *   alive and unchanged) and owns only derived data and workspace, allocated
 *   once in ib_plan_create; no operator call allocates.  Every call is
 *   asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream)
 *   except where a host output (energy, gparams) is requested: then it
 *   synchronises the stream before returning.  Argument errors return
 *   IB_ERR_INVALID_ARG before launching anything; launch failures return
 *   IB_ERR_CUDA.  Conditions found on the device (non-finite or out-of-range
 *   positions, inverted elements) are latched in the plan and reported by
 *   ib_plan_sync_status.  A plan is not thread-safe: calls on one plan must
 *   be ordered on one stream.
 */
#ifndef IBFE_H
#define IBFE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IB_OK = 0,
  IB_ERR_INVALID_ARG = 1,
  IB_ERR_CUDA = 2,
  IB_ERR_NONFINITE = 3,   /* device: a position offset outside [0,1) or NaN/Inf */
  IB_ERR_CAPACITY = 4,    /* a size exceeds a documented limit */
  IB_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  IB_ERR_UNSUPPORTED = 6, /* valid but unsupported configuration */
  IB_ERR_INVERTED = 7     /* device: an element with det(dX/dxi) <= 0 */
} ib_status;

typedef enum {
  IB_NEO_HOOKEAN = 0, /* Psi = a (I1bar - 3) + kappa/2 (ln J)^2 (Section 6.3); params {a, kappa} */
  IB_FIBRE1 = 1,      /* Psi_2 of Section 3; params {C1, af, bf, kappa} */
  IB_HO = 2,          /* Psi_4 Holzapfel-Ogden (Section 3); params {a, b, af, bf, as, bs, afs, bfs, kappa} */
  IB_STD_REINF = 3,   /* Psi_1 modified standard reinforcing model (Section 3), transversely
                         isotropic in I4f and I5f; params {G_T, G_L, E_L, kappa} */
  IB_FIBRE2 = 4       /* Psi_3 fibre-reinforced model 2 (Section 3): C10 (exp[C01 (I1bar - 3)] - 1)
                         + af/(2 bf)(exp[bf (I4f - 1)^2] - 1), fibres also resist compression;
                         params {C10, C01, af, bf, kappa} */
} ib_model;

/* IB_FP32_SPLIT: FP32 arithmetic on split positions; J - 1 (the volumetric
 *   term) and the fibre invariant I4f - 1 (the exponential fibre term near
 *   I4f = 1) are accumulated as compensated FP32 pairs (error-free products
 *   and sums), as accurate as twice the working precision, without FP64
 *   instructions.
 * IB_FP64: every array and every operation in double.
 * IB_FP32_SPLIT_F32STAB: as IB_FP32_SPLIT with those sums in plain FP32,
 *   using the same cancellation-free formulas.  Nodal forces stay within
 *   1e-5 relative L2 of the FP64 definition, but the Hessian-vector product
 *   of ib_fe_force_adj loses accuracy (6.7e-5 relative on a 256^3 ventricle
 *   workload, against 2e-5 with IB_FP32_SPLIT) for no speed gain on GB300.
 * IB_FP32_SPLIT_DFVOL: as IB_FP32_SPLIT, with J - 1 at every force point from
 *   double-float kinematics: node differences formed without rounding from
 *   the split positions and the reference coordinates, the Jacobians
 *   DX = dX/dxi and DU = du/dxi, and det(DX + DU) - det(DX) expanded, all in
 *   pairs of FP32 numbers (no FP64 instruction).  For nearly incompressible
 *   materials, where |J - 1| << |F - I|: there J - 1 from the FP32
 *   displacement gradient (IB_FP32_SPLIT) carries a relative error near
 *   1e-7 |F - I| / |J - 1| (1.3e-3 in the nodal force at kappa / a = 2e4,
 *   |J - 1| <= 6e-5), this option one near 1e-13 |F - I| / |J - 1|.  The
 *   force kernel costs about three times as much. */
typedef enum {
  IB_FP32_SPLIT = 0,
  IB_FP64 = 1,
  IB_FP32_SPLIT_F32STAB = 2,
  IB_FP32_SPLIT_DFVOL = 3
} ib_precision;

#define IB_MAX_MATERIALS 8
/* Width of a parameter-gradient row: the law's n_params parameters from
 * column 0, zeros up to column 8, d/dT_a in column 9. */
#define IB_PARAM_ROW 10

/* Element types.  IB_ELEM_HEX8: trilinear hexahedra, VTK corner order, the
 * 2x2x2 Gauss rule (8 coupling points per element).  IB_ELEM_TET4: linear
 * tetrahedra (the element of the paper's valve meshes, Section 5), VTK order
 * with positive volume, the symmetric 4-point rule of degree 2 (4 coupling
 * points per element); the P1 force is evaluated exactly at the centroid.
 * IB_ELEM_TET10: quadratic tetrahedra (P2, the element of the paper's Cook
 * membrane, Section 5), VTK order: the 4 vertices, then the nodes of edges
 * 01, 12, 02, 03, 13, 23; the same 4-point rule for the force and the
 * coupling (4 coupling points per element); lumped mass by diagonal scaling
 * (the element's sums of w j0 N_a^2, scaled to its volume), since the P2 row
 * sums of a vertex are negative. */
typedef enum { IB_ELEM_HEX8 = 0, IB_ELEM_TET4 = 1, IB_ELEM_TET10 = 2 } ib_elem;

typedef struct {
  int32_t n_nodes, n_elems;
  const int32_t* conn;   /* device [8][n_elems] (hexahedra), [4][n_elems] or [10][n_elems] (tetrahedra) */
  const void* X;         /* device Real [3][n_nodes] reference coordinates */
  const void* fibres;    /* device Real [6][n_elems]: e_f then e_s, or NULL (e_f = x, e_s = y) */
  const int32_t* mat_id; /* device [n_elems] index into the material table, or NULL (all 0) */
  int32_t elem_type;     /* ib_elem; 0 (hexahedra) when zero-initialised */
} ib_mesh;

typedef struct {
  int32_t n[3];
  double h;
  double origin[3];
} ib_grid;

typedef struct {
  const int32_t* cell; /* IB_FP32_SPLIT: device [3][N] */
  const float* off;    /* IB_FP32_SPLIT: device [3][N], each in [0,1) */
  const double* x64;   /* IB_FP64: device [3][N] */
  double grad_unit;    /* position derivatives returned by the adjoints (gx of
                          ib_spread_adj, ib_interp_adj, ib_backward; Hv of
                          ib_fe_force_adj) are per displacement of this length:
                          0 (or 1) = per unit of the grid's length (d/dx); h =
                          per unit of the split offset (d/d off).  Not
                          finite or negative: IB_ERR_INVALID_ARG */
} ib_pos;

typedef struct {
  int32_t model;     /* ib_model */
  int32_t n_params;  /* the model's count: 2, 4, 9, 4 or 5 */
  double params[9];  /* host values */
  double Ta;         /* active fibre tension T_a (Section 6.1) at the current time, in
                        the units of params; 0 = passive.  Adds P^a = T F e_f (x) e_f,
                        T = T_a (1 + 4.9 (sqrt(I4f) - 1)), to the law's stress, and its
                        potential T_a/2 [(1 - 4.9)(I4f - 1) + 4.9 (2/3)(I4f^(3/2) - 1)]
                        to the energy; finite (else IB_ERR_INVALID_ARG) */
} ib_material;

typedef struct ib_plan ib_plan;

/* Coupling points of spreading and interpolation (Section 4.4). */
typedef enum {
  IB_QUAD_GAUSS2 = 0, /* the 2x2x2 Gauss points of every element (8 E points) */
  IB_QUAD_NODAL = 1   /* the nodes (N points): the nodal rule N_q, w_q = m_a */
} ib_quad;

/* Create a plan for one mesh on one grid: validates the mesh, builds the
 * node->(element, corner) incidence lists (a gather index, not a matrix), the
 * lumped mass and the Gauss weights w_q j0, and allocates all workspace.
 * `quad` is an ib_quad, `precision` an ib_precision.  Synchronises `stream`.
 * Returns IB_ERR_INVERTED if an element has a non-positive reference
 * Jacobian at a Gauss point, IB_ERR_INVALID_ARG for an unknown quad or
 * precision. */
ib_status ib_plan_create(const ib_mesh* mesh, const ib_grid* grid, int32_t quad,
                         int32_t precision, void* stream, ib_plan** out);
ib_status ib_plan_destroy(ib_plan* plan);

/* Copy the plan's lumped mass m [N] (Real) into `mass` (device).  m_a is the
 * row sum sum_{e,q} N_a(xi_q) w_q j0 of the consistent mass by the element
 * rule (hexahedra, P1 tetrahedra: the nodal-rule weight of Section 4.4), and
 * for P2 tetrahedra the element diagonal sum_q N_a(xi_q)^2 w_q j0 scaled to
 * the element's volume, summed over the node's elements.  Nodes in no element
 * have m = 0 and receive zero from the projection. */
ib_status ib_lumped_mass(ib_plan* plan, void* mass, void* stream);

/* Nodal forces G (device Real [3][N], overwritten) of Section 4.4 for the
 * material table `mats` (host, n_mats <= IB_MAX_MATERIALS).  If energy is
 * non-NULL (host) the total elastic energy sum_{e,q} Psi(F_q) w_q j0 is
 * written there and the stream is synchronised.  G = -dE/dx. */
ib_status ib_fe_force(ib_plan* plan, const ib_material* mats, int32_t n_mats,
                      const ib_pos* x, void* G, double* energy, void* stream);

/* Spreading: f (device Real [3][n2][n1][n0], every entry overwritten) from
 * nodal forces G (device Real [3][N]).  Gauss rule: F_q = sum_a N_a G_a / m_a,
 * f^c(face) = sum_q F_q^c w_q j0 delta_h(x_face - chi_q).  Nodal rule:
 * f^c(face) = sum_a G_a^c delta_h(x_face - x_a).  The result is bitwise
 * reproducible (fixed summation order, no floating-point atomics). */
ib_status ib_spread(ib_plan* plan, const ib_pos* x, const void* G, void* f, void* stream);

/* Interpolation: U (device Real [3][N], overwritten) from the MAC velocity u
 * (device Real [3][n2][n1][n0]): U^IB_q = sum_faces u h^3 delta_h(x_face - chi_q),
 * Gauss rule: U_a = m_a^-1 sum_q N_a w_q j0 U^IB_q; nodal rule: U_a = U^IB at x_a. */
ib_status ib_interp(ib_plan* plan, const ib_pos* x, const void* u, void* U, void* stream);

/* Forward coupling in one call, sharing one Gauss-point sort:
 * G = fe_force(x), f = spread(x, G), U = interp(x, u). */
ib_status ib_forward(ib_plan* plan, const ib_material* mats, int32_t n_mats,
                     const ib_pos* x, const void* u, void* G, void* f, void* U,
                     void* stream);

/* Adjoint of spreading for the cotangent gf (device Real [3][grid]):
 * gG = (df/dG)^T gf (device Real [3][N]), and, if gx is non-NULL,
 * gx = (df/dx)^T gf (device Real [3][N]).  Both overwritten. */
ib_status ib_spread_adj(ib_plan* plan, const ib_pos* x, const void* G, const void* gf,
                        void* gG, void* gx, void* stream);

/* Adjoint of interpolation for the cotangent gU (device Real [3][N]):
 * gu = (dU/du)^T gU (device Real [3][grid], every entry overwritten, bitwise
 * reproducible), and, if gx is non-NULL, gx = (dU/dx)^T gU (device Real [3][N]). */
ib_status ib_interp_adj(ib_plan* plan, const ib_pos* x, const void* u, const void* gU,
                        void* gu, void* gx, void* stream);

/* Adjoint of the nodal force for the cotangent v (device Real [3][N]):
 * Hv = (dG/dx)^T v = (dG/dx) v = -(d^2 E/dx^2) v (device Real [3][N]), and, if
 * gparams (host double [n_mats][IB_PARAM_ROW]) is non-NULL, gparams[m][k] =
 * v . dG/dtheta_{m,k} for the n_params of material m, gparams[m][9] =
 * v . dG/dT_a (stream synchronised). */
ib_status ib_fe_force_adj(ib_plan* plan, const ib_material* mats, int32_t n_mats,
                          const ib_pos* x, const void* v, void* Hv, double* gparams,
                          void* stream);

/* Backward of ib_forward (its vector-Jacobian product), fused: given the
 * cotangents gG [3][N], gf [3][grid] and gU [3][N] of the forward outputs G,
 * f and U (device Real; any may be NULL, meaning zero), computes
 *   gx = (dG/dx)^T gG_t + (df/dx)^T gf + (dU/dx)^T gU   (device Real [3][N]),
 *        with gG_t = gG + (df/dG)^T gf, the spreading's share of the force cotangent;
 *   gu = (dU/du)^T gU                                   (device Real [3][grid], if gu);
 *   gparams[m][k] = gG_t . dG/dtheta_{m,k}              (device double [n_mats][IB_PARAM_ROW],
 *                                                         column 9 for T_a, if gparams).
 * This is the composition of ib_spread_adj, ib_interp_adj and ib_fe_force_adj
 * (Section 4.4: spreading and interpolation are adjoint to each other), with
 * the Gauss points built and binned once and the force adjoint (FP64-pipe
 * bound) run beside the interpolation adjoint.  G must be the nodal force of
 * the forward at the same x (needed when gf is given).  gx is overwritten;
 * gu must be given when gU is, and is overwritten (bitwise reproducible).
 * Asynchronous on `stream`; errors: IB_ERR_INVALID_ARG (missing or
 * misaligned arguments), the launch and device errors of its parts. */
ib_status ib_backward(ib_plan* plan, const ib_material* mats, int32_t n_mats, const ib_pos* x,
                      const void* u, const void* G, const void* gG, const void* gf,
                      const void* gU, void* gx, void* gu, double* gparams, void* stream);

/* Launch tuning of a plan, four entries:
 *   [0] points per work item of spreading and interpolation, 512..1024
 *       (a tile's points are cut into items of at most this many);
 *   [1] FE-force CTAs per SM in ib_forward, 1..5 (its persistent grid leaves
 *       the rest of each SM to the binning and interpolation beside it);
 *   [2] cap on the spreading CTAs per SM, 1..8;
 *   [3] cap on the interpolation CTAs per SM, 1..8.
 * Defaults {1024, 4, 8, 3} (a cap above the occupancy limit means none).
 * Results do not depend on the tuning for FP32 plans (bitwise); FP64 plans
 * change only in the summation order of the spreading.  get/set are host
 * operations on the plan; set returns IB_ERR_INVALID_ARG out of range. */
ib_status ib_plan_get_tuning(const ib_plan* plan, int32_t tuning[4]);
ib_status ib_plan_set_tuning(ib_plan* plan, const int32_t tuning[4]);

/* Autotuner: times ib_forward on the given inputs for candidate tunings
 * (coordinate descent over the four entries in order, from the plan's
 * current tuning: items of 1024 or 512 points; 1 to 5 force CTAs per SM;
 * spreading and interpolation caps 8, 3 or 2; one warm-up and the median of
 * five timed calls each, every timed call after a write of twice the L2
 * size, so that it starts from a cold cache).  An entry changes only for a
 * candidate more than 2% faster than the best so far.  Writes the choice to
 * `tuning` (host, 4 entries) if non-NULL.  Allocates temporary output buffers and the L2
 * scratch (without the scratch, if that allocation fails) and synchronises
 * `stream`. */
ib_status ib_plan_autotune(ib_plan* plan, const ib_material* mats, int32_t n_mats,
                           const ib_pos* x, const void* u, void* stream, int32_t tuning[4]);

/* Penalty tethers of the solid boundary (Section 5: Cook's membrane's fixed
 * face, kappa = 1e6; the aortic valve's fixed outer tube, kappa = 5e6).  From
 * this call on, the nodal force of the plan's entry points (ib_fe_force,
 * ib_forward, ib_step) includes G_a -= kappa w_a (x_a - X_a) for each listed
 * node a, and the energy kappa/2 sum w_a |x_a - X_a|^2; the force adjoints
 * (ib_fe_force_adj, ib_backward) include its Jacobian, -kappa w_a on the
 * listed nodes (no parameter gradient for kappa).  nodes: device int32 [n],
 * distinct node indices (entries outside [0, N) are ignored); weights: device
 * Real [n], or NULL for the lumped mass m_a (the volume weight of the node).
 * Both arrays are the caller's and must stay valid while set.  n = 0 or
 * kappa = 0 removes the tethers.  Not available to the batched form.
 * Errors: IB_ERR_INVALID_ARG (n < 0 or > N, nodes NULL with n > 0, kappa
 * negative or not finite). */
ib_status ib_plan_set_penalty(ib_plan* plan, const int32_t* nodes, int32_t n,
                              const void* weights, double kappa);

/* ---------------------------------------------------------------------------
 * Batched form: many independent structures, each with its own hexahedral
 * mesh, periodic grid and material table (a parameter sweep, for instance),
 * run together.  The paper runs one structure at a time; batching is a
 * service of this library.
 *
 * ib_batch_create packs the instances into one plan: their meshes laid end
 * to end, their grids' tiles numbered consecutively, with device tables that
 * give every tile and element its instance.  Each stage of the coupling is
 * then one launch over all instances (one force kernel over all elements,
 * one persistent spreading kernel whose work counter spans every instance's
 * tiles, one merge, one persistent interpolation), with each instance's
 * fields and h-dependent scales read from per-instance tables.  The forward
 * (the sequence of ib_forward) and the backward (that of ib_backward, with
 * the parameter gradients kept on the device) are each captured once in a
 * CUDA graph and replayed with one launch.  The packed plan's tuning is
 * chosen by the autotuner of ib_plan_autotune, timed on the batch's own
 * forward.  Every instance's results equal, bit for bit, those of
 * ib_forward / ib_backward on a plan of that instance alone.
 *
 * Instances: IB_ELEM_HEX8 meshes with n_elems > 0, the Gauss rule, FP32
 * split positions (precision must be IB_FP32_SPLIT), 1..IB_MAX_MATERIALS
 * materials each, one common x.grad_unit, f, u (and gf, gu) 16-byte
 * aligned; penalty tethers are not available.  Violations give
 * IB_ERR_INVALID_ARG (grids as ib_plan_create: IB_ERR_UNSUPPORTED).  All
 * pointers in ib_instance are device memory that must stay valid and fixed
 * for the batch's lifetime (the graphs bake them in); update the data in
 * place between replays.  Synchronises `stream` at creation.
 * ------------------------------------------------------------------------- */
typedef struct {
  ib_mesh mesh;
  ib_grid grid;
  int32_t n_mats;
  ib_material mats[IB_MAX_MATERIALS]; /* host copy taken at creation */
  ib_pos x;
  const void* u;  /* [3][grid] */
  void* G;        /* [3][N]   forward outputs */
  void* f;        /* [3][grid] */
  void* U;        /* [3][N] */
  const void* gU; /* [3][N]    backward inputs: cotangents of U, f (NULL: no backward) */
  const void* gf; /* [3][grid] */
  const void* gG; /* [3][N]    cotangent of G, or NULL (zero) */
  void* gu;       /* [3][grid] backward outputs (ib_backward): d/du */
  void* gx;       /* [3][N]    d/dx, all three terms */
} ib_instance;

typedef struct ib_batch ib_batch;

ib_status ib_batch_create(int32_t n, const ib_instance* inst, int32_t precision, void* stream,
                          ib_batch** out);
/* Replay the forward (resp. backward) graph on `stream` (asynchronous). */
ib_status ib_batch_forward(ib_batch* batch, void* stream);
ib_status ib_batch_adjoint(ib_batch* batch, void* stream);
/* Parameter gradients (ib_backward's gparams) of every instance's last
 * backward replay, host double [n][IB_MAX_MATERIALS][IB_PARAM_ROW] (entries past an
 * instance's n_mats are zero); synchronises `stream`. */
ib_status ib_batch_gparams(ib_batch* batch, double* gparams, void* stream);
/* The packed plan's tuning (as ib_plan_get_tuning). */
ib_status ib_batch_get_tuning(const ib_batch* batch, int32_t tuning[4]);
ib_status ib_batch_destroy(ib_batch* batch);

/* ---------------------------------------------------------------------------
 * Fluid step and the explicit IB step (Section 4.2).  The momentum equation
 * is split by Chorin's projection on the periodic MAC grid of a plan:
 *   rho/dt (u* - u^n) - mu Lap_h u* = f,   Lap_h p = div_h u* / dt,
 *   u^{n+1} = u* - dt grad_h p,
 * with (div u)(i) = sum_c (u^c(i+e_c) - u^c(i))/h, (grad p)^c(i) =
 * (p(i) - p(i-e_c))/h and the 7-point Lap_h = div_h grad_h; both solves by
 * geometric multigrid V-cycles (red-black Gauss-Seidel, 2 pre- and 2
 * post-sweeps; levels halve every dimension while all are even, none is
 * below 4 and the largest exceeds 8; the coarsest is solved in one CTA's
 * shared memory).
 * The cycle counts are fixed (default 2 Helmholtz and 6 Poisson cycles in
 * FP32, 3 and 12 in FP64), so a step involves no host round trip (without
 * residuals it runs as one CUDA graph, captured per set of field pointers);
 * ib_fluid_step can report the residuals reached.  Fields: u, f, u_next device Real [3][n2][n1][n0] (component c on
 * the lower c-faces, as everywhere in this API), p device Real [n2][n1][n0]
 * at cell centres with zero mean.  Real is float for the split precisions and
 * double for IB_FP64.  The box is periodic; the paper's no-slip walls are not
 * modelled.
 * ------------------------------------------------------------------------- */
typedef struct ib_fluid ib_fluid;

/* Fluid solver for `grid` (every n_d even, 4..4096; IB_ERR_UNSUPPORTED for an
 * odd size or a coarsest level above 8192 cells, IB_ERR_CAPACITY for
 * 3 n0 n1 n2 >= 2^31) with density rho > 0,
 * viscosity mu >= 0 and time step dt > 0.  Allocates its multigrid hierarchy
 * (about 1.6 field volumes) on the current device. */
ib_status ib_fluid_create(const ib_grid* grid, int32_t precision, double rho, double mu,
                          double dt, void* stream, ib_fluid** out);
ib_status ib_fluid_destroy(ib_fluid* fluid);
/* V-cycles per Helmholtz solve (all three components together) and per
 * Poisson solve, each in [1, 100]. */
ib_status ib_fluid_set_cycles(ib_fluid* fluid, int32_t helmholtz_cycles, int32_t poisson_cycles);
ib_status ib_fluid_get_cycles(const ib_fluid* fluid, int32_t cycles[2]);
/* Number of multigrid levels (the finest included). */
ib_status ib_fluid_levels(const ib_fluid* fluid, int32_t* levels);
/* One projection step: u_next (may alias u) and p (NULL: kept internally)
 * from u and the force density f (NULL: no force).  If residuals (host,
 * 2 doubles) is non-NULL, also the relative residuals ||rhs - A x|| / ||rhs||
 * of the Helmholtz and Poisson solves (synchronises `stream`).  Asynchronous
 * otherwise. */
ib_status ib_fluid_step(ib_fluid* fluid, const void* u, const void* f, void* u_next, void* p,
                        double* residuals, void* stream);

/* One explicit IB step (Section 4.2) on the plan's structure and the fluid's
 * grid (same lattice, spacing and precision as the plan, else
 * IB_ERR_INVALID_ARG): the nodal force G of the configuration x^n, the force
 * density f spread from it at x^n, the fluid step from u^n to u^{n+1}, the
 * new velocity interpolated at x^n (U, onto the nodes as in ib_interp), and
 * the nodes moved by dt U.  x is updated in place (split positions carry
 * whole cells into `cell`, offsets stay in [0,1)); u holds u^n on entry and
 * u^{n+1} on return; G [3][N], f [3][grid], U [3][N] and p [grid] (NULL:
 * kept internally) are outputs.  Asynchronous on `stream`. */
ib_status ib_step(ib_plan* plan, ib_fluid* fluid, const ib_material* mats, int32_t n_mats,
                  const ib_pos* x, void* u, void* G, void* f, void* U, void* p, void* stream);

/* Total elastic energy sum_{e,q} Psi(F_q) w_q j0 of an FP32 split-position
 * hexahedral mesh (IB_ERR_UNSUPPORTED for tetrahedra), without a plan and
 * without allocating anything, for callers that cannot call cudaMalloc:
 * runtimes that hand all device memory to their own pool up front (a
 * cudaMalloc of theirs would fail or fragment it), and loops that must not
 * enter the allocator, which may synchronise the device.  The paper has no
 * counterpart of this entry point; it is a service of this library.
 *   mesh    as for ib_plan_create, X and fibres float; n_elems <= 262144,
 *           else IB_ERR_CAPACITY (nothing is launched).
 *   mats    host material table, n_mats <= IB_MAX_MATERIALS.
 *   x       split positions (cell, off); h is the grid spacing.
 *   energy  device double, written with the result (NaN if the mesh holds a
 *           node index outside [0, n_nodes) or a material index outside
 *           [0, n_mats)).
 * Scratch: a file-scope device array (about 2 MiB) that every GPU loading the
 * library keeps until exit; each call overwrites what it reads, so nothing
 * needs clearing, but calls that overlap on the GPU race on it and must not
 * be issued.  The first call on a device looks up the array's device address
 * (no allocation); make that first call before any stream capture.
 * Asynchronous on `stream`; launch errors return IB_ERR_CUDA. */
ib_status ib_fe_energy_noalloc(const ib_mesh* mesh, const ib_material* mats, int32_t n_mats,
                               const ib_pos* x, double h, double* energy, void* stream);

/* Synchronise `stream` and return (then clear) the first device-detected
 * condition latched since the last call (IB_OK if none). */
ib_status ib_plan_sync_status(ib_plan* plan, void* stream);

/* Per-stage profiling.  While enabled, every operator records a pair of
 * CUDA events around each of its stages on its stream (a few microseconds
 * of overhead per stage; do not enable during CUDA-graph capture).
 * ib_plan_profile synchronises the stream and returns, per stage, the summed
 * elapsed milliseconds (ms, host double[IB_STAGE_COUNT], nullable), the
 * number of operator calls that ran the stage (calls, host int64[...],
 * nullable) and the number of kernels launched in it (launches, host
 * int64[...], nullable; counted whether or not profiling is enabled), since
 * the last reset; reset != 0 clears the counters afterwards.  This is a
 * measurement facility of this library, not part of the method. */
typedef enum {
  IB_STAGE_FORCE = 0,   /* per-element stress and corner forces */
  IB_STAGE_GATHER = 1,  /* element -> node gathers */
  IB_STAGE_POINTS = 2,  /* Gauss-point positions and carried values */
  IB_STAGE_SORT = 3,    /* stable radix sort by Eulerian tile + reorder */
  IB_STAGE_SPREAD = 4,  /* tile-owned spreading onto the grid */
  IB_STAGE_INTERP = 5,  /* Gauss-point interpolation (and its gradients) */
  IB_STAGE_PROJECT = 6, /* Gauss point -> element corner projection */
  IB_STAGE_REDUCE = 7,  /* deterministic energy / parameter reductions */
  IB_STAGE_SPREAD_PUSH = 8, /* the accumulation kernel inside IB_STAGE_SPREAD (FP32 plans; a
                               sub-interval, not additive; its launches count in the stage) */
  IB_STAGE_COUNT = 9
} ib_stage;
ib_status ib_plan_set_profiling(ib_plan* plan, int32_t enable);
ib_status ib_plan_profile(ib_plan* plan, void* stream, double* ms, int64_t* calls,
                          int64_t* launches, int32_t reset);

/* Active tension waveform T_a(t) of Section 6.1 in Pa, t in seconds: 0 for
 * t < 0.5; 84260 (1 - exp(-(t - 0.5)^2 / 0.005)) up to 0.65;
 * 84260 (1 - exp(-(0.8 - t)^2 / 0.005)) up to 0.8; periodic with the 0.8 s
 * cardiac cycle.  Host function (no device work); divide by 1000 for
 * parameter sets in kPa.  The value goes into ib_material.Ta. */
double ib_active_tension(double t);

/* Failure-path diagnostic: one kernel arms an mbarrier for a transaction no
 * copy will deliver and runs the library's bounded wait (the one that guards
 * every TMA box of the interpolation) with a budget of `ms` milliseconds
 * (0 < ms <= 10000); the wait gives up, the kernel latches the timeout bit and
 * returns, and the call returns IB_ERR_TIMEOUT with the context intact.
 * Synchronises `stream`.  Error-path tests may also set the environment
 * variable IBFE_FAULT="entry[:code]", which makes that C entry point (for
 * example ib_forward) return `code` (default IB_ERR_CUDA) before any work. */
ib_status ib_diag_wait_timeout(double ms, void* stream);

/* Static string for a status code. */
const char* ib_status_str(ib_status s);

/* Library version as major*10000 + minor*100 + patch. */
int32_t ib_version(void);

#ifdef __cplusplus
}
#endif
#endif
