/*
 * FP64 CPU oracle for the immersed-boundary coupling step -- TEST
 * INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does.
 *
 * A plain, single-threaded, double-precision evaluation of the definitions of
 * arXiv 2503.22695 (Ma, Cai, Wang, Luo, Gao), written for readability:
 *   - spreading   f = E(X, F)     Section 2 Eq. (1); discrete form Section 4.4
 *   - interpolation U = I(X, u)   Section 2 Eq. (2); Section 4.4 (U^IB, then the
 *                                 L2 projection onto the FE space, lumped)
 *   - nodal force F_i = -sum_q P(X_q):grad phi_i(X_q) w_q     Section 4.4
 *   - stresses P = dPsi/dF for neo-Hookean (Section 6.3), the modified
 *     standard reinforcing model (Psi_1), fibre-reinforced models 1 and 2
 *     (Psi_2, Psi_3) and Holzapfel-Ogden (Psi_4) of Section 3, plus the
 *     active fibre stress of Section 6.1 (T_a given per material)
 *   - the 4-point regularised delta (Peskin, cited in Section 2)
 *   - adjoints (vector-Jacobian products) of the three operators.
 *
 * Conventions shared with the GPU path are fixed by the paper or stated here:
 *   grid     periodic box [origin, origin + n h), fields [3][n2][n1][n0];
 *            component c lives at the lower c-face: face (i0,i1,i2) of
 *            component c sits at origin_d + (i_d + s_cd) h, s_cd = 0 if d == c
 *            else 1/2 (the i+1/2 staggering of Section 4.3/4.4).
 *   mesh     trilinear hexahedra, VTK corner order, conn [8][E] (int32),
 *            reference coordinates X [3][N]; 2x2x2 Gauss rule at +-1/sqrt(3),
 *            Gauss point q = b0 + 2 b1 + 4 b2 with xi_d = (2 b_d - 1)/sqrt(3);
 *            or linear tetrahedra (elem 1), conn [4][E], with the symmetric
 *            4-point rule of degree 2 (point q nearest corner q); or
 *            quadratic tetrahedra (elem 2), conn [10][E] (VTK order: 4
 *            vertices, then edges 01, 12, 02, 03, 13, 23), the same rule.
 *   positions x [3][N] (double; tests rebuild them exactly from the split
 *            cell + offset storage).  Cells are not wrapped; the grid index
 *            is taken modulo n.
 *   materials params per model: NH {a, kappa}; FIBRE1 {C1, af, bf, kappa};
 *            HO {a, b, af, bf, as, bs, afs, bfs, kappa}; STD_REINF {G_T, G_L,
 *            E_L, kappa}; FIBRE2 {C10, C01, af, bf, kappa}; the active tension
 *            T_a in the row's last entry; mat_id [E] selects a row of the
 *            material table (stride 10 doubles).
 *   mass     lumped: m_a = sum_{e,q} N_a(xi_q) w_q j0 (row-sum of the
 *            consistent mass; equal to the nodal-rule weight of Section 4.4).
 *
 * Every function returns 0 on success and a negative value on bad input
 * (non-positive Jacobian, bad sizes).  Outputs are overwritten.
 */
#ifndef IBREF_H
#define IBREF_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t n[3];
  double h;
  double origin[3];
} or_grid;

typedef struct {
  int32_t n_nodes, n_elems;
  const int32_t* conn;   /* [8][E] hexahedra, [4][E] or [10][E] tetrahedra */
  const double* X;       /* [3][N] */
  const double* fibres;  /* [6][E] or NULL */
  const int32_t* mat_id; /* [E] or NULL */
  int32_t elem;          /* 0: trilinear hexahedron, 1: linear, 2: quadratic tetrahedron */
} or_mesh;

typedef struct {
  int32_t n_mats;
  const int32_t* model;  /* [n_mats] */
  const double* params;  /* [n_mats][10]: the law's parameters, then T_a at [9] */
} or_mats;

/* Active tension waveform T_a(t) of Section 6.1 in Pa (period 0.8 s). */
double or_active_tension(double t);

/* 1-D kernel phi(r) and dphi/dr, r in units of h. */
double or_phi(double r);
double or_dphi(double r);

/* Stress P (row-major 3x3, P[3*i+j]) and energy density Psi for one F;
 * params holds 10 doubles (the law's parameters, then T_a at [9]). */
int or_stress(int32_t model, const double* params, const double* F, const double* ef,
              const double* es, double* P, double* psi);
/* Directional derivative dP = (d P / d F)[dF]. */
int or_stress_dir(int32_t model, const double* params, const double* F, const double* dF,
                  const double* ef, const double* es, double* dP);

/* Per Gauss point: wj0 [8][E] (q-major: index q*E + e), J = det F [8][E]. */
int or_gauss_info(const or_mesh* m, const double* x, double* wj0, double* detF);

/* Lumped nodal mass m [N]. */
int or_lumped_mass(const or_mesh* m, double* mass);

/* Nodal forces G [3][N] (G = -dE/dx) and total elastic energy E. */
int or_fe_force(const or_mesh* m, const or_mats* mats, const double* x, double* G,
                double* energy);

/* Hv = (dG/dx) v  [3][N] and gparams[k] = v . dG/dtheta_k, [n_mats][10]
 * (the law's parameters, then T_a at [9]). */
int or_fe_force_adj(const or_mesh* m, const or_mats* mats, const double* x,
                    const double* v, double* Hv, double* gparams);

/* Spread nodal forces G [3][N] onto f [3][n2][n1][n0]. */
int or_spread(const or_grid* g, const or_mesh* m, const double* x, const double* G,
              double* f);

/* Spread evaluated at selected faces only: comp[k], idx[k] = (i0,i1,i2) -> out[k]
 * (a brute-force sum over every Gauss point, for sampled checks). */
int or_spread_at(const or_grid* g, const or_mesh* m, const double* x, const double* G,
                 int64_t n_sel, const int32_t* comp, const int32_t* idx, double* out);

/* Interpolate u [3][grid] to nodal velocities U [3][N]; optionally return the
 * Gauss-point values U^IB [3][8][E] (q-major). */
int or_interp(const or_grid* g, const or_mesh* m, const double* x, const double* u,
              double* U, double* Uq);

/* Adjoint of spreading: gG [3][N] and (optional) gx [3][N] from gf [3][grid]. */
int or_spread_adj(const or_grid* g, const or_mesh* m, const double* x, const double* G,
                  const double* gf, double* gG, double* gx);

/* Adjoint of interpolation: gu [3][grid] and (optional) gx [3][N] from gU [3][N]. */
int or_interp_adj(const or_grid* g, const or_mesh* m, const double* x, const double* u,
                  const double* gU, double* gu, double* gx);

/* Nodal quadrature rule of Section 4.4: the coupling points are the N nodes'
 * displaced positions x [3][N].  Spreading of the nodal forces G [3][N]
 * (f = h^-3 sum_a G_a prod phi), interpolation U_a = sum u prod phi (the
 * nodal rule makes the lumped projection the identity), a brute-force
 * spreading at selected faces, and the two adjoints (gx optional). */
int or_spread_nodal(const or_grid* g, int64_t N, const double* x, const double* G, double* f);
int or_spread_nodal_at(const or_grid* g, int64_t N, const double* x, const double* G,
                       int64_t n_sel, const int32_t* comp, const int32_t* idx, double* out);
int or_interp_nodal(const or_grid* g, int64_t N, const double* x, const double* u, double* U);
int or_spread_nodal_adj(const or_grid* g, int64_t N, const double* x, const double* G,
                        const double* gf, double* gG, double* gx);
int or_interp_nodal_adj(const or_grid* g, int64_t N, const double* x, const double* u,
                        const double* gU, double* gu, double* gx);

/* Number of distinct (component, face) pairs covered by the interpolation
 * stencils of all Gauss points (for the algorithmic-bytes count). */
int64_t or_support_count(const or_grid* g, const or_mesh* m, const double* x);

#ifdef __cplusplus
}
#endif
#endif
