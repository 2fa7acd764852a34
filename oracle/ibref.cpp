// FP64 CPU oracle for the immersed-boundary coupling step -- TEST
// INFRASTRUCTURE ONLY (loaded by the tests, the package smoke check and the
// benchmark's CPU-baseline leg; never by the product path).
//
// Plain, single-threaded double-precision evaluation of the definitions of
// arXiv 2503.22695; conventions are documented in ibref.h.  Each function
// cites the passage it follows.  No blocking, fusion or reordering beyond
// the definitions: one loop over elements, one over Gauss points, one over
// the 4x4x4 stencil.
#include "ibref.h"

#include <cmath>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Forward-mode dual numbers, used only to differentiate the stress function
// (directional derivatives for the Hessian-vector product, and derivatives
// with respect to material parameters).
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual(double v_ = 0.0, double d_ = 0.0) : v(v_), d(d_) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, e * a.d); }
inline Dual log(Dual a) { return Dual(std::log(a.v), a.d / a.v); }
inline Dual sqrt(Dual a) { double r = std::sqrt(a.v); return Dual(r, a.d / (2.0 * r)); }
inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }
using std::exp;
using std::log;
using std::sqrt;

// ---------------------------------------------------------------------------
// 4-point regularised delta kernel (Peskin 2002, cited in Section 2; the
// discrete delta_h(x) = h^-3 prod_d phi(x_d / h) of Section 4.4).
// ---------------------------------------------------------------------------
double phi(double r) {
  double a = std::fabs(r);
  if (a <= 1.0) return (3.0 - 2.0 * a + std::sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
  if (a <= 2.0) return (5.0 - 2.0 * a - std::sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
  return 0.0;
}

double dphi(double r) {
  double a = std::fabs(r), s = r < 0 ? -1.0 : 1.0, g;
  if (a <= 1.0)
    g = (-2.0 + (2.0 - 4.0 * a) / std::sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
  else if (a <= 2.0)
    g = (-2.0 - (6.0 - 4.0 * a) / std::sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
  else
    g = 0.0;
  return s * g;
}

// ---------------------------------------------------------------------------
// Constitutive laws (Section 3 and Section 6.3).  P = dPsi/dF written out as
// the exact derivative of each Psi:
//   dI1bar/dF = 2 J^-2/3 (F - I1/3 F^-T),  d ln J/dF = F^-T,
//   dI4i/dF = 2 F e_i (x) e_i,  dI8fs/dF = F (e_f (x) e_s + e_s (x) e_f).
// Readings of the printed formulas (see the design notes): the HO isotropic
// term carries F^-T (printed F^T), the HO shear term is the exact derivative
// a_fs I8 exp(b_fs I8^2) F (e_f(x)e_s + e_s(x)e_f), and Psi_4's isotropic part
// carries "-1" so that Psi(I) = 0.
// ---------------------------------------------------------------------------
// parameters per model: NH {a, kappa}; Psi_2 {C1, af, bf, kappa};
// Psi_4 {a, b, af, bf, as, bs, afs, bfs, kappa}; Psi_1 {G_T, G_L, E_L, kappa};
// Psi_3 {C10, C01, af, bf, kappa}.  A parameter row holds kRow doubles: the
// law's parameters first, the active tension T_a (Section 6.1) in the last.
constexpr int kRow = 10;
constexpr int kTa = 9;
int n_params_of(int model) {
  switch (model) {
    case 0: return 2;
    case 1: return 4;
    case 2: return 9;
    case 3: return 4;
    case 4: return 5;
  }
  return 0;
}

template <class T>
void stress_t(int model, const T* p, const T F[3][3], const double* ef, const double* es,
              T P[3][3], T& psi) {
  // cofactor matrix: cof_ij = d det F / d F_ij, so F^-T = cof / J
  T cof[3][3];
  cof[0][0] = F[1][1] * F[2][2] - F[1][2] * F[2][1];
  cof[0][1] = F[1][2] * F[2][0] - F[1][0] * F[2][2];
  cof[0][2] = F[1][0] * F[2][1] - F[1][1] * F[2][0];
  cof[1][0] = F[0][2] * F[2][1] - F[0][1] * F[2][2];
  cof[1][1] = F[0][0] * F[2][2] - F[0][2] * F[2][0];
  cof[1][2] = F[0][1] * F[2][0] - F[0][0] * F[2][1];
  cof[2][0] = F[0][1] * F[1][2] - F[0][2] * F[1][1];
  cof[2][1] = F[0][2] * F[1][0] - F[0][0] * F[1][2];
  cof[2][2] = F[0][0] * F[1][1] - F[0][1] * F[1][0];
  T J = F[0][0] * cof[0][0] + F[0][1] * cof[0][1] + F[0][2] * cof[0][2];
  T FiT[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) FiT[i][j] = cof[i][j] / J;
  T I1 = T(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) I1 = I1 + F[i][j] * F[i][j];
  T lnJ = log(J);
  T Jm23 = exp(T(-2.0 / 3.0) * lnJ);
  T I1bar = Jm23 * I1;
  T dev[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) dev[i][j] = Jm23 * (F[i][j] - I1 / T(3.0) * FiT[i][j]);

  int np = n_params_of(model);
  T kappa = p[np - 1];
  // volumetric stabilisation U(J) = kappa/2 (ln J)^2 (Section 3)
  psi = kappa / T(2.0) * lnJ * lnJ;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) P[i][j] = kappa * lnJ * FiT[i][j];

  auto add_iso = [&](T coef) {  // P += coef * dev
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) P[i][j] = P[i][j] + coef * dev[i][j];
  };
  // fibre term a_i/(2 b_i) (exp[b_i (I4i* - 1)^2] - 1), I4i* = max(I4i, 1);
  // with clamp false the plain I4i - 1 (Psi_3)
  auto add_fibre = [&](const double* e, T ai, T bi, bool clamp = true) {
    T Fe[3];
    for (int i = 0; i < 3; ++i) Fe[i] = F[i][0] * e[0] + F[i][1] * e[1] + F[i][2] * e[2];
    T I4 = Fe[0] * Fe[0] + Fe[1] * Fe[1] + Fe[2] * Fe[2];
    T d = (!clamp || val(I4) > 1.0) ? I4 - T(1.0) : T(0.0);
    T ex = exp(bi * d * d);
    psi = psi + ai / (T(2.0) * bi) * (ex - T(1.0));
    T coef = T(2.0) * ai * d * ex;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) P[i][j] = P[i][j] + coef * Fe[i] * T(e[j]);
  };

  if (model == 0) {  // neo-Hookean, Section 6.3: a (I1bar - 3)
    psi = psi + p[0] * (I1bar - T(3.0));
    add_iso(T(2.0) * p[0]);
  } else if (model == 1) {  // Psi_2: C1 (I1bar - 3) + fibre(e_f)
    psi = psi + p[0] * (I1bar - T(3.0));
    add_iso(T(2.0) * p[0]);
    add_fibre(ef, p[1], p[2]);
  } else if (model == 3) {
    // Psi_1 modified standard reinforcing: G_T/2 (I1bar - 3)
    //   + (G_T - G_L)/2 (2 I4f - I5f - 1) + (E_L + G_T - 4 G_L)/8 (I4f - 1)^2,
    // dI5f/dF = 2 (F e (x) C e + F C e (x) e)
    T GT = p[0], GL = p[1], EL = p[2];
    psi = psi + GT / T(2.0) * (I1bar - T(3.0));
    add_iso(GT);
    T Fe[3], Ce[3], FCe[3];
    for (int i = 0; i < 3; ++i) Fe[i] = F[i][0] * ef[0] + F[i][1] * ef[1] + F[i][2] * ef[2];
    for (int j = 0; j < 3; ++j) Ce[j] = F[0][j] * Fe[0] + F[1][j] * Fe[1] + F[2][j] * Fe[2];
    for (int i = 0; i < 3; ++i) FCe[i] = F[i][0] * Ce[0] + F[i][1] * Ce[1] + F[i][2] * Ce[2];
    T I4 = Fe[0] * Fe[0] + Fe[1] * Fe[1] + Fe[2] * Fe[2];
    T I5 = Ce[0] * Ce[0] + Ce[1] * Ce[1] + Ce[2] * Ce[2];
    T k4 = (EL + GT - T(4.0) * GL);
    psi = psi + (GT - GL) / T(2.0) * (T(2.0) * I4 - I5 - T(1.0)) +
          k4 / T(8.0) * (I4 - T(1.0)) * (I4 - T(1.0));
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        P[i][j] = P[i][j] +
                  (GT - GL) * (T(2.0) * Fe[i] * T(ef[j]) - Fe[i] * Ce[j] - FCe[i] * T(ef[j])) +
                  k4 / T(2.0) * (I4 - T(1.0)) * Fe[i] * T(ef[j]);
  } else if (model == 4) {
    // Psi_3 fibre-reinforced model 2: C10 (exp[C01 (I1bar - 3)] - 1) + fibre
    // term without the tension-only clamp
    T ex = exp(p[1] * (I1bar - T(3.0)));
    psi = psi + p[0] * (ex - T(1.0));
    add_iso(T(2.0) * p[0] * p[1] * ex);
    add_fibre(ef, p[2], p[3], false);
  } else {  // Psi_4 Holzapfel-Ogden
    T ex = exp(p[1] * (I1bar - T(3.0)));
    psi = psi + p[0] / (T(2.0) * p[1]) * (ex - T(1.0));
    add_iso(p[0] * ex);
    add_fibre(ef, p[2], p[3]);
    add_fibre(es, p[4], p[5]);
    T Fef[3], Fes[3];
    for (int i = 0; i < 3; ++i) {
      Fef[i] = F[i][0] * ef[0] + F[i][1] * ef[1] + F[i][2] * ef[2];
      Fes[i] = F[i][0] * es[0] + F[i][1] * es[1] + F[i][2] * es[2];
    }
    T I8 = Fef[0] * Fes[0] + Fef[1] * Fes[1] + Fef[2] * Fes[2];
    T ex8 = exp(p[7] * I8 * I8);
    psi = psi + p[6] / (T(2.0) * p[7]) * (ex8 - T(1.0));
    T coef = p[6] * I8 * ex8;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        P[i][j] = P[i][j] + coef * (Fef[i] * T(es[j]) + Fes[i] * T(ef[j]));
  }

  // Active stress, Section 6.1: P^a = F S_a with S_a = T(t, I4f) e_f (x) e_f,
  // T = T_a (1 + 4.9 (sqrt(I4f) - 1)); T_a = p[kTa] is the value of the
  // waveform at the current time.  T depends on F only through I4f, so P^a
  // = 2 dW_a/dI4f F e_f (x) e_f is the derivative of the potential
  //   W_a = T_a/2 [(1 - 4.9)(I4f - 1) + 4.9 (2/3)(I4f^(3/2) - 1)],
  // which is added to the energy.  No tension-only clamp; T_a = 0 adds zeros.
  {
    T Ta = p[kTa];
    T Fe[3];
    for (int i = 0; i < 3; ++i) Fe[i] = F[i][0] * ef[0] + F[i][1] * ef[1] + F[i][2] * ef[2];
    T I4 = Fe[0] * Fe[0] + Fe[1] * Fe[1] + Fe[2] * Fe[2];
    T s = sqrt(I4);
    T tension = Ta * (T(1.0) + T(4.9) * (s - T(1.0)));
    psi = psi + Ta / T(2.0) *
                    (T(1.0 - 4.9) * (I4 - T(1.0)) + T(4.9 * 2.0 / 3.0) * (I4 * s - T(1.0)));
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) P[i][j] = P[i][j] + tension * Fe[i] * T(ef[j]);
  }
}


const double kUnitX[3] = {1.0, 0.0, 0.0};
const double kUnitY[3] = {0.0, 1.0, 0.0};

// ---------------------------------------------------------------------------
// Elements and their rules (the element rule H_q of Section 4.4):
//   elem 0: trilinear hexahedron, VTK corner order, 2x2x2 Gauss rule at
//           +-1/sqrt(3) with unit weights;
//   elem 1: linear tetrahedron (P1; VTK order, positive volume), N_0 =
//           1 - xi - eta - zeta, N_1 = xi, N_2 = eta, N_3 = zeta on the unit
//           reference tetrahedron, with the symmetric 4-point rule of degree 2:
//           barycentric coordinates (a, b, b, b) and permutations,
//           a = (5 + 3 sqrt 5)/20, b = (5 - sqrt 5)/20, weights 1/24 each
//           (the reference volume 1/6 in four).  The force integrand of P1 is
//           constant per element, so this rule gives it exactly too.
//   elem 2: quadratic tetrahedron (P2, the element of the Cook membrane of
//           Section 5), VTK order: vertices 0-3 as in P1, then the mid-edge
//           nodes of edges (0,1), (1,2), (0,2), (0,3), (1,3), (2,3).  With the
//           barycentric coordinates L_0..L_3 above, N = L_i (2 L_i - 1) at a
//           vertex and N = 4 L_i L_j at the node of edge (i, j).  The same
//           4-point rule of degree 2 serves the force (its integrand
//           P : grad N is of degree 2 on an affine element under an affine
//           deformation, so the patch test holds) and the coupling.
// ---------------------------------------------------------------------------
constexpr int kMaxC = 10;  // nodes of the largest element
const int kCorner[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                           {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
// P2 edge nodes: the two vertices of each edge, VTK order
const int kTetEdge[6][2] = {{0, 1}, {1, 2}, {0, 2}, {0, 3}, {1, 3}, {2, 3}};

int nc_of(const or_mesh* m) { return m->elem == 2 ? 10 : (m->elem == 1 ? 4 : 8); }  // nodes
int nq_of(const or_mesh* m) { return m->elem == 0 ? 8 : 4; }  // rule points

struct GaussPt {
  double N[kMaxC];
  double dNdX[kMaxC][3];
  double wj0;
};

bool gauss_point(const or_mesh* m, const double Xe[kMaxC][3], int q, GaussPt& g) {
  const int nc = nc_of(m);
  double dNdxi[kMaxC][3] = {{0}};
  double wq = 1.0;
  for (int a = 0; a < kMaxC; ++a) g.N[a] = 0.0;
  if (m->elem == 1 || m->elem == 2) {
    const double ta = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, tb = (5.0 - std::sqrt(5.0)) / 20.0;
    // barycentric coordinates of rule point q and their xi-gradients
    double L[4], dL[4][3] = {{-1.0, -1.0, -1.0}, {1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};
    for (int i = 0; i < 4; ++i) L[i] = i == q ? ta : tb;
    if (m->elem == 1) {
      for (int a = 0; a < 4; ++a) {
        g.N[a] = L[a];
        for (int d = 0; d < 3; ++d) dNdxi[a][d] = dL[a][d];
      }
    } else {
      for (int a = 0; a < 4; ++a) {
        g.N[a] = L[a] * (2.0 * L[a] - 1.0);
        for (int d = 0; d < 3; ++d) dNdxi[a][d] = (4.0 * L[a] - 1.0) * dL[a][d];
      }
      for (int k = 0; k < 6; ++k) {
        const int i = kTetEdge[k][0], j = kTetEdge[k][1];
        g.N[4 + k] = 4.0 * L[i] * L[j];
        for (int d = 0; d < 3; ++d) dNdxi[4 + k][d] = 4.0 * (L[i] * dL[j][d] + L[j] * dL[i][d]);
      }
    }
    wq = 1.0 / 24.0;
  } else {
    double xi[3];
    for (int d = 0; d < 3; ++d) xi[d] = (((q >> d) & 1) ? 1.0 : -1.0) / std::sqrt(3.0);
    for (int a = 0; a < 8; ++a) {
      double f[3];
      for (int d = 0; d < 3; ++d) f[d] = 1.0 + kCorner[a][d] * xi[d];
      g.N[a] = f[0] * f[1] * f[2] / 8.0;
      dNdxi[a][0] = kCorner[a][0] * f[1] * f[2] / 8.0;
      dNdxi[a][1] = kCorner[a][1] * f[0] * f[2] / 8.0;
      dNdxi[a][2] = kCorner[a][2] * f[0] * f[1] / 8.0;
    }
  }
  double J0[3][3] = {{0}};
  for (int a = 0; a < nc; ++a)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) J0[i][j] += Xe[a][i] * dNdxi[a][j];
  double det = J0[0][0] * (J0[1][1] * J0[2][2] - J0[1][2] * J0[2][1]) -
               J0[0][1] * (J0[1][0] * J0[2][2] - J0[1][2] * J0[2][0]) +
               J0[0][2] * (J0[1][0] * J0[2][1] - J0[1][1] * J0[2][0]);
  if (!(det > 0.0)) return false;
  double inv[3][3];
  inv[0][0] = (J0[1][1] * J0[2][2] - J0[1][2] * J0[2][1]) / det;
  inv[0][1] = (J0[0][2] * J0[2][1] - J0[0][1] * J0[2][2]) / det;
  inv[0][2] = (J0[0][1] * J0[1][2] - J0[0][2] * J0[1][1]) / det;
  inv[1][0] = (J0[1][2] * J0[2][0] - J0[1][0] * J0[2][2]) / det;
  inv[1][1] = (J0[0][0] * J0[2][2] - J0[0][2] * J0[2][0]) / det;
  inv[1][2] = (J0[0][2] * J0[1][0] - J0[0][0] * J0[1][2]) / det;
  inv[2][0] = (J0[1][0] * J0[2][1] - J0[1][1] * J0[2][0]) / det;
  inv[2][1] = (J0[0][1] * J0[2][0] - J0[0][0] * J0[2][1]) / det;
  inv[2][2] = (J0[0][0] * J0[1][1] - J0[0][1] * J0[1][0]) / det;
  // dN/dX_i = sum_j dN/dxi_j (dxi_j/dX_i), dxi/dX = J0^-1
  for (int a = 0; a < kMaxC; ++a)
    for (int i = 0; i < 3; ++i) {
      double s = 0.0;
      for (int j = 0; j < 3; ++j) s += dNdxi[a][j] * inv[j][i];
      g.dNdX[a][i] = s;
    }
  g.wj0 = wq * det;
  return true;
}

// Gather an element's corners of a [3][N] array (zeros past the last corner).
void gather(const or_mesh* m, const double* A, int e, double out[kMaxC][3]) {
  int64_t E = m->n_elems, N = m->n_nodes;
  for (int a = 0; a < kMaxC; ++a) {
    if (a >= nc_of(m)) {
      for (int i = 0; i < 3; ++i) out[a][i] = 0.0;
      continue;
    }
    int64_t node = m->conn[(int64_t)a * E + e];
    for (int i = 0; i < 3; ++i) out[a][i] = A[(int64_t)i * N + node];
  }
}

bool check_mesh(const or_mesh* m) {
  if (!m || m->n_nodes <= 0 || m->n_elems < 0 || !m->conn || !m->X) return false;
  if (m->elem != 0 && m->elem != 1 && m->elem != 2) return false;
  for (int64_t k = 0; k < (int64_t)nc_of(m) * m->n_elems; ++k)
    if (m->conn[k] < 0 || m->conn[k] >= m->n_nodes) return false;
  return true;
}

void fibres_of(const or_mesh* m, int e, double ef[3], double es[3]) {
  for (int i = 0; i < 3; ++i) {
    ef[i] = m->fibres ? m->fibres[(int64_t)i * m->n_elems + e] : kUnitX[i];
    es[i] = m->fibres ? m->fibres[(int64_t)(3 + i) * m->n_elems + e] : kUnitY[i];
  }
}

int mat_of(const or_mesh* m, int e) { return m->mat_id ? m->mat_id[e] : 0; }

// ---------------------------------------------------------------------------
// Grid helpers: the staggering s_cd and the periodic stencil of a point.
// ---------------------------------------------------------------------------
int64_t wrap(int64_t i, int64_t n) {
  int64_t r = i % n;
  return r < 0 ? r + n : r;
}

struct Stencil {
  int64_t idx[3][4];  // wrapped face indices per dimension
  double w[3][4];     // phi(r) per dimension
  double dw[3][4];    // dphi/dr per dimension
};

// Stencil of component c for a point at chi: along dimension d the faces sit
// at origin_d + (i + s_cd) h; t = (chi_d - origin_d)/h - s_cd, faces
// floor(t)-1 .. floor(t)+2 cover every |r| < 2, r = t - i.
void stencil(const or_grid* g, int c, const double chi[3], Stencil& s) {
  for (int d = 0; d < 3; ++d) {
    double sh = (d == c) ? 0.0 : 0.5;
    double t = (chi[d] - g->origin[d]) / g->h - sh;
    int64_t base = (int64_t)std::floor(t);
    for (int j = 0; j < 4; ++j) {
      int64_t i = base - 1 + j;
      double r = t - (double)i;
      s.idx[d][j] = wrap(i, g->n[d]);
      s.w[d][j] = phi(r);
      s.dw[d][j] = dphi(r);
    }
  }
}

int64_t face_index(const or_grid* g, int c, int64_t i0, int64_t i1, int64_t i2) {
  return (((int64_t)c * g->n[2] + i2) * g->n[1] + i1) * g->n[0] + i0;
}

bool check_grid(const or_grid* g) {
  return g && g->h > 0.0 && g->n[0] > 0 && g->n[1] > 0 && g->n[2] > 0;
}

// Per Gauss point data shared by spread and interp: chi_q = sum_a N_a x_a.
void point_of(const GaussPt& gp, const double xe[kMaxC][3], double chi[3]) {
  for (int i = 0; i < 3; ++i) {
    chi[i] = 0.0;
    for (int a = 0; a < kMaxC; ++a) chi[i] += gp.N[a] * xe[a][i];
  }
}

}  // namespace

extern "C" {

// Active tension waveform T_a(t) of Section 6.1, in Pa: zero before 0.5 s, a
// Gaussian-shaped rise 84260 (1 - exp(-(t - 0.5)^2 / 0.005)) to 0.65 s, the
// mirrored fall 84260 (1 - exp(-(0.8 - t)^2 / 0.005)) to 0.8 s; repeated with
// the 0.8 s period of the cardiac cycle.
double or_active_tension(double t) {
  const double period = 0.8, peak = 84260.0, width = 0.005;
  double tc = std::fmod(t, period);
  if (tc < 0.0) tc += period;
  if (tc < 0.5) return 0.0;
  const double r = tc < 0.65 ? tc - 0.5 : period - tc;
  return peak * (1.0 - std::exp(-r * r / width));
}

double or_phi(double r) { return phi(r); }
double or_dphi(double r) { return dphi(r); }

int or_stress(int32_t model, const double* params, const double* F, const double* ef,
              const double* es, double* P, double* psi) {
  if (n_params_of(model) == 0) return -1;
  double Fm[3][3], Pm[3][3], ps;
  for (int i = 0; i < 9; ++i) Fm[i / 3][i % 3] = F[i];
  stress_t<double>(model, params, Fm, ef ? ef : kUnitX, es ? es : kUnitY, Pm, ps);
  for (int i = 0; i < 9; ++i) P[i] = Pm[i / 3][i % 3];
  if (psi) *psi = ps;
  return 0;
}

int or_stress_dir(int32_t model, const double* params, const double* F, const double* dF,
                  const double* ef, const double* es, double* dP) {
  if (n_params_of(model) == 0) return -1;
  Dual Fm[3][3], Pm[3][3], ps, pp[kRow];
  for (int k = 0; k < kRow; ++k) pp[k] = Dual(params[k], 0.0);
  for (int i = 0; i < 9; ++i) Fm[i / 3][i % 3] = Dual(F[i], dF[i]);
  stress_t<Dual>(model, pp, Fm, ef ? ef : kUnitX, es ? es : kUnitY, Pm, ps);
  for (int i = 0; i < 9; ++i) dP[i] = Pm[i / 3][i % 3].d;
  return 0;
}

int or_gauss_info(const or_mesh* m, const double* x, double* wj0, double* detF) {
  if (!check_mesh(m)) return -1;
  int64_t E = m->n_elems;
  for (int e = 0; e < E; ++e) {
    double Xe[kMaxC][3], xe[kMaxC][3];
    gather(m, m->X, e, Xe);
    gather(m, x, e, xe);
    for (int q = 0; q < nq_of(m); ++q) {
      GaussPt gp;
      if (!gauss_point(m, Xe, q, gp)) return -2;
      wj0[q * E + e] = gp.wj0;
      double F[3][3] = {{0}};
      for (int a = 0; a < nc_of(m); ++a)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) F[i][j] += xe[a][i] * gp.dNdX[a][j];
      detF[q * E + e] = F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) -
                        F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
                        F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
    }
  }
  return 0;
}

// Lumped mass.  Hexahedra and P1: row sums of the consistent mass matrix
// int phi_a phi_b dX by the element Gauss rule; equals the nodal quadrature
// weight w_q = int phi_q of Section 4.4.  P2: the row sums of a vertex are
// negative (int N_vertex dX = -V/20), so the element's diagonal is scaled
// instead (Hinton, Rock and Zienkiewicz 1976): m_a = d_a V / sum_b d_b with
// d_a = sum_q w_q j0 N_a(xi_q)^2 and V = sum_q w_q j0, by the same rule;
// every m_a > 0 and the element's masses sum to its volume.
int or_lumped_mass(const or_mesh* m, double* mass) {
  if (!check_mesh(m)) return -1;
  std::memset(mass, 0, sizeof(double) * m->n_nodes);
  int64_t E = m->n_elems;
  for (int e = 0; e < E; ++e) {
    double Xe[kMaxC][3];
    gather(m, m->X, e, Xe);
    double d[kMaxC] = {0}, V = 0.0;
    for (int q = 0; q < nq_of(m); ++q) {
      GaussPt gp;
      if (!gauss_point(m, Xe, q, gp)) return -2;
      V += gp.wj0;
      for (int a = 0; a < nc_of(m); ++a)
        d[a] += m->elem == 2 ? gp.N[a] * gp.N[a] * gp.wj0 : gp.N[a] * gp.wj0;
    }
    if (m->elem == 2) {
      double D = 0.0;
      for (int a = 0; a < nc_of(m); ++a) D += d[a];
      for (int a = 0; a < nc_of(m); ++a) d[a] *= V / D;
    }
    for (int a = 0; a < nc_of(m); ++a) mass[m->conn[a * E + e]] += d[a];
  }
  return 0;
}

// Nodal force of Section 4.4: F_i = -sum_{q in H_q} P(X_q) : grad_X phi_i(X_q) w_q,
// i.e. G_a = -sum_{e,q} P(F_q) grad_X N_a w_q j0 with F = sum_a x_a (x) grad_X N_a
// (Section 2 deformation gradient), and E = sum_{e,q} Psi(F_q) w_q j0.
int or_fe_force(const or_mesh* m, const or_mats* mats, const double* x, double* G,
                double* energy) {
  if (!check_mesh(m) || !mats || mats->n_mats <= 0) return -1;
  int64_t E = m->n_elems, N = m->n_nodes;
  std::memset(G, 0, sizeof(double) * 3 * N);
  double en = 0.0;
  for (int e = 0; e < E; ++e) {
    int mid = mat_of(m, e);
    if (mid < 0 || mid >= mats->n_mats) return -1;
    const double* p = mats->params + kRow * mid;
    int model = mats->model[mid];
    double Xe[kMaxC][3], xe[kMaxC][3], ef[3], es[3];
    gather(m, m->X, e, Xe);
    gather(m, x, e, xe);
    fibres_of(m, e, ef, es);
    for (int q = 0; q < nq_of(m); ++q) {
      GaussPt gp;
      if (!gauss_point(m, Xe, q, gp)) return -2;
      double F[3][3] = {{0}}, P[3][3], psi;
      for (int a = 0; a < nc_of(m); ++a)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) F[i][j] += xe[a][i] * gp.dNdX[a][j];
      stress_t<double>(model, p, F, ef, es, P, psi);
      en += psi * gp.wj0;
      for (int a = 0; a < nc_of(m); ++a) {
        int64_t node = m->conn[a * E + e];
        for (int i = 0; i < 3; ++i) {
          double s = 0.0;
          for (int j = 0; j < 3; ++j) s += P[i][j] * gp.dNdX[a][j];
          G[i * N + node] -= s * gp.wj0;
        }
      }
    }
  }
  if (energy) *energy = en;
  return 0;
}

// Hv = (dG/dx) v: with dF = sum_b v_b (x) grad_X N_b, Hv_a = -sum_q dP[dF] grad_X N_a w_q j0.
// gparams[k] = v . dG/dtheta_k = -sum_q (dP/dtheta_k) : dF w_q j0.
int or_fe_force_adj(const or_mesh* m, const or_mats* mats, const double* x,
                    const double* v, double* Hv, double* gparams) {
  if (!check_mesh(m) || !mats || mats->n_mats <= 0) return -1;
  int64_t E = m->n_elems, N = m->n_nodes;
  std::memset(Hv, 0, sizeof(double) * 3 * N);
  if (gparams) std::memset(gparams, 0, sizeof(double) * kRow * mats->n_mats);
  for (int e = 0; e < E; ++e) {
    int mid = mat_of(m, e);
    if (mid < 0 || mid >= mats->n_mats) return -1;
    const double* p = mats->params + kRow * mid;
    int model = mats->model[mid];
    int np = n_params_of(model);
    double Xe[kMaxC][3], xe[kMaxC][3], ve[kMaxC][3], ef[3], es[3];
    gather(m, m->X, e, Xe);
    gather(m, x, e, xe);
    gather(m, v, e, ve);
    fibres_of(m, e, ef, es);
    for (int q = 0; q < nq_of(m); ++q) {
      GaussPt gp;
      if (!gauss_point(m, Xe, q, gp)) return -2;
      double F[3][3] = {{0}}, dF[3][3] = {{0}};
      for (int a = 0; a < nc_of(m); ++a)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            F[i][j] += xe[a][i] * gp.dNdX[a][j];
            dF[i][j] += ve[a][i] * gp.dNdX[a][j];
          }
      // directional derivative of P along dF
      Dual Fd[3][3], Pd[3][3], psid, pd[kRow];
      for (int k = 0; k < kRow; ++k) pd[k] = Dual(p[k], 0.0);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Fd[i][j] = Dual(F[i][j], dF[i][j]);
      stress_t<Dual>(model, pd, Fd, ef, es, Pd, psid);
      for (int a = 0; a < nc_of(m); ++a) {
        int64_t node = m->conn[a * E + e];
        for (int i = 0; i < 3; ++i) {
          double s = 0.0;
          for (int j = 0; j < 3; ++j) s += Pd[i][j].d * gp.dNdX[a][j];
          Hv[i * N + node] -= s * gp.wj0;
        }
      }
      if (gparams) {
        for (int k = 0; k < kRow; ++k) {
          if (k >= np && k != kTa) continue;  // the law's parameters and T_a
          for (int kk = 0; kk < kRow; ++kk) pd[kk] = Dual(p[kk], kk == k ? 1.0 : 0.0);
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Fd[i][j] = Dual(F[i][j], 0.0);
          stress_t<Dual>(model, pd, Fd, ef, es, Pd, psid);
          double s = 0.0;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) s += Pd[i][j].d * dF[i][j];
          gparams[kRow * mid + k] -= s * gp.wj0;
        }
      }
    }
  }
  return 0;
}

// Spreading, Section 4.4: f^c(face) = int F^c(X) delta_h(x_face - chi(X)) dX,
// with the integral taken by the element Gauss rule and F_h the lumped L2
// projection of the nodal forces: F_q = sum_a N_a(xi_q) G_a / m_a, so each
// Gauss point carries P_q = F_q w_q j0.
int or_spread(const or_grid* g, const or_mesh* m, const double* x, const double* G,
              double* f) {
  if (!check_grid(g) || !check_mesh(m)) return -1;
  int64_t E = m->n_elems, N = m->n_nodes;
  int64_t cells = (int64_t)g->n[0] * g->n[1] * g->n[2];
  std::memset(f, 0, sizeof(double) * 3 * cells);
  std::vector<double> mass(N);
  int rc = or_lumped_mass(m, mass.data());
  if (rc) return rc;
  std::vector<double> Fn(3 * N);
  for (int i = 0; i < 3; ++i)
    for (int64_t a = 0; a < N; ++a) Fn[i * N + a] = G[i * N + a] / mass[a];
  double h3 = g->h * g->h * g->h;
  for (int e = 0; e < E; ++e) {
    double Xe[kMaxC][3], xe[kMaxC][3], Fe[kMaxC][3];
    gather(m, m->X, e, Xe);
    gather(m, x, e, xe);
    gather(m, Fn.data(), e, Fe);
    for (int q = 0; q < nq_of(m); ++q) {
      GaussPt gp;
      if (!gauss_point(m, Xe, q, gp)) return -2;
      double chi[3], Pq[3];
      point_of(gp, xe, chi);
      for (int i = 0; i < 3; ++i) {
        Pq[i] = 0.0;
        for (int a = 0; a < nc_of(m); ++a) Pq[i] += gp.N[a] * Fe[a][i];
        Pq[i] *= gp.wj0;
      }
      for (int c = 0; c < 3; ++c) {
        Stencil s;
        stencil(g, c, chi, s);
        for (int kz = 0; kz < 4; ++kz)
          for (int ky = 0; ky < 4; ++ky)
            for (int kx = 0; kx < 4; ++kx)
              f[face_index(g, c, s.idx[0][kx], s.idx[1][ky], s.idx[2][kz])] +=
                  Pq[c] * s.w[0][kx] * s.w[1][ky] * s.w[2][kz] / h3;
      }
    }
  }
  return 0;
}

// Brute-force spreading at selected faces: every Gauss point, the nearest
// periodic image of each distance, phi evaluated directly (no stencil).
int or_spread_at(const or_grid* g, const or_mesh* m, const double* x, const double* G,
                 int64_t n_sel, const int32_t* comp, const int32_t* idx, double* out) {
  if (!check_grid(g) || !check_mesh(m)) return -1;
  int64_t E = m->n_elems, N = m->n_nodes, Q = (int64_t)nq_of(m) * E;
  std::vector<double> mass(N);
  int rc = or_lumped_mass(m, mass.data());
  if (rc) return rc;
  std::vector<double> chi(3 * Q), Pq(3 * Q);
  for (int e = 0; e < E; ++e) {
    double Xe[kMaxC][3], xe[kMaxC][3], Ge[kMaxC][3];
    gather(m, m->X, e, Xe);
    gather(m, x, e, xe);
    gather(m, G, e, Ge);
    for (int q = 0; q < nq_of(m); ++q) {
      GaussPt gp;
      if (!gauss_point(m, Xe, q, gp)) return -2;
      double c3[3];
      point_of(gp, xe, c3);
      for (int i = 0; i < 3; ++i) {
        chi[3 * (q * E + e) + i] = c3[i];
        double s = 0.0;
        for (int a = 0; a < nc_of(m); ++a) s += gp.N[a] * Ge[a][i] / mass[m->conn[a * E + e]];
        Pq[3 * (q * E + e) + i] = s * gp.wj0;
      }
    }
  }
  double h3 = g->h * g->h * g->h;
  for (int64_t k = 0; k < n_sel; ++k) {
    int c = comp[k];
    double acc = 0.0;
    for (int64_t p = 0; p < Q; ++p) {
      double w = 1.0;
      for (int d = 0; d < 3 && w != 0.0; ++d) {
        double sh = (d == c) ? 0.0 : 0.5;
        double r = (chi[3 * p + d] - g->origin[d]) / g->h - sh - idx[3 * k + d];
        r -= g->n[d] * std::floor(r / g->n[d] + 0.5);  // nearest periodic image
        w *= phi(r);
      }
      acc += Pq[3 * p + c] * w / h3;
    }
    out[k] = acc;
  }
  return 0;
}

// Interpolation, Section 4.4: U^IB_q = sum_faces u^c delta_h(x_face - chi_q) dx^3,
// then U_h is the L2 projection of U^IB onto the FE space with the lumped
// mass: U_a = m_a^-1 sum_{(e,q) containing a} N_a(xi_q) w_q j0 U^IB_q.
int or_interp(const or_grid* g, const or_mesh* m, const double* x, const double* u,
              double* U, double* Uq) {
  if (!check_grid(g) || !check_mesh(m)) return -1;
  int64_t E = m->n_elems, N = m->n_nodes;
  std::vector<double> mass(N);
  int rc = or_lumped_mass(m, mass.data());
  if (rc) return rc;
  std::memset(U, 0, sizeof(double) * 3 * N);
  for (int e = 0; e < E; ++e) {
    double Xe[kMaxC][3], xe[kMaxC][3];
    gather(m, m->X, e, Xe);
    gather(m, x, e, xe);
    for (int q = 0; q < nq_of(m); ++q) {
      GaussPt gp;
      if (!gauss_point(m, Xe, q, gp)) return -2;
      double chi[3], UIB[3];
      point_of(gp, xe, chi);
      for (int c = 0; c < 3; ++c) {
        Stencil s;
        stencil(g, c, chi, s);
        double acc = 0.0;
        for (int kz = 0; kz < 4; ++kz)
          for (int ky = 0; ky < 4; ++ky)
            for (int kx = 0; kx < 4; ++kx)
              acc += u[face_index(g, c, s.idx[0][kx], s.idx[1][ky], s.idx[2][kz])] *
                     s.w[0][kx] * s.w[1][ky] * s.w[2][kz];
        UIB[c] = acc;
        if (Uq) Uq[(int64_t)c * nq_of(m) * E + q * E + e] = acc;
      }
      for (int a = 0; a < nc_of(m); ++a) {
        int64_t node = m->conn[a * E + e];
        for (int c = 0; c < 3; ++c) U[c * N + node] += gp.N[a] * gp.wj0 * UIB[c];
      }
    }
  }
  for (int c = 0; c < 3; ++c)
    for (int64_t a = 0; a < N; ++a) U[c * N + a] /= mass[a];
  return 0;
}

// Adjoint of spreading.  With P_q = w_q j0 sum_a N_a G_a/m_a and
// f = h^-3 sum_q P_q prod_d phi(r_d):
//   gG_a = m_a^-1 sum_q N_a w_q j0 gP_q,  gP_q^c = h^-3 sum_faces gf^c prod phi,
//   gx_a = sum_q N_a gchi_q,  gchi_q,d = sum_c P_q^c h^-4 sum_faces gf^c phi'(r_d) prod_{d'!=d} phi.
int or_spread_adj(const or_grid* g, const or_mesh* m, const double* x, const double* G,
                  const double* gf, double* gG, double* gx) {
  if (!check_grid(g) || !check_mesh(m)) return -1;
  int64_t E = m->n_elems, N = m->n_nodes;
  std::vector<double> mass(N);
  int rc = or_lumped_mass(m, mass.data());
  if (rc) return rc;
  std::memset(gG, 0, sizeof(double) * 3 * N);
  if (gx) std::memset(gx, 0, sizeof(double) * 3 * N);
  double h = g->h, h3 = h * h * h;
  for (int e = 0; e < E; ++e) {
    double Xe[kMaxC][3], xe[kMaxC][3], Ge[kMaxC][3];
    gather(m, m->X, e, Xe);
    gather(m, x, e, xe);
    gather(m, G, e, Ge);
    for (int q = 0; q < nq_of(m); ++q) {
      GaussPt gp;
      if (!gauss_point(m, Xe, q, gp)) return -2;
      double chi[3], Pq[3], gP[3], gchi[3] = {0, 0, 0};
      point_of(gp, xe, chi);
      for (int i = 0; i < 3; ++i) {
        Pq[i] = 0.0;
        for (int a = 0; a < nc_of(m); ++a) Pq[i] += gp.N[a] * Ge[a][i] / mass[m->conn[a * E + e]];
        Pq[i] *= gp.wj0;
      }
      for (int c = 0; c < 3; ++c) {
        Stencil s;
        stencil(g, c, chi, s);
        double acc = 0.0, d0 = 0.0, d1 = 0.0, d2 = 0.0;
        for (int kz = 0; kz < 4; ++kz)
          for (int ky = 0; ky < 4; ++ky)
            for (int kx = 0; kx < 4; ++kx) {
              double v = gf[face_index(g, c, s.idx[0][kx], s.idx[1][ky], s.idx[2][kz])];
              acc += v * s.w[0][kx] * s.w[1][ky] * s.w[2][kz];
              d0 += v * s.dw[0][kx] * s.w[1][ky] * s.w[2][kz];
              d1 += v * s.w[0][kx] * s.dw[1][ky] * s.w[2][kz];
              d2 += v * s.w[0][kx] * s.w[1][ky] * s.dw[2][kz];
            }
        gP[c] = acc / h3;
        gchi[0] += Pq[c] * d0 / (h3 * h);
        gchi[1] += Pq[c] * d1 / (h3 * h);
        gchi[2] += Pq[c] * d2 / (h3 * h);
      }
      for (int a = 0; a < nc_of(m); ++a) {
        int64_t node = m->conn[a * E + e];
        for (int c = 0; c < 3; ++c) {
          gG[c * N + node] += gp.N[a] * gp.wj0 * gP[c] / mass[node];
          if (gx) gx[c * N + node] += gp.N[a] * gchi[c];
        }
      }
    }
  }
  return 0;
}

// Adjoint of interpolation.  With U_a = m_a^-1 sum_q N_a w_q j0 U^IB_q and
// U^IB_q = sum_faces u^c prod phi:
//   gU^IB_q = w_q j0 sum_a N_a gU_a / m_a,  gu^c(face) = sum_q gU^IB_q^c prod phi,
//   gx_a = sum_q N_a gchi_q,  gchi_q,d = sum_c gU^IB_q^c h^-1 sum_faces u^c phi'(r_d) prod phi.
int or_interp_adj(const or_grid* g, const or_mesh* m, const double* x, const double* u,
                  const double* gU, double* gu, double* gx) {
  if (!check_grid(g) || !check_mesh(m)) return -1;
  int64_t E = m->n_elems, N = m->n_nodes;
  int64_t cells = (int64_t)g->n[0] * g->n[1] * g->n[2];
  std::vector<double> mass(N);
  int rc = or_lumped_mass(m, mass.data());
  if (rc) return rc;
  std::memset(gu, 0, sizeof(double) * 3 * cells);
  if (gx) std::memset(gx, 0, sizeof(double) * 3 * N);
  double h = g->h;
  for (int e = 0; e < E; ++e) {
    double Xe[kMaxC][3], xe[kMaxC][3], gUe[kMaxC][3];
    gather(m, m->X, e, Xe);
    gather(m, x, e, xe);
    gather(m, gU, e, gUe);
    for (int q = 0; q < nq_of(m); ++q) {
      GaussPt gp;
      if (!gauss_point(m, Xe, q, gp)) return -2;
      double chi[3], gq[3], gchi[3] = {0, 0, 0};
      point_of(gp, xe, chi);
      for (int i = 0; i < 3; ++i) {
        gq[i] = 0.0;
        for (int a = 0; a < nc_of(m); ++a) gq[i] += gp.N[a] * gUe[a][i] / mass[m->conn[a * E + e]];
        gq[i] *= gp.wj0;
      }
      for (int c = 0; c < 3; ++c) {
        Stencil s;
        stencil(g, c, chi, s);
        double d0 = 0.0, d1 = 0.0, d2 = 0.0;
        for (int kz = 0; kz < 4; ++kz)
          for (int ky = 0; ky < 4; ++ky)
            for (int kx = 0; kx < 4; ++kx) {
              int64_t fi = face_index(g, c, s.idx[0][kx], s.idx[1][ky], s.idx[2][kz]);
              gu[fi] += gq[c] * s.w[0][kx] * s.w[1][ky] * s.w[2][kz];
              double v = u[fi];
              d0 += v * s.dw[0][kx] * s.w[1][ky] * s.w[2][kz];
              d1 += v * s.w[0][kx] * s.dw[1][ky] * s.w[2][kz];
              d2 += v * s.w[0][kx] * s.w[1][ky] * s.dw[2][kz];
            }
        gchi[0] += gq[c] * d0 / h;
        gchi[1] += gq[c] * d1 / h;
        gchi[2] += gq[c] * d2 / h;
      }
      if (gx)
        for (int a = 0; a < nc_of(m); ++a) {
          int64_t node = m->conn[a * E + e];
          for (int c = 0; c < 3; ++c) gx[c * N + node] += gp.N[a] * gchi[c];
        }
    }
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Nodal quadrature rule (Section 4.4, the rule N_q of the nodes): the
// coupling points are the nodes' displaced positions x_a.
//   U^IB_a = sum_faces u^c(face) prod_d phi(r_d)              (interpolation; with
//            the nodal rule the lumped L2 projection leaves U_a = U^IB_a)
//   f^c(face) = sum_a F_a^c delta_h(x_face - x_a) = h^-3 sum_a G_a^c prod phi
//            (spreading of the mean nodal force contributions F_i = G)
// ---------------------------------------------------------------------------
int or_spread_nodal(const or_grid* g, int64_t N, const double* x, const double* G, double* f) {
  if (!check_grid(g) || N < 0) return -1;
  int64_t cells = (int64_t)g->n[0] * g->n[1] * g->n[2];
  std::memset(f, 0, sizeof(double) * 3 * cells);
  double h3 = g->h * g->h * g->h;
  for (int64_t a = 0; a < N; ++a) {
    double chi[3] = {x[a], x[N + a], x[2 * N + a]};
    for (int c = 0; c < 3; ++c) {
      Stencil s;
      stencil(g, c, chi, s);
      for (int kz = 0; kz < 4; ++kz)
        for (int ky = 0; ky < 4; ++ky)
          for (int kx = 0; kx < 4; ++kx)
            f[face_index(g, c, s.idx[0][kx], s.idx[1][ky], s.idx[2][kz])] +=
                G[c * N + a] * s.w[0][kx] * s.w[1][ky] * s.w[2][kz] / h3;
    }
  }
  return 0;
}

// Brute force at selected faces: every node, the nearest periodic image of
// each distance, phi evaluated directly.
int or_spread_nodal_at(const or_grid* g, int64_t N, const double* x, const double* G,
                       int64_t n_sel, const int32_t* comp, const int32_t* idx, double* out) {
  if (!check_grid(g) || N < 0) return -1;
  double h3 = g->h * g->h * g->h;
  for (int64_t k = 0; k < n_sel; ++k) {
    int c = comp[k];
    double acc = 0.0;
    for (int64_t a = 0; a < N; ++a) {
      double w = 1.0;
      for (int d = 0; d < 3 && w != 0.0; ++d) {
        double sh = (d == c) ? 0.0 : 0.5;
        double r = (x[d * N + a] - g->origin[d]) / g->h - sh - idx[3 * k + d];
        r -= g->n[d] * std::floor(r / g->n[d] + 0.5);
        w *= phi(r);
      }
      acc += G[c * N + a] * w / h3;
    }
    out[k] = acc;
  }
  return 0;
}

int or_interp_nodal(const or_grid* g, int64_t N, const double* x, const double* u, double* U) {
  if (!check_grid(g) || N < 0) return -1;
  for (int64_t a = 0; a < N; ++a) {
    double chi[3] = {x[a], x[N + a], x[2 * N + a]};
    for (int c = 0; c < 3; ++c) {
      Stencil s;
      stencil(g, c, chi, s);
      double acc = 0.0;
      for (int kz = 0; kz < 4; ++kz)
        for (int ky = 0; ky < 4; ++ky)
          for (int kx = 0; kx < 4; ++kx)
            acc += u[face_index(g, c, s.idx[0][kx], s.idx[1][ky], s.idx[2][kz])] *
                   s.w[0][kx] * s.w[1][ky] * s.w[2][kz];
      U[c * N + a] = acc;
    }
  }
  return 0;
}

// Adjoint of nodal spreading: gG_a^c = h^-3 sum_faces gf^c prod phi and
// gx_a,d = h^-4 sum_c G_a^c sum_faces gf^c phi'(r_d) prod_{d' != d} phi.
int or_spread_nodal_adj(const or_grid* g, int64_t N, const double* x, const double* G,
                        const double* gf, double* gG, double* gx) {
  if (!check_grid(g) || N < 0) return -1;
  double h = g->h, h3 = h * h * h;
  for (int64_t a = 0; a < N; ++a) {
    double chi[3] = {x[a], x[N + a], x[2 * N + a]}, gchi[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c) {
      Stencil s;
      stencil(g, c, chi, s);
      double acc = 0.0, d0 = 0.0, d1 = 0.0, d2 = 0.0;
      for (int kz = 0; kz < 4; ++kz)
        for (int ky = 0; ky < 4; ++ky)
          for (int kx = 0; kx < 4; ++kx) {
            double v = gf[face_index(g, c, s.idx[0][kx], s.idx[1][ky], s.idx[2][kz])];
            acc += v * s.w[0][kx] * s.w[1][ky] * s.w[2][kz];
            d0 += v * s.dw[0][kx] * s.w[1][ky] * s.w[2][kz];
            d1 += v * s.w[0][kx] * s.dw[1][ky] * s.w[2][kz];
            d2 += v * s.w[0][kx] * s.w[1][ky] * s.dw[2][kz];
          }
      gG[c * N + a] = acc / h3;
      gchi[0] += G[c * N + a] * d0 / (h3 * h);
      gchi[1] += G[c * N + a] * d1 / (h3 * h);
      gchi[2] += G[c * N + a] * d2 / (h3 * h);
    }
    if (gx)
      for (int d = 0; d < 3; ++d) gx[d * N + a] = gchi[d];
  }
  return 0;
}

// Adjoint of nodal interpolation: gu^c(face) = sum_a gU_a^c prod phi and
// gx_a,d = h^-1 sum_c gU_a^c sum_faces u^c phi'(r_d) prod_{d' != d} phi.
int or_interp_nodal_adj(const or_grid* g, int64_t N, const double* x, const double* u,
                        const double* gU, double* gu, double* gx) {
  if (!check_grid(g) || N < 0) return -1;
  int64_t cells = (int64_t)g->n[0] * g->n[1] * g->n[2];
  std::memset(gu, 0, sizeof(double) * 3 * cells);
  double h = g->h;
  for (int64_t a = 0; a < N; ++a) {
    double chi[3] = {x[a], x[N + a], x[2 * N + a]}, gchi[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c) {
      Stencil s;
      stencil(g, c, chi, s);
      double d0 = 0.0, d1 = 0.0, d2 = 0.0;
      for (int kz = 0; kz < 4; ++kz)
        for (int ky = 0; ky < 4; ++ky)
          for (int kx = 0; kx < 4; ++kx) {
            int64_t fi = face_index(g, c, s.idx[0][kx], s.idx[1][ky], s.idx[2][kz]);
            gu[fi] += gU[c * N + a] * s.w[0][kx] * s.w[1][ky] * s.w[2][kz];
            double v = u ? u[fi] : 0.0;
            d0 += v * s.dw[0][kx] * s.w[1][ky] * s.w[2][kz];
            d1 += v * s.w[0][kx] * s.dw[1][ky] * s.w[2][kz];
            d2 += v * s.w[0][kx] * s.w[1][ky] * s.dw[2][kz];
          }
      gchi[0] += gU[c * N + a] * d0 / h;
      gchi[1] += gU[c * N + a] * d1 / h;
      gchi[2] += gU[c * N + a] * d2 / h;
    }
    if (gx)
      for (int d = 0; d < 3; ++d) gx[d * N + a] = gchi[d];
  }
  return 0;
}

int64_t or_support_count(const or_grid* g, const or_mesh* m, const double* x) {
  if (!check_grid(g) || !check_mesh(m)) return -1;
  int64_t E = m->n_elems;
  int64_t cells = (int64_t)g->n[0] * g->n[1] * g->n[2];
  std::vector<unsigned char> mark(3 * cells, 0);
  for (int e = 0; e < E; ++e) {
    double Xe[kMaxC][3], xe[kMaxC][3];
    gather(m, m->X, e, Xe);
    gather(m, x, e, xe);
    for (int q = 0; q < nq_of(m); ++q) {
      GaussPt gp;
      if (!gauss_point(m, Xe, q, gp)) return -2;
      double chi[3];
      point_of(gp, xe, chi);
      for (int c = 0; c < 3; ++c) {
        Stencil s;
        stencil(g, c, chi, s);
        for (int kz = 0; kz < 4; ++kz)
          for (int ky = 0; ky < 4; ++ky)
            for (int kx = 0; kx < 4; ++kx)
              mark[face_index(g, c, s.idx[0][kx], s.idx[1][ky], s.idx[2][kz])] = 1;
      }
    }
  }
  int64_t count = 0;
  for (int64_t i = 0; i < 3 * cells; ++i) count += mark[i];
  return count;
}

}  // extern "C"
