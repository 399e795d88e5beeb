// Oracle for the space-time (p,delta)-Navier-Stokes slab operator.
//
// TEST INFRASTRUCTURE ONLY.  This is a plain, slow, FP64 CPU restatement of
// what the method computes on one time slab S_n = Omega x I_n:
//   * the slab residual R_n(U) = -[(K_t (x) M_x) V - (m_t (x) M_x) v^-; 0]
//                                + (M_t (x) I) F(U)                (eq. slab-underint, Sec. 5.2)
//   * the slab Jacobian J_n = [[K_t (x) M_x, 0], [0, 0]]
//                                + (M_t (x) I) diag(J_1..J_{k+1})  (eq. slab-underint-jac)
//     with the Pic / exN / modN constitutive tangents (Sec. 4.2-4.4),
//   * the block mass-weighted norm (Sec. 6.1).
// Everything is done by plain element loops: basis functions are evaluated
// pointwise at every quadrature point, element matrices are formed entry by
// entry, nothing is sum-factorised, fused or reordered.
//
// Only the tests, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
// load this library.  It shares no code with the CUDA library.
//
// Discretisation (readings of the paper, shared with the CUDA path only as
// mathematics):
//   * uniform box mesh [0,Lx]x[0,Ly](x[0,Lz]) of nx x ny (x nz) cells;
//   * Q2 continuous velocity; Q1 continuous pressure (Taylor-Hood, Sec. 3.1)
//     or, with pressure_space = 1, the discontinuous P1 pressure of the
//     paper's experiments (Q2/P1disc, Sec. 7): per cell the basis 1 and
//     2 r_a - 1 (r_a the reference coordinates), cell-wise dofs;
//   * tensor 3-point Gauss quadrature in cells, 3x3 on faces;
//   * DG(k) in time, Lagrange basis on right Gauss-Radau nodes (Sec. 3.1,
//     Rem. 3.2); time integrals by the (k+1)-point Radau rule (Sec. 5.2);
//   * Nitsche terms B_gamma = B^c + B^s + B^r_gamma (eq. def-b-gam) with the
//     viscous coefficients frozen at the lifting g_hat (Sec. 3.2); the sign of
//     the (u.n, q) term in B^s is the parameter q_sign (-1 = the printed text);
//   * h_GammaD = cell edge length normal to the face;
//   * CIP (eq. scip-def, weight gamma_cip; 0 = off) on the interior faces,
//     its advecting field lagged in the Jacobian (Sec. 4.3); h_F = the
//     diameter (diagonal) of the face.
//
// Unknown layout: U = [V_1 .. V_{k+1} | P_1 .. P_{k+1}], V_mu component-major,
// each component lexicographic (x fastest) on the Q2 node grid
// (2nx+1)(2ny+1)(2nz+1); P_mu lexicographic on the Q1 grid.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {
struct OrParams {
  int dim, nx, ny, nz;
  double Lx, Ly, Lz;
  int k;
  double t0, dt;
  double p, delta, nu, nu_inf, sigma_max;
  double gamma1, gamma2;
  unsigned dirichlet_mask;  // bit s (s = 2*axis + upper) set: side s is Gamma_D
  int inflow_profile;       // 0: g_D = 0; 1: parabolic x-inflow, lifting constant in x
  double vbar;
  double q_sign;            // coefficient of (u.n, q)_{Gamma_D} in B^s
  double gamma_cip;         // CIP weight gamma_CIP of eq. scip-def (0: no CIP)
  int pressure_space;       // 0: Q1 continuous (Taylor-Hood); 1: P1disc (Sec. 7)
};
}

namespace {

enum { PIC = 0, EXN = 1, MODN = 2 };

// term mask bits for the linearised spatial form (all set = the full J_mu)
enum {
  T_VISC = 1,       // (T(D du), D z)
  T_CONV = 2,       // convection volume + boundary + inflow terms
  T_PRES = 4,       // -(div z, dpi) - (div du, q) + (dpi, z.n)_GD
  T_VFLUX = 8,      // -(T(D du) n, z)_GD
  T_BS = 16,        // -(du, DS(D g_hat)(D z) n)_GD
  T_BR = 32,        // gamma1/h (eta_D du, z) + gamma2/h (du.n, z.n)
  T_BQ = 64,        // q_sign (du.n, q)_GD
  T_ALL = 127
};

// ---------------------------------------------------------------- 1D tables
double legendre(int n, double s) {
  if (n == 0) return 1.0;
  double p0 = 1.0, p1 = s;
  for (int m = 1; m < n; ++m) {
    double p2 = ((2.0 * m + 1.0) * s * p1 - m * p0) / (m + 1.0);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// Gauss-Legendre rule with n points mapped to [0,1], ascending.
void gauss01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double s = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double pn = legendre(n, s), pm = legendre(n - 1, s);
      dp = n * (s * pn - pm) / (s * s - 1.0);
      double ds = pn / dp;
      s -= ds;
      if (std::fabs(ds) < 1e-16) break;
    }
    double pn = legendre(n, s), pm = legendre(n - 1, s);
    dp = n * (s * pn - pm) / (s * s - 1.0);
    x[i] = 0.5 * (s + 1.0);
    w[i] = 1.0 / ((1.0 - s * s) * dp * dp);  // (2/((1-s^2)P'^2)) / 2
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (x[j] < x[i]) {
        std::swap(x[i], x[j]);
        std::swap(w[i], w[j]);
      }
}

// Right-sided (k+1)-point Gauss-Radau nodes on [0,1]: the zeros of
// P_{k+1}(s) - P_k(s) on [-1,1] (s = 1 is one of them), found by bisection.
void radau_right01(int k, double* t) {
  const int n = k + 1;
  auto f = [&](double s) { return legendre(n, s) - legendre(n - 1, s); };
  int found = 0;
  const int grid = 20000;
  double a = -1.0, fa = f(a);
  for (int i = 1; i <= grid && found < k; ++i) {
    double b = -1.0 + 2.0 * i / grid * (1.0 - 1e-7);
    double fb = f(b);
    if (fa * fb < 0.0) {
      double lo = a, hi = b, flo = fa;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi), fm = f(mid);
        if ((fm < 0.0) == (flo < 0.0)) {
          lo = mid;
          flo = fm;
        } else {
          hi = mid;
        }
      }
      t[found++] = 0.5 * (0.5 * (lo + hi) + 1.0);
    }
    a = b;
    fa = fb;
  }
  t[k] = 1.0;
}

double lagrange(const double* nodes, int n, int i, double x) {
  double r = 1.0;
  for (int j = 0; j < n; ++j)
    if (j != i) r *= (x - nodes[j]) / (nodes[i] - nodes[j]);
  return r;
}

double lagrange_d(const double* nodes, int n, int i, double x) {
  double s = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m == i) continue;
    double r = 1.0 / (nodes[i] - nodes[m]);
    for (int j = 0; j < n; ++j)
      if (j != i && j != m) r *= (x - nodes[j]) / (nodes[i] - nodes[j]);
    s += r;
  }
  return s;
}

struct TimeTables {
  int k;
  double t[8], w[8];      // Radau nodes/weights on [0,1]
  double Kt[8][8], mt[8];  // temporal matrices of Sec. 5.2 (reference interval)
  double Mt[8][8];         // reference mass (diagonal in exact arithmetic)
};

void time_tables(int k, TimeTables& T) {
  T.k = k;
  const int n = k + 1;
  radau_right01(k, T.t);
  double gx[16], gw[16];
  const int ng = k + 3;  // exact for polynomial degree <= 2k+5
  gauss01(ng, gx, gw);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int q = 0; q < ng; ++q) s += gw[q] * lagrange(T.t, n, i, gx[q]);
    T.w[i] = s;
    T.mt[i] = lagrange(T.t, n, i, 0.0);
    for (int j = 0; j < n; ++j) {
      double kij = 0.0, mij = 0.0;
      for (int q = 0; q < ng; ++q) {
        kij += gw[q] * lagrange_d(T.t, n, j, gx[q]) * lagrange(T.t, n, i, gx[q]);
        mij += gw[q] * lagrange(T.t, n, j, gx[q]) * lagrange(T.t, n, i, gx[q]);
      }
      T.Kt[i][j] = kij + lagrange(T.t, n, j, 0.0) * lagrange(T.t, n, i, 0.0);
      T.Mt[i][j] = mij;
    }
  }
}

// ------------------------------------------------------------------- mesh
struct Geo {
  int d, k;
  int n[3];
  double h[3];
  long g2[3], g1[3];  // global Q2 / Q1 points per direction (1 in an absent dir)
  int l2[3], l1[3], lq[3];
  long Nq2, Nq1, Mv, Mp, Nst;
  int nv, np, ne;  // local velocity dofs, local pressure dofs, total per node
  long ncells;
  bool pdisc;      // P1disc pressure
};

Geo make_geo(const OrParams& P) {
  Geo G;
  G.d = P.dim;
  G.k = P.k;
  int nn[3] = {P.nx, P.ny, P.dim == 3 ? P.nz : 1};
  double L[3] = {P.Lx, P.Ly, P.dim == 3 ? P.Lz : 1.0};
  G.Nq2 = 1;
  G.Nq1 = 1;
  G.ncells = 1;
  int nloc2 = 1, nloc1 = 1;
  for (int a = 0; a < 3; ++a) {
    bool act = a < P.dim;
    G.n[a] = nn[a];
    G.h[a] = act ? L[a] / nn[a] : 1.0;
    G.g2[a] = act ? 2L * nn[a] + 1 : 1;
    G.g1[a] = act ? (long)nn[a] + 1 : 1;
    G.l2[a] = act ? 3 : 1;
    G.l1[a] = act ? 2 : 1;
    G.lq[a] = act ? 3 : 1;
    G.Nq2 *= G.g2[a];
    G.Nq1 *= G.g1[a];
    G.ncells *= nn[a];
    nloc2 *= G.l2[a];
    nloc1 *= G.l1[a];
  }
  G.pdisc = P.pressure_space == 1;
  if (G.pdisc) {
    nloc1 = G.d + 1;                      // 1, 2 r_0 - 1, .., 2 r_{d-1} - 1 on every cell
    G.Nq1 = G.ncells * (long)nloc1;
  }
  G.Mv = G.d * G.Nq2;
  G.Mp = G.Nq1;
  G.Nst = (long)(G.k + 1) * (G.Mv + G.Mp);
  G.nv = G.d * nloc2;
  G.np = nloc1;
  G.ne = G.nv + G.np;
  return G;
}

struct CellPos {
  int e[3];
};

CellPos cell_pos(const Geo& G, long cell) {
  CellPos c;
  c.e[0] = (int)(cell % G.n[0]);
  c.e[1] = (int)((cell / G.n[0]) % G.n[1]);
  c.e[2] = (int)(cell / ((long)G.n[0] * G.n[1]));
  return c;
}

// Spatial local dof -> global index within one time node's block
// (velocity: c*Nq2 + node, pressure: Mv + node1).  Local order: velocity
// component-major, local nodes lexicographic; then pressure nodes.
void cell_spatial_dofs(const Geo& G, long cell, long* out) {
  CellPos c = cell_pos(G, cell);
  int idx = 0;
  for (int comp = 0; comp < G.d; ++comp)
    for (int z = 0; z < G.l2[2]; ++z)
      for (int y = 0; y < G.l2[1]; ++y)
        for (int x = 0; x < G.l2[0]; ++x) {
          long gx = 2L * c.e[0] + x, gy = 2L * c.e[1] + y, gz = (G.d == 3) ? 2L * c.e[2] + z : 0;
          out[idx++] = comp * G.Nq2 + gx + G.g2[0] * (gy + G.g2[1] * gz);
        }
  if (G.pdisc) {
    for (int j = 0; j < G.np; ++j) out[idx++] = G.Mv + cell * G.np + j;
    return;
  }
  for (int z = 0; z < G.l1[2]; ++z)
    for (int y = 0; y < G.l1[1]; ++y)
      for (int x = 0; x < G.l1[0]; ++x) {
        long gx = c.e[0] + x, gy = c.e[1] + y, gz = (G.d == 3) ? c.e[2] + z : 0;
        out[idx++] = G.Mv + gx + G.g1[0] * (gy + G.g1[1] * gz);
      }
}

// spatial block index -> global slab index for time node mu
long st_index(const Geo& G, int mu, long sidx) {
  if (sidx < G.Mv) return (long)mu * G.Mv + sidx;
  return (long)(G.k + 1) * G.Mv + (long)mu * G.Mp + (sidx - G.Mv);
}

// --------------------------------------------------------- basis at a point
// Values/gradients of all local Q2 and Q1 basis functions at a point given by
// its reference coordinates r[a] in the cell (absent directions: unused).
struct PointBasis {
  double phi[27], dphi[27][3];  // Q2 scalar basis
  double psi[8];                // pressure basis (Q1, or P1disc)
};

const double Q2N[3] = {0.0, 0.5, 1.0};
const double Q1N[2] = {0.0, 1.0};

void point_basis(const Geo& G, const double r[3], PointBasis& B) {
  double v2[3][3], d2[3][3], v1[3][2];
  for (int a = 0; a < 3; ++a) {
    if (a < G.d) {
      for (int i = 0; i < 3; ++i) {
        v2[a][i] = lagrange(Q2N, 3, i, r[a]);
        d2[a][i] = lagrange_d(Q2N, 3, i, r[a]) / G.h[a];
      }
      for (int i = 0; i < 2; ++i) v1[a][i] = lagrange(Q1N, 2, i, r[a]);
    } else {
      v2[a][0] = 1.0;
      d2[a][0] = 0.0;
      v1[a][0] = 1.0;
    }
  }
  int idx = 0;
  for (int z = 0; z < G.l2[2]; ++z)
    for (int y = 0; y < G.l2[1]; ++y)
      for (int x = 0; x < G.l2[0]; ++x) {
        B.phi[idx] = v2[0][x] * v2[1][y] * v2[2][z];
        B.dphi[idx][0] = d2[0][x] * v2[1][y] * v2[2][z];
        B.dphi[idx][1] = v2[0][x] * d2[1][y] * v2[2][z];
        B.dphi[idx][2] = v2[0][x] * v2[1][y] * d2[2][z];
        ++idx;
      }
  idx = 0;
  if (G.pdisc) {
    B.psi[idx++] = 1.0;
    for (int a = 0; a < G.d; ++a) B.psi[idx++] = 2.0 * r[a] - 1.0;
    return;
  }
  for (int z = 0; z < G.l1[2]; ++z)
    for (int y = 0; y < G.l1[1]; ++y)
      for (int x = 0; x < G.l1[0]; ++x) B.psi[idx++] = v1[0][x] * v1[1][y] * v1[2][z];
}

// Quadrature points of a cell (volume) or of one of its faces, with weights
// including the Jacobian of the affine map.  side < 0: volume.
struct QPoint {
  double r[3];
  double w;
};

std::vector<QPoint> quad_points(const Geo& G, int side) {
  double gx[3], gw[3];
  gauss01(3, gx, gw);
  std::vector<QPoint> pts;
  int axis = side >= 0 ? side / 2 : -1;
  int upper = side >= 0 ? side % 2 : 0;
  int cnt[3];
  for (int a = 0; a < 3; ++a) cnt[a] = (a < G.d && a != axis) ? 3 : 1;
  for (int z = 0; z < cnt[2]; ++z)
    for (int y = 0; y < cnt[1]; ++y)
      for (int x = 0; x < cnt[0]; ++x) {
        int id[3] = {x, y, z};
        QPoint q;
        q.w = 1.0;
        for (int a = 0; a < 3; ++a) {
          if (a == axis) {
            q.r[a] = upper ? 1.0 : 0.0;
          } else if (a < G.d) {
            q.r[a] = gx[id[a]];
            q.w *= gw[id[a]] * G.h[a];
          } else {
            q.r[a] = 0.0;
          }
        }
        pts.push_back(q);
      }
  return pts;
}

// ---------------------------------------------------------- tensor helpers
template <class S>
S ddot(const S A[3][3], const S B[3][3]) {
  S s = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) s += A[i][j] * B[i][j];
  return s;
}

template <class S>
void sym_grad(const S g[3][3], S A[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) A[i][j] = 0.5 * (g[i][j] + g[j][i]);
}

// effective viscosity eta(A) = nu_inf + nu (delta^2 + |A|^2)^((p-2)/2), eq. constitutive-law
template <class S>
S eta_of(const OrParams& P, const S A[3][3]) {
  using std::pow;
  return P.nu_inf + P.nu * pow(P.delta * P.delta + ddot(A, A), 0.5 * (P.p - 2.0));
}

// S(A) = eta(A) A
template <class S>
void stress(const OrParams& P, const S A[3][3], S out[3][3]) {
  S e = eta_of(P, A);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) out[i][j] = e * A[i][j];
}

// Frechet derivative DS(A)(B) = eta(A) B + nu (p-2)(delta^2+|A|^2)^((p-4)/2) (A:B) A, eq. pns-dstress
void dstress(const OrParams& P, const double A[3][3], const double B[3][3], double out[3][3]) {
  double D2 = P.delta * P.delta + ddot(A, A);
  double e = P.nu_inf + P.nu * std::pow(D2, 0.5 * (P.p - 2.0));
  double beta = P.nu * (P.p - 2.0) * std::pow(D2, 0.5 * (P.p - 4.0));
  double ab = ddot(A, B);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) out[i][j] = e * B[i][j] + beta * ab * A[i][j];
}

// Constitutive tangents at the iterate A = A^m (Sec. 4.1-4.4):
//   Pic : T(B) = eta B                                           eq. local-tangent-picard
//   exN : T(B) = eta B + (p-2) mu/Delta^2 (A:B) A                 eq. local-tangent-exact
//   modN: T(B) = eta B + s theta (sigma:B) sigma, sigma = mu A,
//         s = min{1, sigma_max/|sigma|} (0 if sigma = 0),
//         theta = (p-2)/(mu Delta^2)                              eq. local-tangent-clip
void tangent(const OrParams& P, int var, const double A[3][3], const double B[3][3], double T[3][3]) {
  double D2 = P.delta * P.delta + ddot(A, A);
  double mu = P.nu * std::pow(D2, 0.5 * (P.p - 2.0));
  double eta = P.nu_inf + mu;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) T[i][j] = eta * B[i][j];
  if (var == EXN) {
    double c = (P.p - 2.0) * mu / D2 * ddot(A, B);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) T[i][j] += c * A[i][j];
  } else if (var == MODN) {
    double sigma[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) sigma[i][j] = mu * A[i][j];
    double ns = std::sqrt(ddot(sigma, sigma));
    double s = ns > 0.0 ? std::min(1.0, P.sigma_max / ns) : 0.0;
    if (s > 0.0) {
      double theta = (P.p - 2.0) / (mu * D2);
      double c = s * theta * ddot(sigma, B);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[i][j] += c * sigma[i][j];
    }
  }
}

// Lifting g_hat of the Dirichlet data and its gradient (grad[i][j] = d_j g_i).
// inflow_profile 1: g_hat = (vbar * 6 y(1-y) [* 6 z(1-z)], 0, 0) in scaled
// coordinates, constant in x.  Optional nodal field gnod (Q2 coefficients of
// a velocity field) replaces it when given (test hook).
struct Lift {
  double g[3];
  double grad[3][3];
};

void lifting_analytic(const OrParams& P, const double x[3], Lift& L) {
  for (int i = 0; i < 3; ++i) {
    L.g[i] = 0.0;
    for (int j = 0; j < 3; ++j) L.grad[i][j] = 0.0;
  }
  if (P.inflow_profile != 1) return;
  double y = x[1] / P.Ly;
  double fy = 6.0 * y * (1.0 - y), dfy = 6.0 * (1.0 - 2.0 * y) / P.Ly;
  double fz = 1.0, dfz = 0.0;
  if (P.dim == 3) {
    double z = x[2] / P.Lz;
    fz = 6.0 * z * (1.0 - z);
    dfz = 6.0 * (1.0 - 2.0 * z) / P.Lz;
  }
  L.g[0] = P.vbar * fy * fz;
  L.grad[0][1] = P.vbar * dfy * fz;
  if (P.dim == 3) L.grad[0][2] = P.vbar * fy * dfz;
}

double neg_part(double y) { return 0.5 * (std::fabs(y) - y); }  // "(y)_-" of Sec. 3.2

struct Ctx {
  OrParams P;
  Geo G;
  TimeTables T;
  std::vector<QPoint> vol;
  std::vector<QPoint> face[6];
};

void make_ctx(const OrParams* P, Ctx& C) {
  C.P = *P;
  C.G = make_geo(*P);
  time_tables(P->k, C.T);
  C.vol = quad_points(C.G, -1);
  for (int s = 0; s < 2 * C.G.d; ++s) C.face[s] = quad_points(C.G, s);
}

bool on_side(const Geo& G, const CellPos& c, int side) {
  int axis = side / 2, upper = side % 2;
  return upper ? (c.e[axis] == G.n[axis] - 1) : (c.e[axis] == 0);
}

void phys_point(const Geo& G, const CellPos& c, const double r[3], double x[3]) {
  for (int a = 0; a < 3; ++a) x[a] = a < G.d ? (c.e[a] + r[a]) * G.h[a] : 0.0;
}

// Lifting at a point: analytic, or interpolated from gnod on this cell.
void lifting_at(const Ctx& C, const CellPos& c, const long* sd, const PointBasis& B, const double r[3],
                const double* gnod, Lift& L) {
  if (!gnod) {
    double x[3];
    phys_point(C.G, c, r, x);
    lifting_analytic(C.P, x, L);
    return;
  }
  const Geo& G = C.G;
  int nl = G.nv / G.d;
  for (int i = 0; i < 3; ++i) {
    L.g[i] = 0.0;
    for (int j = 0; j < 3; ++j) L.grad[i][j] = 0.0;
  }
  for (int comp = 0; comp < G.d; ++comp)
    for (int a = 0; a < nl; ++a) {
      double v = gnod[sd[comp * nl + a]];
      L.g[comp] += v * B.phi[a];
      for (int j = 0; j < 3; ++j) L.grad[comp][j] += v * B.dphi[a][j];
    }
}

// ------------------------------------------------------------ residual
// Local residual of one cell, all time nodes: Rloc[mu*ne + i].
// F_mu = RHS_mu - LHS_mu where (eq. disc, def-a-gam, def-b-gam, Defc)
//  LHS(z,q) = (S(Du),Dz) - (u(x)u, grad z) - (pi, div z) - (div u, q)
//           + ((u.n)u, z)_Gamma
//           + on Gamma_D: -(S(Du)n, z) + (pi, z.n) - ((u.n)_- u, z)
//                         - (u, DS(Dg)(Dz)n) + q_sign (u.n, q)
//                         + gamma1/h (eta_D u, z) + gamma2/h (u.n, z.n)
//  RHS(z,q) = (f, z) + the same B_gamma terms with u -> g_D.
// f enters through its Q2 nodal interpolant per time node.
template <class S>
void cell_residual(const Ctx& C, long cell, const S* U, const double* vprev, const double* f, const double* gnod,
                   S* Rloc) {
  const Geo& G = C.G;
  const OrParams& P = C.P;
  const int K1 = G.k + 1;
  const int nl = G.nv / G.d;  // local Q2 nodes
  const int ne = G.ne;
  long sd[128];
  cell_spatial_dofs(G, cell, sd);
  CellPos cp = cell_pos(G, cell);
  for (int i = 0; i < K1 * ne; ++i) Rloc[i] = 0.0;

  std::vector<S> ue(ne);
  std::vector<double> fe(G.nv);
  PointBasis B;
  for (int mu = 0; mu < K1; ++mu) {
    for (int i = 0; i < ne; ++i) ue[i] = U[st_index(G, mu, sd[i])];
    if (f)
      for (int i = 0; i < G.nv; ++i) fe[i] = f[(long)mu * G.Mv + sd[i]];
    std::vector<S> F(ne, S(0.0));
    // volume
    for (const QPoint& q : C.vol) {
      point_basis(G, q.r, B);
      S u[3] = {0.0, 0.0, 0.0}, gu[3][3] = {}, pi = 0.0;
      double fq[3] = {0.0, 0.0, 0.0};
      for (int comp = 0; comp < G.d; ++comp)
        for (int a = 0; a < nl; ++a) {
          S v = ue[comp * nl + a];
          u[comp] += v * B.phi[a];
          for (int j = 0; j < 3; ++j) gu[comp][j] += v * B.dphi[a][j];
          if (f) fq[comp] += fe[comp * nl + a] * B.phi[a];
        }
      for (int a = 0; a < G.np; ++a) pi += ue[G.nv + a] * B.psi[a];
      S A[3][3], Sg[3][3];
      sym_grad(gu, A);
      stress(P, A, Sg);
      S divu = 0.0;
      for (int j = 0; j < G.d; ++j) divu += gu[j][j];
      for (int comp = 0; comp < G.d; ++comp)
        for (int a = 0; a < nl; ++a) {
          S lhs = 0.0;
          for (int j = 0; j < G.d; ++j) lhs += (Sg[comp][j] - u[comp] * u[j]) * B.dphi[a][j];
          lhs -= pi * B.dphi[a][comp];
          F[comp * nl + a] += q.w * (fq[comp] * B.phi[a] - lhs);
        }
      for (int a = 0; a < G.np; ++a) F[G.nv + a] += q.w * (divu * B.psi[a]);  // -(-(div u, q))
    }
    // boundary faces
    for (int side = 0; side < 2 * G.d; ++side) {
      if (!on_side(G, cp, side)) continue;
      const int axis = side / 2;
      double nrm[3] = {0.0, 0.0, 0.0};
      nrm[axis] = (side % 2) ? 1.0 : -1.0;
      const bool isD = (P.dirichlet_mask >> side) & 1u;
      const double hD = G.h[axis];
      for (const QPoint& q : C.face[side]) {
        point_basis(G, q.r, B);
        S u[3] = {0.0, 0.0, 0.0}, gu[3][3] = {}, pi = 0.0;
        for (int comp = 0; comp < G.d; ++comp)
          for (int a = 0; a < nl; ++a) {
            S v = ue[comp * nl + a];
            u[comp] += v * B.phi[a];
            for (int j = 0; j < 3; ++j) gu[comp][j] += v * B.dphi[a][j];
          }
        for (int a = 0; a < G.np; ++a) pi += ue[G.nv + a] * B.psi[a];
        S un = 0.0;
        for (int j = 0; j < G.d; ++j) un += u[j] * nrm[j];
        // convective boundary term on all of Gamma: LHS += ((u.n)u, z)
        for (int comp = 0; comp < G.d; ++comp)
          for (int a = 0; a < nl; ++a) F[comp * nl + a] -= q.w * un * u[comp] * B.phi[a];
        if (!isD) continue;
        Lift L;
        lifting_at(C, cp, sd, B, q.r, gnod, L);
        double Dg[3][3];
        sym_grad(L.grad, Dg);
        const double etaD = eta_of(P, Dg);
        double gn = 0.0;
        for (int j = 0; j < G.d; ++j) gn += L.g[j] * nrm[j];
        S A[3][3], Sg[3][3];
        sym_grad(gu, A);
        stress(P, A, Sg);
        // lagged-free real part of u.n decides the inflow factor (identical
        // for real arguments; for complex-step it freezes the factor)
        const double unr = std::real(un);
        const S wneg_u = neg_part(unr);
        const double wneg_g = neg_part(gn);
        // the difference u - g enters B^s and B^r (RHS - LHS)
        S dlt[3];
        for (int j = 0; j < 3; ++j) dlt[j] = (j < G.d) ? (u[j] - L.g[j]) : S(0.0);
        S dn = 0.0;
        for (int j = 0; j < G.d; ++j) dn += dlt[j] * nrm[j];
        for (int comp = 0; comp < G.d; ++comp)
          for (int a = 0; a < nl; ++a) {
            const double ph = B.phi[a];
            // LHS consistency terms: -(S(Du)n, z) + (pi, z.n)
            S Sn = 0.0;
            for (int j = 0; j < G.d; ++j) Sn += Sg[comp][j] * nrm[j];
            S lhs = -Sn * ph + pi * nrm[comp] * ph;
            // B^c: LHS -((u.n)_- u, z); RHS -((g.n)_- g, z)
            lhs += -wneg_u * u[comp] * ph;
            S rhs = -wneg_g * L.g[comp] * ph;
            // B^s viscous part on (u - g): -(dlt, DS(Dg)(Dz) n), Dz for z = phi e_comp
            double Bz[3][3] = {}, gz[3][3] = {};
            for (int j = 0; j < 3; ++j) gz[comp][j] = B.dphi[a][j];
            sym_grad(gz, Bz);
            double DSz[3][3];
            dstress(P, Dg, Bz, DSz);
            S bs = 0.0;
            for (int i = 0; i < G.d; ++i)
              for (int j = 0; j < G.d; ++j) bs += dlt[i] * DSz[i][j] * nrm[j];
            // B^r on (u - g)
            S br = P.gamma1 / hD * etaD * dlt[comp] * ph + P.gamma2 / hD * dn * nrm[comp] * ph;
            // F += RHS - LHS; B terms on u (LHS) and g (RHS) combine to -(B(u)-B(g))
            F[comp * nl + a] += q.w * (rhs - lhs - (-bs + br));
          }
        // B^s pressure part: q_sign (u.n, q) on LHS, q_sign (g.n, q) on RHS
        for (int a = 0; a < G.np; ++a) F[G.nv + a] -= q.w * P.q_sign * dn * B.psi[a];
      }
    }
    const double tw = P.dt * C.T.w[mu];
    for (int i = 0; i < ne; ++i) Rloc[mu * ne + i] += tw * F[i];
  }
  // temporal terms: -(K_t (x) M_x) V + (m_t (x) M_x) v^-
  std::vector<double> Me((size_t)nl * nl, 0.0);
  for (const QPoint& q : C.vol) {
    point_basis(G, q.r, B);
    for (int a = 0; a < nl; ++a)
      for (int b = 0; b < nl; ++b) Me[a * nl + b] += q.w * B.phi[a] * B.phi[b];
  }
  for (int i = 0; i < K1; ++i)
    for (int comp = 0; comp < G.d; ++comp)
      for (int a = 0; a < nl; ++a) {
        S s = 0.0;
        for (int b = 0; b < nl; ++b) {
          long sidx = sd[comp * nl + b];
          S mix = 0.0;
          for (int j = 0; j < K1; ++j) mix += C.T.Kt[i][j] * U[st_index(G, j, sidx)];
          double vp = vprev ? vprev[sidx] : 0.0;
          s += Me[a * nl + b] * (mix - C.T.mt[i] * vp);
        }
        Rloc[i * ne + comp * nl + a] -= s;
      }
}

// ------------------------------------------------------ spatial Jacobian
// Spatial element matrix Je[test*ne + trial] of the linearised left-hand
// side at one time node (J_mu = -D F_mu for the chosen variant), for the
// velocity state ue (local velocity values at that node).
//   viscous:  (T(D du), D z) - (T(D du) n, z)_GD
//   convection exN/modN: -(du(x)u + u(x)du, grad z) + ((du.n)u + (u.n)du, z)_Gamma
//                        - ((u.n)_- du, z)_GD        [(.)_- lagged, Sec. 4.1]
//   convection Pic: -(du(x)u, grad z) + ((u.n)du, z)_Gamma - ((u.n)_- du, z)_GD
//             (the advecting factor u_j of u_i u_j d_j z_i is lagged)
//   pressure: -(dpi, div z) - (div du, q) + (dpi, z.n)_GD
//   Nitsche:  -(du, DS(Dg)(Dz) n)_GD + q_sign (du.n, q)_GD
//             + gamma1/h (eta_D du, z)_GD + gamma2/h (du.n, z.n)_GD
void cell_spatial_jacobian(const Ctx& C, long cell, int var, const double* ue, const double* gnod, int mask,
                           double* Je) {
  const Geo& G = C.G;
  const OrParams& P = C.P;
  const int nl = G.nv / G.d;
  const int ne = G.ne;
  long sd[128];
  cell_spatial_dofs(G, cell, sd);
  CellPos cp = cell_pos(G, cell);
  for (int i = 0; i < ne * ne; ++i) Je[i] = 0.0;
  PointBasis B;
  // trial fluxes: for trial dof j, gradient-test flux Gf[j][c][m] (coefficient
  // of d_m z_c), value-test flux Vf[j][c] and pressure-test flux Qf[j]
  std::vector<double> Gf((size_t)ne * 9), Vf((size_t)ne * 3), Qf(ne);
  auto accumulate = [&](double w) {
    for (int t = 0; t < ne; ++t) {
      for (int j = 0; j < ne; ++j) {
        double s = 0.0;
        if (t < G.nv) {
          int comp = t / nl, a = t % nl;
          for (int m = 0; m < G.d; ++m) s += Gf[j * 9 + comp * 3 + m] * B.dphi[a][m];
          s += Vf[j * 3 + comp] * B.phi[a];
        } else {
          s += Qf[j] * B.psi[t - G.nv];
        }
        Je[t * ne + j] += w * s;
      }
    }
  };
  auto state_at = [&](double u[3], double gu[3][3]) {
    for (int i = 0; i < 3; ++i) {
      u[i] = 0.0;
      for (int j = 0; j < 3; ++j) gu[i][j] = 0.0;
    }
    for (int comp = 0; comp < G.d; ++comp)
      for (int a = 0; a < nl; ++a) {
        u[comp] += ue[comp * nl + a] * B.phi[a];
        for (int j = 0; j < 3; ++j) gu[comp][j] += ue[comp * nl + a] * B.dphi[a][j];
      }
  };
  // trial function j: du (value), grad du, dpi
  auto trial = [&](int j, double du[3], double gdu[3][3], double& dpi) {
    for (int i = 0; i < 3; ++i) {
      du[i] = 0.0;
      for (int m = 0; m < 3; ++m) gdu[i][m] = 0.0;
    }
    dpi = 0.0;
    if (j < G.nv) {
      int comp = j / nl, a = j % nl;
      du[comp] = B.phi[a];
      for (int m = 0; m < 3; ++m) gdu[comp][m] = B.dphi[a][m];
    } else {
      dpi = B.psi[j - G.nv];
    }
  };

  for (const QPoint& q : C.vol) {
    point_basis(G, q.r, B);
    double u[3], gu[3][3], A[3][3];
    state_at(u, gu);
    sym_grad(gu, A);
    for (int j = 0; j < ne; ++j) {
      double du[3], gdu[3][3], dpi, Bd[3][3], T[3][3];
      trial(j, du, gdu, dpi);
      sym_grad(gdu, Bd);
      tangent(P, var, A, Bd, T);
      double ddiv = 0.0;
      for (int m = 0; m < G.d; ++m) ddiv += gdu[m][m];
      for (int c = 0; c < 3; ++c) {
        Vf[j * 3 + c] = 0.0;
        for (int m = 0; m < 3; ++m) {
          double g = 0.0;
          if (mask & T_VISC) g += T[c][m];
          if (mask & T_CONV) {
            g -= du[c] * u[m];
            if (var != PIC) g -= u[c] * du[m];
          }
          if ((mask & T_PRES) && c == m) g -= dpi;
          Gf[j * 9 + c * 3 + m] = g;
        }
      }
      Qf[j] = (mask & T_PRES) ? -ddiv : 0.0;
    }
    accumulate(q.w);
  }

  for (int side = 0; side < 2 * G.d; ++side) {
    if (!on_side(G, cp, side)) continue;
    const int axis = side / 2;
    double nrm[3] = {0.0, 0.0, 0.0};
    nrm[axis] = (side % 2) ? 1.0 : -1.0;
    const bool isD = (P.dirichlet_mask >> side) & 1u;
    const double hD = G.h[axis];
    for (const QPoint& q : C.face[side]) {
      point_basis(G, q.r, B);
      double u[3], gu[3][3], A[3][3];
      state_at(u, gu);
      sym_grad(gu, A);
      double un = 0.0;
      for (int m = 0; m < G.d; ++m) un += u[m] * nrm[m];
      Lift L;
      double Dg[3][3] = {}, etaD = 0.0;
      if (isD) {
        lifting_at(C, cp, sd, B, q.r, gnod, L);
        sym_grad(L.grad, Dg);
        etaD = eta_of(P, Dg);
      }
      const double wneg = neg_part(un);
      for (int j = 0; j < ne; ++j) {
        double du[3], gdu[3][3], dpi;
        trial(j, du, gdu, dpi);
        double dun = 0.0;
        for (int m = 0; m < G.d; ++m) dun += du[m] * nrm[m];
        for (int c = 0; c < 3; ++c) {
          double v = 0.0;
          if (mask & T_CONV) {
            v += un * du[c];
            if (var != PIC) v += dun * u[c];
          }
          Vf[j * 3 + c] = v;
          for (int m = 0; m < 3; ++m) Gf[j * 9 + c * 3 + m] = 0.0;
        }
        Qf[j] = 0.0;
        if (isD) {
          double Bd[3][3], T[3][3];
          sym_grad(gdu, Bd);
          tangent(P, var, A, Bd, T);
          for (int c = 0; c < G.d; ++c) {
            double Tn = 0.0;
            for (int m = 0; m < G.d; ++m) Tn += T[c][m] * nrm[m];
            if (mask & T_VFLUX) Vf[j * 3 + c] -= Tn;
            if (mask & T_PRES) Vf[j * 3 + c] += dpi * nrm[c];
            if (mask & T_CONV) Vf[j * 3 + c] -= wneg * du[c];
            if (mask & T_BR) Vf[j * 3 + c] += P.gamma1 / hD * etaD * du[c] + P.gamma2 / hD * dun * nrm[c];
          }
          // -(du, DS(Dg)(Dz) n) = -DS(Dg)(sym(du (x) n)) : grad z   (DS is self-adjoint)
          if (mask & T_BS) {
            double dn[3][3] = {}, Bdn[3][3], DSd[3][3];
            for (int c = 0; c < G.d; ++c)
              for (int m = 0; m < G.d; ++m) dn[c][m] = du[c] * nrm[m];
            sym_grad(dn, Bdn);
            dstress(P, Dg, Bdn, DSd);
            for (int c = 0; c < G.d; ++c)
              for (int m = 0; m < G.d; ++m) Gf[j * 9 + c * 3 + m] -= DSd[c][m];
          }
          if (mask & T_BQ) Qf[j] = P.q_sign * dun;
        }
      }
      accumulate(q.w);
    }
  }
}

void cell_mass(const Ctx& C, int pressure, double* Me) {
  const Geo& G = C.G;
  const int n = pressure ? G.np : G.nv / G.d;
  for (int i = 0; i < n * n; ++i) Me[i] = 0.0;
  PointBasis B;
  for (const QPoint& q : C.vol) {
    point_basis(G, q.r, B);
    const double* b = pressure ? B.psi : B.phi;
    for (int a = 0; a < n; ++a)
      for (int c = 0; c < n; ++c) Me[a * n + c] += q.w * b[a] * b[c];
  }
}

// space-time element matrix, block (mu, nu) of size ne x ne, row = test:
//   vel-vel: K_t[mu][nu] M_e (per component);  plus delta_{mu nu} tau w_mu Je_mu
void cell_st_matrix(const Ctx& C, long cell, int var, const double* U, const double* gnod, int mask, int with_time,
                    double* Jst) {
  const Geo& G = C.G;
  const int K1 = G.k + 1, ne = G.ne, nl = G.nv / G.d, N = K1 * ne;
  long sd[128];
  cell_spatial_dofs(G, cell, sd);
  for (long i = 0; i < (long)N * N; ++i) Jst[i] = 0.0;
  std::vector<double> Je((size_t)ne * ne), ue(G.nv), Me((size_t)nl * nl);
  for (int mu = 0; mu < K1; ++mu) {
    for (int i = 0; i < G.nv; ++i) ue[i] = U[st_index(G, mu, sd[i])];
    cell_spatial_jacobian(C, cell, var, ue.data(), gnod, mask, Je.data());
    const double tw = C.P.dt * C.T.w[mu];
    for (int t = 0; t < ne; ++t)
      for (int j = 0; j < ne; ++j) Jst[(long)(mu * ne + t) * N + mu * ne + j] += tw * Je[t * ne + j];
  }
  if (!with_time) return;
  cell_mass(C, 0, Me.data());
  for (int mu = 0; mu < K1; ++mu)
    for (int nu = 0; nu < K1; ++nu)
      for (int comp = 0; comp < G.d; ++comp)
        for (int a = 0; a < nl; ++a)
          for (int b = 0; b < nl; ++b)
            Jst[(long)(mu * ne + comp * nl + a) * N + nu * ne + comp * nl + b] += C.T.Kt[mu][nu] * Me[a * nl + b];
}

// ------------------------------------------------------------------- CIP
// Convection-aligned CIP term of eq. scip-def on the interior faces F:
//   s(uhat; u, v) = sum_F gamma_cip h_F^2 (|uhat.n_F| [d_n u], [d_n v])_F,
// d_n = derivative along n_F = e_a for the faces normal to axis a, [w] = w on
// the upper cell minus w on the lower cell, h_F the diameter of F (its
// diagonal), 3-point Gauss quadrature per tangential direction.  In the slab
// forms the term is taken at every Radau node with the weight tau w_mu of M_t.
// It is evaluated cell by cell: the jump of the test function is the
// difference of its two one-sided traces, so cell K adds
//   sign_K * weight * [d_n u] * d_n phi_i|K     (sign_K = +1 if K is the
// upper cell of F, -1 if it is the lower one)
// to its own test functions phi_i; the sum over the cells is the face sum.
// Rloc[mu*ne + i] += scale * (that), for u = X; the weight |uhat.n_F| is taken
// from the real field Uhat (the lagged advecting field).
template <class S>
void cell_cip(const Ctx& C, long cell, const S* X, const double* Uhat, double scale, S* Rloc) {
  const Geo& G = C.G;
  const OrParams& P = C.P;
  const int K1 = G.k + 1, nl = G.nv / G.d, ne = G.ne;
  const long cstride[3] = {1, (long)G.n[0], (long)G.n[0] * G.n[1]};
  CellPos cp = cell_pos(G, cell);
  long so[128], sn[128];
  cell_spatial_dofs(G, cell, so);
  for (int side = 0; side < 2 * G.d; ++side) {
    if (on_side(G, cp, side)) continue;  // boundary faces are not in the interior skeleton
    const int a = side / 2, up = side % 2;
    const long nb = up ? cell + cstride[a] : cell - cstride[a];
    cell_spatial_dofs(G, nb, sn);
    double hF2 = 0.0;
    for (int b = 0; b < G.d; ++b)
      if (b != a) hF2 += G.h[b] * G.h[b];
    const double signK = up ? -1.0 : 1.0;
    for (const QPoint& q : C.face[side]) {
      double rn[3] = {q.r[0], q.r[1], q.r[2]};
      rn[a] = up ? 0.0 : 1.0;  // the same point seen from the neighbour
      PointBasis Bo, Bn;
      point_basis(G, q.r, Bo);
      point_basis(G, rn, Bn);
      for (int mu = 0; mu < K1; ++mu) {
        double un = 0.0;
        for (int i = 0; i < nl; ++i) un += Uhat[st_index(G, mu, so[a * nl + i])] * Bo.phi[i];
        const double w = P.gamma_cip * hF2 * std::fabs(un) * q.w * P.dt * C.T.w[mu];
        for (int comp = 0; comp < G.d; ++comp) {
          S dn_own = 0.0, dn_nb = 0.0;
          for (int i = 0; i < nl; ++i) {
            dn_own += X[st_index(G, mu, so[comp * nl + i])] * Bo.dphi[i][a];
            dn_nb += X[st_index(G, mu, sn[comp * nl + i])] * Bn.dphi[i][a];
          }
          const S jump = up ? (dn_nb - dn_own) : (dn_own - dn_nb);
          for (int i = 0; i < nl; ++i) Rloc[mu * ne + comp * nl + i] += scale * signK * w * jump * Bo.dphi[i][a];
        }
      }
    }
  }
}

std::vector<long> cell_list(const Geo& G, long ncells, const long* cells) {
  std::vector<long> v;
  if (cells) {
    v.assign(cells, cells + ncells);
  } else {
    v.resize(G.ncells);
    for (long c = 0; c < G.ncells; ++c) v[c] = c;
  }
  return v;
}

int num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // namespace

// ================================================================ C ABI
extern "C" {

int or_num_threads() { return num_threads(); }

// Radau nodes t[k+1], weights w[k+1], K_t, m_t, reference M_t (row-major)
int or_time_tables(int k, double* t, double* w, double* Kt, double* mt, double* Mt) {
  if (k < 0 || k > 6) return 1;
  TimeTables T;
  time_tables(k, T);
  for (int i = 0; i <= k; ++i) {
    t[i] = T.t[i];
    w[i] = T.w[i];
    mt[i] = T.mt[i];
    for (int j = 0; j <= k; ++j) {
      Kt[i * (k + 1) + j] = T.Kt[i][j];
      Mt[i * (k + 1) + j] = T.Mt[i][j];
    }
  }
  return 0;
}

int or_gauss01(int n, double* x, double* w) {
  if (n < 1 || n > 32) return 1;
  gauss01(n, x, w);
  return 0;
}

// sizes: out[0..7] = Nq2, Nq1, Mv, Mp, Nst, ne, nv, ncells
int or_sizes(const OrParams* P, long* out) {
  Geo G = make_geo(*P);
  out[0] = G.Nq2;
  out[1] = G.Nq1;
  out[2] = G.Mv;
  out[3] = G.Mp;
  out[4] = G.Nst;
  out[5] = G.ne;
  out[6] = G.nv;
  out[7] = G.ncells;
  return 0;
}

// space-time dofs of cells: out[c*(k+1)*ne + mu*ne + i]
int or_cell_dofs(const OrParams* P, long ncells, const long* cells, long* out) {
  Geo G = make_geo(*P);
  long sd[128];
  const int K1 = G.k + 1;
  for (long c = 0; c < ncells; ++c) {
    cell_spatial_dofs(G, cells[c], sd);
    for (int mu = 0; mu < K1; ++mu)
      for (int i = 0; i < G.ne; ++i) out[(c * K1 + mu) * G.ne + i] = st_index(G, mu, sd[i]);
  }
  return 0;
}

// spatial dofs (one time node block, velocity then pressure) of cells
int or_cell_spatial_dofs(const OrParams* P, long ncells, const long* cells, long* out) {
  Geo G = make_geo(*P);
  for (long c = 0; c < ncells; ++c) cell_spatial_dofs(G, cells[c], out + c * G.ne);
  return 0;
}

// Pointwise constitutive maps on 3x3 row-major matrices.
// which: 0 = S(A), 1 = DS(A)(B), 2 = tangent(var)(A)(B), 3 = eta(A) (out[0])
int or_pointwise(const OrParams* P, int which, int var, const double* A9, const double* B9, double* out9) {
  double A[3][3], B[3][3], R[3][3];
  for (int i = 0; i < 9; ++i) {
    A[i / 3][i % 3] = A9[i];
    B[i / 3][i % 3] = B9 ? B9[i] : 0.0;
  }
  if (which == 0) stress(*P, A, R);
  else if (which == 1) dstress(*P, A, B, R);
  else if (which == 2) tangent(*P, var, A, B, R);
  else if (which == 3) {
    out9[0] = eta_of(*P, A);
    return 0;
  } else return 1;
  for (int i = 0; i < 9; ++i) out9[i] = R[i / 3][i % 3];
  return 0;
}

// Residual R_n (accumulated into R, which the caller zeroes) over the given
// cells (cells == NULL: all).  f, vprev, gnod may be NULL.
int or_residual(const OrParams* P, const double* U, const double* vprev, const double* f, const double* gnod,
                long ncells, const long* cells, double* R) {
  Ctx C;
  make_ctx(P, C);
  std::vector<long> cl = cell_list(C.G, ncells, cells);
  const int K1 = C.G.k + 1, ne = C.G.ne;
  std::vector<double> loc((size_t)cl.size() * K1 * ne);
#pragma omp parallel for schedule(dynamic, 16)
  for (long c = 0; c < (long)cl.size(); ++c) {
    cell_residual<double>(C, cl[c], U, vprev, f, gnod, &loc[c * K1 * ne]);
    if (P->gamma_cip > 0.0) cell_cip<double>(C, cl[c], U, U, -1.0, &loc[c * K1 * ne]);  // part of the left side
  }
  long sd[128];
  for (size_t c = 0; c < cl.size(); ++c) {
    cell_spatial_dofs(C.G, cl[c], sd);
    for (int mu = 0; mu < K1; ++mu)
      for (int i = 0; i < ne; ++i) R[st_index(C.G, mu, sd[i])] += loc[(c * K1 + mu) * ne + i];
  }
  return 0;
}

// Complex-step residual: Rim = Im R(U + i h dU) / h (the inflow factor is
// frozen at Re(u.n), the CIP weight at Re(u)).  Accumulates into Rim.
int or_residual_cs(const OrParams* P, const double* U, const double* dU, double h, const double* vprev,
                   const double* f, const double* gnod, long ncells, const long* cells, double* Rim) {
  typedef std::complex<double> Z;
  Ctx C;
  make_ctx(P, C);
  std::vector<long> cl = cell_list(C.G, ncells, cells);
  const int K1 = C.G.k + 1, ne = C.G.ne;
  std::vector<Z> Uz(C.G.Nst);
  for (long i = 0; i < C.G.Nst; ++i) Uz[i] = Z(U[i], h * dU[i]);
  std::vector<Z> loc((size_t)cl.size() * K1 * ne);
#pragma omp parallel for schedule(dynamic, 16)
  for (long c = 0; c < (long)cl.size(); ++c) {
    cell_residual<Z>(C, cl[c], Uz.data(), vprev, f, gnod, &loc[c * K1 * ne]);
    if (P->gamma_cip > 0.0) cell_cip<Z>(C, cl[c], Uz.data(), U, -1.0, &loc[c * K1 * ne]);
  }
  long sd[128];
  for (size_t c = 0; c < cl.size(); ++c) {
    cell_spatial_dofs(C.G, cl[c], sd);
    for (int mu = 0; mu < K1; ++mu)
      for (int i = 0; i < ne; ++i) Rim[st_index(C.G, mu, sd[i])] += loc[(c * K1 + mu) * ne + i].imag() / h;
  }
  return 0;
}

// Space-time element matrices (row = test) for the given cells:
// out[c * N * N], N = (k+1) ne, dof order of or_cell_dofs.
int or_st_element_matrices(const OrParams* P, int var, const double* U, const double* gnod, int mask, int with_time,
                           long ncells, const long* cells, double* out) {
  Ctx C;
  make_ctx(P, C);
  const long N = (long)(C.G.k + 1) * C.G.ne;
#pragma omp parallel for schedule(dynamic, 4)
  for (long c = 0; c < ncells; ++c) cell_st_matrix(C, cells[c], var, U, gnod, mask, with_time, out + c * N * N);
  return 0;
}

// Spatial element matrices at one time node for a velocity field u (d*Nq2
// values, component-major): out[c * ne * ne].
int or_spatial_element_matrices(const OrParams* P, int var, const double* u, const double* gnod, int mask,
                                long ncells, const long* cells, double* out) {
  Ctx C;
  make_ctx(P, C);
  const int ne = C.G.ne;
#pragma omp parallel for schedule(dynamic, 4)
  for (long c = 0; c < ncells; ++c) {
    long sd[128];
    cell_spatial_dofs(C.G, cells[c], sd);
    std::vector<double> ue(C.G.nv);
    for (int i = 0; i < C.G.nv; ++i) ue[i] = u[sd[i]];
    cell_spatial_jacobian(C, cells[c], var, ue.data(), gnod, mask, out + c * (long)ne * ne);
  }
  return 0;
}

// element mass matrix of one scalar Q2 (pressure = 0) or Q1 (pressure = 1)
// field on a cell (all cells of a uniform mesh share it)
int or_element_mass(const OrParams* P, int pressure, double* out) {
  Ctx C;
  make_ctx(P, C);
  cell_mass(C, pressure, out);
  return 0;
}

// Jacobian action out += J_n(U) dU over the given cells (cells == NULL: all),
// by forming each cell's space-time element matrix and multiplying, plus the
// CIP term with its weight lagged at U (Sec. 4.2-4.4) when gamma_cip > 0.
int or_jacobian_apply(const OrParams* P, int var, const double* U, const double* dU, long ncells, const long* cells,
                      double* out) {
  Ctx C;
  make_ctx(P, C);
  std::vector<long> cl = cell_list(C.G, ncells, cells);
  const int K1 = C.G.k + 1, ne = C.G.ne;
  const long N = (long)K1 * ne;
  std::vector<double> loc((size_t)cl.size() * N);
#pragma omp parallel
  {
    std::vector<double> Jst((size_t)N * N), xe(N);
    std::vector<long> dofs(N);
#pragma omp for schedule(dynamic, 4)
    for (long c = 0; c < (long)cl.size(); ++c) {
      long sd[128];
      cell_spatial_dofs(C.G, cl[c], sd);
      for (int mu = 0; mu < K1; ++mu)
        for (int i = 0; i < ne; ++i) dofs[mu * ne + i] = st_index(C.G, mu, sd[i]);
      cell_st_matrix(C, cl[c], var, U, nullptr, T_ALL, 1, Jst.data());
      for (long i = 0; i < N; ++i) xe[i] = dU[dofs[i]];
      for (long i = 0; i < N; ++i) {
        double s = 0.0;
        for (long j = 0; j < N; ++j) s += Jst[i * N + j] * xe[j];
        loc[c * N + i] = s;
      }
      if (P->gamma_cip > 0.0) cell_cip<double>(C, cl[c], dU, U, 1.0, &loc[c * N]);
    }
  }
  long sd[128];
  for (size_t c = 0; c < cl.size(); ++c) {
    cell_spatial_dofs(C.G, cl[c], sd);
    for (int mu = 0; mu < K1; ++mu)
      for (int i = 0; i < ne; ++i) out[st_index(C.G, mu, sd[i])] += loc[c * N + mu * ne + i];
  }
  return 0;
}

// CIP matrix of the slab (lagged weight at U) as dense blocks, one per
// (cell, side, mu, comp) in that order: rows = the cell's own Q2 nodes of
// component comp at node mu (nl slab indices), cols = own then neighbour
// nodes (2 nl), vals[nl][2 nl].  Sides on the boundary give zero blocks (the
// neighbour columns then repeat the own ones).  The same evaluation as
// cell_cip with the jump expanded in the nodal values.
int or_cip_blocks(const OrParams* P, const double* U, long* rows, long* cols, double* vals) {
  Ctx C;
  make_ctx(P, C);
  const Geo& G = C.G;
  const int K1 = G.k + 1, nl = G.nv / G.d, d = G.d;
  const long cstride[3] = {1, (long)G.n[0], (long)G.n[0] * G.n[1]};
#pragma omp parallel for schedule(dynamic, 4)
  for (long cell = 0; cell < G.ncells; ++cell) {
    CellPos cp = cell_pos(G, cell);
    long so[128], sn[128];
    cell_spatial_dofs(G, cell, so);
    for (int side = 0; side < 2 * d; ++side) {
      const bool interior = !on_side(G, cp, side);
      const int a = side / 2, up = side % 2;
      const long nb = !interior ? cell : (up ? cell + cstride[a] : cell - cstride[a]);
      cell_spatial_dofs(G, nb, sn);
      double hF2 = 0.0;
      for (int b = 0; b < d; ++b)
        if (b != a) hF2 += G.h[b] * G.h[b];
      const double signK = up ? -1.0 : 1.0;
      for (int mu = 0; mu < K1; ++mu)
        for (int comp = 0; comp < d; ++comp) {
          const long blk = ((cell * 2 * d + side) * K1 + mu) * d + comp;
          long* r = rows + blk * nl;
          long* cc = cols + blk * 2 * nl;
          double* v = vals + blk * 2 * nl * nl;
          for (int i = 0; i < nl; ++i) {
            r[i] = st_index(G, mu, so[comp * nl + i]);
            cc[i] = r[i];
            cc[nl + i] = st_index(G, mu, sn[comp * nl + i]);
          }
          for (int i = 0; i < 2 * nl * nl; ++i) v[i] = 0.0;
          if (!interior) continue;
          for (const QPoint& q : C.face[side]) {
            double rn[3] = {q.r[0], q.r[1], q.r[2]};
            rn[a] = up ? 0.0 : 1.0;
            PointBasis Bo, Bn;
            point_basis(G, q.r, Bo);
            point_basis(G, rn, Bn);
            double un = 0.0;
            for (int i = 0; i < nl; ++i) un += U[st_index(G, mu, so[a * nl + i])] * Bo.phi[i];
            const double w = P->gamma_cip * hF2 * std::fabs(un) * q.w * P->dt * C.T.w[mu];
            // [d_n u] = sum_j jo[j] u_own[j] + jn[j] u_nb[j]
            for (int i = 0; i < nl; ++i)
              for (int j = 0; j < nl; ++j) {
                const double jo = up ? -Bo.dphi[j][a] : Bo.dphi[j][a];
                const double jn = up ? Bn.dphi[j][a] : -Bn.dphi[j][a];
                v[i * 2 * nl + j] += signK * w * Bo.dphi[i][a] * jo;
                v[i * 2 * nl + nl + j] += signK * w * Bo.dphi[i][a] * jn;
              }
          }
        }
    }
  }
  return 0;
}

// Squared L2(I_n; L2(Omega)) norm of div u over the slab, by the cell Gauss
// rule in space and the Radau rule in time: sum_mu tau w_mu (div u_mu, div u_mu)
// (the divergence error of Table conv-pns; the exact velocity is solenoidal).
double or_div_norm2(const OrParams* P, const double* U) {
  Ctx C;
  make_ctx(P, C);
  const Geo& G = C.G;
  const int K1 = G.k + 1, nl = G.nv / G.d;
  double total = 0.0;
  long sd[128];
  for (long cell = 0; cell < G.ncells; ++cell) {
    cell_spatial_dofs(G, cell, sd);
    for (const QPoint& q : C.vol) {
      PointBasis B;
      point_basis(G, q.r, B);
      for (int mu = 0; mu < K1; ++mu) {
        double dv = 0.0;
        for (int comp = 0; comp < G.d; ++comp)
          for (int i = 0; i < nl; ++i) dv += U[st_index(G, mu, sd[comp * nl + i])] * B.dphi[i][comp];
        total += P->dt * C.T.w[mu] * q.w * dv * dv;
      }
    }
  }
  return total;
}

// Block mass-weighted squared norm (Sec. 6.1), literal reading:
//   r_v^T (M_t (x) M_x) r_v + r_p^T (M_t (x) M_{x,p}) r_p,  M_t = tau diag(w)
double or_mnorm2(const OrParams* P, const double* r) {
  Ctx C;
  make_ctx(P, C);
  const Geo& G = C.G;
  const int K1 = G.k + 1, nl = G.nv / G.d;
  std::vector<double> Mv((size_t)nl * nl), Mp((size_t)G.np * G.np);
  cell_mass(C, 0, Mv.data());
  cell_mass(C, 1, Mp.data());
  double total = 0.0;
  long sd[128];
  for (long cell = 0; cell < G.ncells; ++cell) {
    cell_spatial_dofs(G, cell, sd);
    for (int mu = 0; mu < K1; ++mu) {
      double s = 0.0;
      for (int comp = 0; comp < G.d; ++comp)
        for (int a = 0; a < nl; ++a)
          for (int b = 0; b < nl; ++b)
            s += r[st_index(G, mu, sd[comp * nl + a])] * Mv[a * nl + b] * r[st_index(G, mu, sd[comp * nl + b])];
      for (int a = 0; a < G.np; ++a)
        for (int b = 0; b < G.np; ++b)
          s += r[st_index(G, mu, sd[G.nv + a])] * Mp[a * G.np + b] * r[st_index(G, mu, sd[G.nv + b])];
      total += P->dt * C.T.w[mu] * s;
    }
  }
  return total;
}

}  // extern "C"
