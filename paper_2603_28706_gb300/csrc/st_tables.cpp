// Reference tables of the discretisation, computed on the host.
//
// Space: Q2 Lagrange basis on the nodes {0, 1/2, 1} and Q1 on {0, 1} of the
// unit interval, 3-point Gauss rule (closed form).  Time: right-sided
// (k+1)-point Gauss-Radau nodes of Sec. 3.1 (Rem. 3.2): t = 1 and the zeros
// of the Jacobi polynomial P_k^{(1,0)} mapped from [-1,1]; weights from the
// moment equations; the temporal matrices K_t, m_t of Sec. 5.2 from the
// monomial coefficients of the Lagrange basis.

#include <cmath>
#include <complex>

#include "st_internal.h"

namespace st {

namespace {

// Q2 basis on {0, 1/2, 1}: L0 = (2x-1)(x-1), L1 = 4x(1-x), L2 = x(2x-1)
double q2(int a, double x) {
  switch (a) {
    case 0: return (2.0 * x - 1.0) * (x - 1.0);
    case 1: return 4.0 * x * (1.0 - x);
    default: return x * (2.0 * x - 1.0);
  }
}
double q2d(int a, double x) {
  switch (a) {
    case 0: return 4.0 * x - 3.0;
    case 1: return 4.0 - 8.0 * x;
    default: return 4.0 * x - 1.0;
  }
}

// Jacobi polynomial P_n^{(1,0)}(s) by its three-term recurrence
double jacobi10(int n, double s) {
  const double a = 1.0, b = 0.0;
  if (n == 0) return 1.0;
  double p0 = 1.0;
  double p1 = 0.5 * (a - b) + 0.5 * (a + b + 2.0) * s;
  for (int m = 2; m <= n; ++m) {
    double c = 2.0 * m + a + b;
    double a1 = 2.0 * m * (m + a + b) * (c - 2.0);
    double a2 = (c - 1.0) * (a * a - b * b);
    double a3 = (c - 2.0) * (c - 1.0) * c;
    double a4 = 2.0 * (m + a - 1.0) * (m + b - 1.0) * c;
    double p2 = ((a2 + a3 * s) * p1 - a4 * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// Solve the dense system A x = b (n <= 8) by Gaussian elimination with pivoting.
bool solve_small(int n, double* A, double* b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    if (piv != c) {
      for (int j = 0; j < n; ++j) std::swap(A[c * n + j], A[piv * n + j]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int j = r + 1; j < n; ++j) s -= A[r * n + j] * b[j];
    b[r] = s / A[r * n + r];
  }
  return true;
}

}  // namespace

void make_ref_tables(RefTables& R) {
  const double g[3] = {0.5 - std::sqrt(15.0) / 10.0, 0.5, 0.5 + std::sqrt(15.0) / 10.0};
  R.W[0] = 5.0 / 18.0;
  R.W[1] = 8.0 / 18.0;
  R.W[2] = 5.0 / 18.0;
  for (int q = 0; q < 3; ++q)
    for (int a = 0; a < 3; ++a) {
      R.B[q * 3 + a] = q2(a, g[q]);
      R.Bt[a * 3 + q] = q2(a, g[q]);
    }
  // derivative at g[q] of the Lagrange polynomial through the Gauss points
  // that is one at g[j]
  for (int q = 0; q < 3; ++q)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int m = 0; m < 3; ++m) {
        if (m == j) continue;
        double r = 1.0 / (g[j] - g[m]);
        for (int l = 0; l < 3; ++l)
          if (l != j && l != m) r *= (g[q] - g[l]) / (g[j] - g[l]);
        s += r;
      }
      R.Dc[q * 3 + j] = s;
    }
  // The Gauss points are symmetric about 1/2, so B is centro-symmetric and Dc
  // centro-antisymmetric (zero centre entry) in exact arithmetic; impose both
  // exactly (the kernels use the symmetry to skip work)
  for (int i = 0; i < 4; ++i) {
    const double b = 0.5 * (R.B[i] + R.B[8 - i]);
    R.B[i] = R.B[8 - i] = b;
    const double d = 0.5 * (R.Dc[i] - R.Dc[8 - i]);
    R.Dc[i] = d;
    R.Dc[8 - i] = -d;
  }
  R.Dc[4] = 0.0;
  for (int q = 0; q < 3; ++q)
    for (int a = 0; a < 3; ++a) R.Bt[a * 3 + q] = R.B[q * 3 + a];
  for (int q = 0; q < 3; ++q) {
    R.B1[q * 2 + 0] = 1.0 - g[q];
    R.B1[q * 2 + 1] = g[q];
  }
  for (int e = 0; e < 2; ++e)
    for (int a = 0; a < 3; ++a) {
      R.E[e * 3 + a] = q2(a, (double)e);
      R.ED[e * 3 + a] = q2d(a, (double)e);
    }
  // exact 1D Q2 mass matrix on [0,1]
  const double M[9] = {2.0 / 15, 1.0 / 15, -1.0 / 30, 1.0 / 15, 8.0 / 15, 1.0 / 15, -1.0 / 30, 1.0 / 15, 2.0 / 15};
  for (int i = 0; i < 9; ++i) R.M1[i] = M[i];
  // nested prolongation: fine nodes x = i/4 of the coarse cell
  for (int i = 0; i < 5; ++i)
    for (int a = 0; a < 3; ++a) R.P2[i * 3 + a] = q2(a, 0.25 * i);
  for (int i = 0; i < 3; ++i) {
    R.P1[i * 2 + 0] = 1.0 - 0.5 * i;
    R.P1[i * 2 + 1] = 0.5 * i;
  }
}

bool make_time_tables(int k, TimeTab& T) {
  if (k < 0 || k >= MAX_K1) return false;
  const int n = k + 1;
  T.k = k;
  // interior right-Radau nodes: zeros of P_k^{(1,0)} on (-1,1); Newton from
  // Chebyshev-Gauss guesses with deflation by the roots already found
  double s[MAX_K1];
  for (int i = 0; i < k; ++i) {
    double x = -std::cos(M_PI * (2.0 * i + 1.0) / (2.0 * k));
    for (int it = 0; it < 200; ++it) {
      const double hh = 1e-7;
      double f = jacobi10(k, x);
      double df = (jacobi10(k, x + hh) - jacobi10(k, x - hh)) / (2.0 * hh);
      double defl = 0.0;
      for (int j = 0; j < i; ++j) defl += 1.0 / (x - s[j]);
      double dx = f / (df - f * defl);
      x -= dx;
      if (std::fabs(dx) < 1e-15) break;
    }
    s[i] = x;
  }
  for (int i = 0; i < k; ++i)
    for (int j = i + 1; j < k; ++j)
      if (s[j] < s[i]) std::swap(s[i], s[j]);
  for (int i = 0; i < k; ++i) T.t[i] = 0.5 * (s[i] + 1.0);
  T.t[k] = 1.0;
  // weights: sum_i w_i t_i^m = 1/(m+1), m = 0..k
  double V[MAX_K1 * MAX_K1], b[MAX_K1];
  for (int m = 0; m < n; ++m) {
    for (int i = 0; i < n; ++i) V[m * n + i] = std::pow(T.t[i], m);
    b[m] = 1.0 / (m + 1.0);
  }
  if (!solve_small(n, V, b)) return false;
  for (int i = 0; i < n; ++i) T.w[i] = b[i];
  // monomial coefficients c[i][m] of the Lagrange basis: sum_m c[i][m] t_j^m = delta_ij
  double C[MAX_K1][MAX_K1];
  for (int i = 0; i < n; ++i) {
    double A[MAX_K1 * MAX_K1], rhs[MAX_K1];
    for (int j = 0; j < n; ++j) {
      for (int m = 0; m < n; ++m) A[j * n + m] = std::pow(T.t[j], m);
      rhs[j] = (i == j) ? 1.0 : 0.0;
    }
    if (!solve_small(n, A, rhs)) return false;
    for (int m = 0; m < n; ++m) C[i][m] = rhs[m];
  }
  // (K_t)_ij = int_0^1 xi_j' xi_i dt + xi_j(0) xi_i(0);  (m_t)_i = xi_i(0)
  for (int i = 0; i < n; ++i) {
    T.mt[i] = C[i][0];
    double lr = 0.0;
    for (int m = 0; m < n; ++m) lr += C[i][m] * std::pow(0.5, m);
    T.lrep[i] = lr;
    for (int j = 0; j < n; ++j) {
      double v = 0.0;
      for (int m = 1; m < n; ++m)
        for (int l = 0; l < n; ++l) v += C[j][m] * m * C[i][l] / (double)(m + l);
      T.Kt[i * n + j] = v + C[j][0] * C[i][0];
    }
  }
  return true;
}


// ---------------------------------------------------------------------
// Eigen-decomposition of B = W^{-1} K_t (K1 <= 4, real, non-symmetric):
// characteristic polynomial by the Faddeev-LeVerrier recursion, its roots by
// the Durand-Kerner (Weierstrass) iteration, eigenvectors as null vectors of
// B - lambda I (complex elimination with full pivoting), X^{-1} by
// Gauss-Jordan; checked by |X diag(lambda) X^{-1} - B| <= 1e-10 |B|.
namespace {

using cd = std::complex<double>;

bool cinvert(int n, cd A[MAX_K1][MAX_K1], cd Ai[MAX_K1][MAX_K1]) {
  cd M[MAX_K1][2 * MAX_K1];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) M[i][j] = j < n ? A[i][j] : cd(i == j - n ? 1.0 : 0.0);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::abs(M[i][k]) > std::abs(M[p][k])) p = i;
    if (std::abs(M[p][k]) == 0.0) return false;
    for (int j = 0; j < 2 * n; ++j) std::swap(M[k][j], M[p][j]);
    const cd d = M[k][k];
    for (int j = 0; j < 2 * n; ++j) M[k][j] /= d;
    for (int i = 0; i < n; ++i)
      if (i != k) {
        const cd f = M[i][k];
        for (int j = 0; j < 2 * n; ++j) M[i][j] -= f * M[k][j];
      }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ai[i][j] = M[i][j + n];
  return true;
}

// a null vector of the n x n matrix A (rank n - 1), largest entry 1
void null_vector(int n, cd A[MAX_K1][MAX_K1], cd v[MAX_K1]) {
  cd M[MAX_K1][MAX_K1];
  int col[MAX_K1];
  for (int i = 0; i < n; ++i) {
    col[i] = i;
    for (int j = 0; j < n; ++j) M[i][j] = A[i][j];
  }
  for (int k = 0; k < n - 1; ++k) {  // full pivoting on the leading n-1 steps
    int pi = k, pj = k;
    for (int i = k; i < n; ++i)
      for (int j = k; j < n; ++j)
        if (std::abs(M[i][j]) > std::abs(M[pi][pj])) {
          pi = i;
          pj = j;
        }
    for (int j = 0; j < n; ++j) std::swap(M[k][j], M[pi][j]);
    for (int i = 0; i < n; ++i) std::swap(M[i][k], M[i][pj]);
    std::swap(col[k], col[pj]);
    for (int i = k + 1; i < n; ++i) {
      const cd f = M[i][k] / M[k][k];
      for (int j = k; j < n; ++j) M[i][j] -= f * M[k][j];
    }
  }
  cd y[MAX_K1];
  y[n - 1] = 1.0;
  for (int k = n - 2; k >= 0; --k) {
    cd acc = 0.0;
    for (int j = k + 1; j < n; ++j) acc += M[k][j] * y[j];
    y[k] = -acc / M[k][k];
  }
  double big = 0.0;
  int ib = 0;
  for (int i = 0; i < n; ++i) {
    v[col[i]] = y[i];
  }
  for (int i = 0; i < n; ++i)
    if (std::abs(v[i]) > big) {
      big = std::abs(v[i]);
      ib = i;
    }
  const cd s = v[ib];
  for (int i = 0; i < n; ++i) v[i] /= s;
}

}  // namespace

bool make_time_eig(const TimeTab& T, TimeEig& out) {
  const int n = T.k + 1;
  double B[MAX_K1][MAX_K1];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) B[i][j] = T.Kt[i * n + j] * T.w[0] / T.w[i];
  // characteristic polynomial lambda^n + c[n-1] lambda^{n-1} + .. + c[0]
  double c[MAX_K1 + 1];
  {
    double Mk[MAX_K1][MAX_K1] = {}, AM[MAX_K1][MAX_K1];
    c[n] = 1.0;
    for (int k = 1; k <= n; ++k) {
      // M_k = B M_{k-1} + c_{n-k+1} I, c_{n-k} = -tr(B M_k) / k
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          double acc = 0.0;
          for (int l = 0; l < n; ++l) acc += B[i][l] * Mk[l][j];
          AM[i][j] = acc + (i == j ? c[n - k + 1] : 0.0);
        }
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Mk[i][j] = AM[i][j];
      double tr = 0.0;
      for (int i = 0; i < n; ++i)
        for (int l = 0; l < n; ++l) tr += B[i][l] * Mk[l][i];
      c[n - k] = -tr / k;
    }
  }
  cd z[MAX_K1];
  for (int i = 0; i < n; ++i) z[i] = std::pow(cd(0.4, 0.9), i) * 2.0;
  for (int it = 0; it < 500; ++it) {
    double moved = 0.0;
    for (int i = 0; i < n; ++i) {
      cd pv = 1.0;
      for (int k = n - 1; k >= 0; --k) pv = pv * z[i] + c[k];
      cd den = 1.0;
      for (int j = 0; j < n; ++j)
        if (j != i) den *= (z[i] - z[j]);
      const cd dz = pv / den;
      z[i] -= dz;
      moved = std::max(moved, std::abs(dz));
    }
    if (moved < 1e-15) break;
  }
  double bn = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) bn = std::max(bn, std::fabs(B[i][j]));
  // order: real eigenvalues first, then each pair as (im > 0, conjugate)
  cd lam[MAX_K1];
  int cnt = 0;
  bool used[MAX_K1] = {};
  for (int i = 0; i < n; ++i)
    if (std::fabs(z[i].imag()) <= 1e-10 * bn) {
      lam[cnt++] = cd(z[i].real(), 0.0);
      used[i] = true;
    }
  const int nreal = cnt;
  for (int i = 0; i < n; ++i)
    if (!used[i] && z[i].imag() > 0.0) {
      lam[cnt++] = z[i];
      lam[cnt++] = std::conj(z[i]);
    }
  if (cnt != n) return false;
  cd X[MAX_K1][MAX_K1], Xi[MAX_K1][MAX_K1];
  for (int e = 0; e < n; ++e) {
    cd A[MAX_K1][MAX_K1], v[MAX_K1];
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) A[i][j] = cd(B[i][j]) - (i == j ? lam[e] : cd(0.0));
    null_vector(n, A, v);
    if (e < nreal)
      for (int i = 0; i < n; ++i) v[i] = cd(v[i].real(), 0.0);
    if (e >= nreal && ((e - nreal) & 1))  // the conjugate of the previous one
      for (int i = 0; i < n; ++i) v[i] = std::conj(X[i][e - 1]);
    for (int i = 0; i < n; ++i) X[i][e] = v[i];
  }
  if (!cinvert(n, X, Xi)) return false;
  double err = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      cd acc = 0.0;
      for (int e = 0; e < n; ++e) acc += X[i][e] * lam[e] * Xi[e][j];
      err = std::max(err, std::abs(acc - B[i][j]));
    }
  if (!(err <= 1e-10 * (bn > 0 ? bn : 1.0))) return false;
  out.nb = 0;
  for (int e = 0; e < n; ++e) {
    const bool pair = e >= nreal;
    if (pair && ((e - nreal) & 1)) continue;  // kept: the first of a pair
    const int b = out.nb++;
    out.lam[b][0] = lam[e].real();
    out.lam[b][1] = lam[e].imag();
    for (int mu = 0; mu < n; ++mu) {
      const cd ti = Xi[e][mu] * (T.w[0] / T.w[mu]);  // X^{-1} W^{-1}
      const cd to = X[mu][e] * (pair ? 2.0 : 1.0);
      out.tin[b][mu][0] = ti.real();
      out.tin[b][mu][1] = ti.imag();
      out.tout[b][mu][0] = to.real();
      out.tout[b][mu][1] = to.imag();
    }
  }
  return true;
}

}  // namespace st
