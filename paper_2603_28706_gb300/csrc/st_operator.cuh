// Matrix-free space-time slab operator kernels (sm_103a).
//
// One kernel template computes, for the cells of one colour class (the 2^d
// parity classes of the cell grid; cells of one class share no node, so the
// scatter-add needs no atomics):
//   OP_LIN: the FP64 coefficient cache of the linearisation at the iterate
//           (Sec. 4.1: A^m, Delta^{m,2}, mu^m, eta^m and the tangent's rank-one
//           factor: 0 for Pic, (p-2) mu/Delta^2 for exN, s (p-2) mu/Delta^2 for
//           modN, eq. local-tangent-picard/-exact/-clip), at every cell
//           quadrature point and boundary-face point and every Radau node;
//   OP_JAC: out += J_n(U) dU (eq. slab-underint-jac) from that cache;
//   OP_RES: out += R_n(U) (eq. slab-underint, eq. disc, def-a-gam, def-b-gam).
//
// Work decomposition: a CTA owns a contiguous, balanced chunk of the colour
// class and processes it in batches of C cells.  A batch holds C*(k+1)
// "slots" (cell, Radau node) in shared memory.  Every stage of the
// sum-factorised evaluation is a flat list of independent items (one 3-point
// line of a slot, or one quadrature point of a slot) spread over all threads,
// so all lanes carry work; stages are separated by __syncthreads.
//   gather -> 3 value passes (Q2 basis at Gauss points) -> derivative passes
//   in collocation form -> pointwise flux at every quadrature point ->
//   transposed derivative chain -> 3 transposed value passes -> boundary faces
//   (in rounds, one face per slot per round) -> scatter-add.
#pragma once

#include <cuda_runtime.h>

#include "st_internal.h"

namespace st {

// mesh-independent reference tables in constant memory (double and float)
struct ConstTables {
  double B[9], Bt[9], Dc[9], W[3], B1[6], E[6], ED[6];
  double WQ3[27], WQ2[9];    // tensor Gauss weights on the unit cell
  double PSI3[27 * 8], PSI2[9 * 4];  // Q1 basis at the cell Gauss points
  double FW3[9], FW2[3];     // tensor Gauss weights on a unit face
  double FPSI3[9 * 4], FPSI2[3 * 2]; // face Q1 basis at face points
};
struct ConstTablesF {
  float B[9], Bt[9], Dc[9], W[3], B1[6], E[6], ED[6];
  float WQ3[27], WQ2[9];
  float PSI3[27 * 8], PSI2[9 * 4];
  float FW3[9], FW2[3];
  float FPSI3[9 * 4], FPSI2[3 * 2];
};

// one copy per translation unit (no relocatable device code needed)
static __constant__ ConstTables cT;
static __constant__ ConstTablesF cTf;

template <typename T> struct CT;
template <> struct CT<double> {
  static __device__ __forceinline__ const ConstTables& t() { return cT; }
};
template <> struct CT<float> {
  static __device__ __forceinline__ const ConstTablesF& t() { return cTf; }
};

// index of the first node of line l along direction dir of a 3^DIM block
template <int DIM>
__device__ __forceinline__ void line_idx(int dir, int l, int& base, int& stride) {
  if (DIM == 2) {
    if (dir == 0) { base = 3 * l; stride = 1; }
    else { base = l; stride = 3; }
  } else {
    if (dir == 0) { base = 3 * l; stride = 1; }
    else if (dir == 1) { base = (l % 3) + 9 * (l / 3); stride = 3; }
    else { base = l; stride = 9; }
  }
}

// y = M x along a line (M row-major 3x3 of type T or double)
template <typename T, typename M>
__device__ __forceinline__ void apply3(const M* m, T x0, T x1, T x2, T& y0, T& y1, T& y2) {
  y0 = (T)m[0] * x0 + (T)m[1] * x1 + (T)m[2] * x2;
  y1 = (T)m[3] * x0 + (T)m[4] * x1 + (T)m[5] * x2;
  y2 = (T)m[6] * x0 + (T)m[7] * x1 + (T)m[8] * x2;
}

template <int DIM, typename T>
__device__ __forceinline__ void line_pass(T* arr, int dir, int l, const T* m, T* dst) {
  int b, s;
  line_idx<DIM>(dir, l, b, s);
  T y0, y1, y2;
  apply3<T, T>(m, arr[b], arr[b + s], arr[b + 2 * s], y0, y1, y2);
  dst[b] = y0;
  dst[b + s] = y1;
  dst[b + 2 * s] = y2;
}

// dst = acc + M x along a line
template <int DIM, typename T>
__device__ __forceinline__ void line_pass_acc(const T* x, int dir, int l, const T* m, const T* acc, T* dst) {
  int b, s;
  line_idx<DIM>(dir, l, b, s);
  const T x0 = x[b], x1 = x[b + s], x2 = x[b + 2 * s];
  const T a0 = acc[b], a1 = acc[b + s], a2 = acc[b + 2 * s];
  dst[b] = a0 + m[0] * x0 + m[1] * x1 + m[2] * x2;
  dst[b + s] = a1 + m[3] * x0 + m[4] * x1 + m[5] * x2;
  dst[b + 2 * s] = a2 + m[6] * x0 + m[7] * x1 + m[8] * x2;
}

// symmetric tensor storage: 3D (00,11,22,01,02,12), 2D (00,11,01)
template <int DIM> __device__ __forceinline__ int sym_idx(int i, int j) {
  if (DIM == 2) return i == j ? i : 2;
  if (i == j) return i;
  int a = i < j ? i : j, b = i < j ? j : i;
  return a == 0 ? (b == 1 ? 3 : 4) : 5;
}

// lifting g_hat (eq. def-b-gam, Sec. 3.2): inflow profile 1 is
// (vbar 6y(1-y) [6z(1-z)], 0, 0) in coordinates scaled by the box, constant
// in x; grad[i*3+j] = d_j g_i
__device__ __forceinline__ void lifting(const OpArgs& a, const double x[3], double g[3], double grad[9]) {
  for (int i = 0; i < 3; ++i) g[i] = 0.0;
  for (int i = 0; i < 9; ++i) grad[i] = 0.0;
  if (a.inflow != 1) return;
  const double y = x[1] / a.L[1];
  const double fy = 6.0 * y * (1.0 - y), dfy = 6.0 * (1.0 - 2.0 * y) / a.L[1];
  double fz = 1.0, dfz = 0.0;
  if (a.g2[2] > 1) {
    const double z = x[2] / a.L[2];
    fz = 6.0 * z * (1.0 - z);
    dfz = 6.0 * (1.0 - 2.0 * z) / a.L[2];
  }
  g[0] = a.vbar * fy * fz;
  grad[1] = a.vbar * dfy * fz;
  grad[2] = a.vbar * fy * dfz;
}

template <int DIM, int K1, typename T>
struct OpCfg {
  using D = Dims<DIM>;
  static constexpr int C = DIM == 3 ? ((sizeof(T) == 8 ? 28 : 48) / K1) : (96 / K1);
  static constexpr int S = C * K1;
  // per-slot shared arrays (elements of T)
  static constexpr int SX = D::NC * D::NQ;
  static constexpr int SG = D::NC * DIM * D::NQ;
  static constexpr int SP = D::NP;
  static constexpr int per_slot = SX + SG + SP + SX + SP;
  static constexpr size_t smem_bytes = (size_t)S * per_slot * sizeof(T) + (size_t)S * 4 * sizeof(int) + 64;
};

template <int DIM, int K1, typename T, int MODE, int TAN>
__global__ void __launch_bounds__(OP_THREADS) st_op_kernel(const OpArgs a) {
  using D = Dims<DIM>;
  using Cfg = OpCfg<DIM, K1, T>;
  constexpr int NQ = D::NQ, NC = D::NC, NP = D::NP, NL = D::NL, NFQ = D::NFQ, NS = D::NS;
  constexpr int C = Cfg::C, S = Cfg::S;
  const auto& ct = CT<T>::t();

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sX = reinterpret_cast<T*>(smem_raw);
  T* sG = sX + S * Cfg::SX;
  T* sP = sG + S * Cfg::SG;
  T* sO = sP + S * Cfg::SP;   // TV, then velocity output
  T* sOp = sO + S * Cfg::SX;  // pressure output
  int* sCell = reinterpret_cast<int*>(sOp + S * Cfg::SP);  // linear cell id of batch cell
  int* sFside = sCell + S;    // per slot: side of the face in this round
  int* sFid = sFside + S;     // per slot: face id
  int* sAct = sFid + S;       // compacted list of slots with a face
  __shared__ int sNact;
  __shared__ int sBfaces;     // max number of boundary faces of a batch cell

  const T* in = reinterpret_cast<const T*>(a.in);
  T* out = reinterpret_cast<T*>(a.out);

  // balanced chunk of the colour class
  const long ncol = a.ncol;
  const long cbeg = (long)blockIdx.x * ncol / gridDim.x;
  const long cend = (long)(blockIdx.x + 1) * ncol / gridDim.x;

  const T* Dd[3] = {nullptr, nullptr, nullptr};
  const T* Ddt[3] = {nullptr, nullptr, nullptr};
  // scaled derivative matrices in the precision of the kernel
  __shared__ T sDd[3][9], sDdt[3][9], sM1[3][9];
  if (threadIdx.x < 27) {
    const int d = threadIdx.x / 9, e = threadIdx.x % 9;
    sDd[d][e] = (T)a.Dd[d][e];
    sDdt[d][e] = (T)a.Ddt[d][e];
    sM1[d][e] = (T)a.M1d[d][e];
  }
  for (int d = 0; d < 3; ++d) {
    Dd[d] = sDd[d];
    Ddt[d] = sDdt[d];
  }
  __syncthreads();

  for (long b0 = cbeg; b0 < cend; b0 += C) {
    const int nc = (int)min((long)C, cend - b0);
    const int ns = nc * K1;

    // ---- batch setup: cell ids, boundary-face counts
    if (threadIdx.x == 0) sBfaces = 0;
    __syncthreads();
    for (int ci = threadIdx.x; ci < nc; ci += blockDim.x) {
      const long li = b0 + ci;  // index within the colour class
      const int i = (int)(li % a.cn[0]);
      const int j = (int)((li / a.cn[0]) % a.cn[1]);
      const int l = (int)(li / ((long)a.cn[0] * a.cn[1]));
      const int ex = a.c0[0] + 2 * i, ey = a.c0[1] + 2 * j, ez = (DIM == 3) ? a.c0[2] + 2 * l : 0;
      sCell[ci] = ex + a.n[0] * (ey + a.n[1] * ez);
      int nb = 0;
      const int e3[3] = {ex, ey, ez};
      for (int ax = 0; ax < DIM; ++ax) nb += (e3[ax] == 0) + (e3[ax] == a.n[ax] - 1);
      atomicMax(&sBfaces, nb);
    }
    __syncthreads();

    // ---- S0: gather nodal values of every slot (velocity, pressure)
    for (int it = threadIdx.x; it < ns * (NC * NQ + NP); it += blockDim.x) {
      const int s = it / (NC * NQ + NP), r = it % (NC * NQ + NP);
      const int ci = s / K1, mu = s % K1;
      const int cell = sCell[ci];
      const int ex = cell % a.n[0], ey = (cell / a.n[0]) % a.n[1], ez = (DIM == 3) ? cell / (a.n[0] * a.n[1]) : 0;
      if (r < NC * NQ) {
        const int c = r / NQ, q = r % NQ;
        const int qx = q % 3, qy = (q / 3) % 3, qz = (DIM == 3) ? q / 9 : 0;
        const long g = (2L * ex + qx) + a.g2[0] * ((2L * ey + qy) + a.g2[1] * (2L * ez + qz));
        sX[s * Cfg::SX + r] = in[(long)mu * a.Mv + c * a.Nq2 + g];
      } else {
        const int m = r - NC * NQ;
        const int mx = m & 1, my = (m >> 1) & 1, mz = (DIM == 3) ? (m >> 2) : 0;
        const long g = (ex + mx) + a.g1[0] * ((ey + my) + a.g1[1] * (ez + mz));
        sP[s * NP + m] = in[(long)K1 * a.Mv + (long)mu * a.Mp + g];
      }
    }
    __syncthreads();

    // ---- S1: values at the Gauss points, one pass per direction (in place)
    for (int dir = 0; dir < DIM; ++dir) {
      for (int it = threadIdx.x; it < ns * NC * NL; it += blockDim.x) {
        const int s = it / (NC * NL), r = it % (NC * NL);
        T* x = sX + s * Cfg::SX + (r / NL) * NQ;
        line_pass<DIM, T>(x, dir, r % NL, ct.B, x);
      }
      __syncthreads();
    }

    // ---- S2: gradients in collocation form; time mixing of the values (JAC)
    {
      const int n_grad = ns * NC * DIM * NL;
      const int n_mix = (MODE == OP_JAC) ? nc * NC * NQ : 0;
      for (int it = threadIdx.x; it < n_grad + n_mix; it += blockDim.x) {
        if (it < n_grad) {
          const int s = it / (NC * DIM * NL), r = it % (NC * DIM * NL);
          const int c = r / (DIM * NL), dir = (r / NL) % DIM, l = r % NL;
          const T* x = sX + s * Cfg::SX + c * NQ;
          T* g = sG + s * Cfg::SG + (c * DIM + dir) * NQ;
          int b, st;
          line_idx<DIM>(dir, l, b, st);
          T y0, y1, y2;
          apply3<T, T>(Dd[dir], x[b], x[b + st], x[b + 2 * st], y0, y1, y2);
          g[b] = y0;
          g[b + st] = y1;
          g[b + 2 * st] = y2;
        } else {
          // tv_i(q) = W(q) sum_j (K_t vol)_ij du_j(q): the K_t (x) M_x block at the quadrature points
          const int r = it - n_grad;
          const int ci = r / (NC * NQ), c = (r / NQ) % NC, q = r % NQ;
          T xj[K1];
#pragma unroll
          for (int j = 0; j < K1; ++j) xj[j] = sX[(ci * K1 + j) * Cfg::SX + c * NQ + q];
          const T wq = (DIM == 3) ? ct.WQ3[q] : ct.WQ2[q];
#pragma unroll
          for (int i = 0; i < K1; ++i) {
            T sacc = (T)a.KtV[i * K1] * xj[0];
#pragma unroll
            for (int j = 1; j < K1; ++j) sacc += (T)a.KtV[i * K1 + j] * xj[j];
            sO[(ci * K1 + i) * Cfg::SX + c * NQ + q] = sacc * wq;
          }
        }
      }
      __syncthreads();
    }

    // ---- S3: pointwise work at every quadrature point of every slot
    for (int it = threadIdx.x; it < ns * NQ; it += blockDim.x) {
      const int s = it / NQ, q = it % NQ;
      const int ci = s / K1, mu = s % K1;
      const long gidx = a.col_start + b0 + ci;  // colour-ordered cell index
      T u[3] = {0, 0, 0}, g[3][3];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        u[c] = sX[s * Cfg::SX + c * NQ + q];
#pragma unroll
        for (int j = 0; j < DIM; ++j) g[c][j] = sG[s * Cfg::SG + (c * DIM + j) * NQ + q];
      }
      const T wq = (DIM == 3) ? ct.WQ3[q] : ct.WQ2[q];
      if constexpr (MODE == OP_LIN) {
        // coefficients of the linearisation, FP64 (Sec. 4.1)
        double A[NS];
#pragma unroll
        for (int i = 0; i < DIM; ++i) A[i] = (double)g[i][i];
        A[DIM] = 0.5 * ((double)g[0][1] + (double)g[1][0]);
        if (DIM == 3) {
          A[4] = 0.5 * ((double)g[0][2] + (double)g[2][0]);
          A[5] = 0.5 * ((double)g[1][2] + (double)g[2][1]);
        }
        double a2 = 0.0;
#pragma unroll
        for (int i = 0; i < NS; ++i) a2 += (i < DIM ? 1.0 : 2.0) * A[i] * A[i];
        const double D2 = a.delta * a.delta + a2;
        const double mu_m = a.nu * pow(D2, 0.5 * (a.p - 2.0));
        const double eta = a.nu_inf + mu_m;
        double cfac = 0.0;
        if (a.tangent == ST_EXN) {
          cfac = (a.p - 2.0) * mu_m / D2;
        } else if (a.tangent == ST_MODN) {
          const double sig = mu_m * sqrt(a2);
          const double sc = sig > 0.0 ? fmin(1.0, a.sigma_max / sig) : 0.0;
          cfac = sc * (a.p - 2.0) * mu_m / D2;
        }
        const double tw = (double)wq * a.vol * a.tw[mu];
        double* cp = a.wcache + ((gidx * K1 + mu) * (long)D::NF_VOL) * NQ + q;
        cp[0 * NQ] = eta * tw;
        cp[1 * NQ] = cfac * tw;
#pragma unroll
        for (int i = 0; i < NS; ++i) cp[(2 + i) * NQ] = A[i];
#pragma unroll
        for (int c = 0; c < NC; ++c) cp[(2 + NS + c) * NQ] = -(double)u[c] * tw;
      } else if constexpr (MODE == OP_JAC) {
        const T* cp = reinterpret_cast<const T*>(a.cache) + ((gidx * K1 + mu) * (long)D::NF_VOL) * NQ + q;
        const T etaw = cp[0];
        T nuw[3] = {0, 0, 0};
#pragma unroll
        for (int c = 0; c < NC; ++c) nuw[c] = cp[(2 + NS + c) * NQ];
        // pressure increment at q
        const T* psi = (DIM == 3) ? &ct.PSI3[q * 8] : &ct.PSI2[q * 4];
        T dpi = 0;
#pragma unroll
        for (int m = 0; m < NP; ++m) dpi += psi[m] * sP[s * NP + m];
        const T tw = wq * (T)(a.vol * a.tw[mu]);
        const T pd = -dpi * tw;
        T G[3][3];
        if constexpr (TAN == 1) {
          // T(B) = eta B + c (A:B) A with B = D(du); convection -(du (x) u + u (x) du)
          const T cw = cp[NQ];
          T Am[NS];
#pragma unroll
          for (int i = 0; i < NS; ++i) Am[i] = cp[(2 + i) * NQ];
          T bo[3];  // 2 * off-diagonal entries of D(du)
          bo[0] = g[0][1] + g[1][0];
          if (DIM == 3) {
            bo[1] = g[0][2] + g[2][0];
            bo[2] = g[1][2] + g[2][1];
          }
          T AB = Am[0] * g[0][0] + Am[1] * g[1][1];
          if (DIM == 3) AB += Am[2] * g[2][2] + Am[3] * bo[0] + Am[4] * bo[1] + Am[5] * bo[2];
          else AB += Am[2] * bo[0];
          const T sfac = cw * AB;
          const T hw = (T)0.5 * etaw;
#pragma unroll
          for (int i = 0; i < DIM; ++i) {
            const T du2 = u[i] + u[i];
            G[i][i] = etaw * g[i][i] + (sfac * Am[i] + (du2 * nuw[i] + pd));
          }
          {
            const T v01 = hw * bo[0] + (sfac * Am[DIM] + (u[0] * nuw[1] + u[1] * nuw[0]));
            G[0][1] = v01;
            G[1][0] = v01;
          }
          if (DIM == 3) {
            const T v02 = hw * bo[1] + (sfac * Am[4] + (u[0] * nuw[2] + u[2] * nuw[0]));
            const T v12 = hw * bo[2] + (sfac * Am[5] + (u[1] * nuw[2] + u[2] * nuw[1]));
            G[0][2] = v02;
            G[2][0] = v02;
            G[1][2] = v12;
            G[2][1] = v12;
          }
        } else {
          // Picard: T(B) = eta B, convection -(du (x) u) with the advecting u lagged
          const T hw = (T)0.5 * etaw;
#pragma unroll
          for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) {
              const T bij = (i == j) ? etaw * g[i][i] : hw * (g[i][j] + g[j][i]);
              G[i][j] = bij + u[i] * nuw[j] + (i == j ? pd : (T)0);
            }
        }
        T div = g[0][0] + g[1][1];
        if (DIM == 3) div += g[2][2];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int j = 0; j < DIM; ++j) sG[s * Cfg::SG + (c * DIM + j) * NQ + q] = G[c][j];
        sX[s * Cfg::SX + q] = -div * tw;  // pressure test flux (aliases the value array)
      } else {  // OP_RES: F = RHS - LHS, gradient-test flux -(S(Du) - u (x) u - pi I)
        const T* psi = (DIM == 3) ? &ct.PSI3[q * 8] : &ct.PSI2[q * 4];
        T pi = 0;
#pragma unroll
        for (int m = 0; m < NP; ++m) pi += psi[m] * sP[s * NP + m];
        T A[3][3];
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
          for (int j = 0; j < DIM; ++j) A[i][j] = (T)0.5 * (g[i][j] + g[j][i]);
        T a2 = 0;
#pragma unroll
        for (int i = 0; i < DIM; ++i)
#pragma unroll
          for (int j = 0; j < DIM; ++j) a2 += A[i][j] * A[i][j];
        const T eta = (T)a.nu_inf + (T)a.nu * pow((T)(a.delta * a.delta) + a2, (T)(0.5 * (a.p - 2.0)));
        const T tw = wq * (T)(a.vol * a.tw[mu]);
        T div = 0;
#pragma unroll
        for (int i = 0; i < DIM; ++i) div += g[i][i];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int j = 0; j < DIM; ++j)
            sG[s * Cfg::SG + (c * DIM + j) * NQ + q] = -(eta * A[c][j] - u[c] * u[j] - (c == j ? pi : (T)0)) * tw;
        sX[s * Cfg::SX + q] = div * tw;
      }
    }
    __syncthreads();

    if constexpr (MODE != OP_LIN) {
      // ---- integration: collocation-space sum of the derivative tests (chain)
      for (int dir = 0; dir < DIM; ++dir) {
        const int n_lines = ns * NC * NL;
        const int n_pt = (dir == 0) ? ns * NP : 0;
        for (int it = threadIdx.x; it < n_lines + n_pt; it += blockDim.x) {
          if (it < n_lines) {
            const int s = it / (NC * NL), r = it % (NC * NL);
            const int c = r / NL, l = r % NL;
            T* gsl = sG + s * Cfg::SG + (c * DIM + dir) * NQ;
            if (dir == 0) {
              if (MODE == OP_JAC) {
                line_pass_acc<DIM, T>(gsl, 0, l, Ddt[0], sO + s * Cfg::SX + c * NQ, gsl);
              } else {
                line_pass<DIM, T>(gsl, 0, l, Ddt[0], gsl);
              }
            } else {
              line_pass_acc<DIM, T>(gsl, dir, l, Ddt[dir], gsl - NQ, gsl);
            }
          } else {
            // pressure test: out_m = sum_q psi_m(q) Q(q)
            const int r = it - n_lines;
            const int s = r / NP, m = r % NP;
            T acc = 0;
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc += ((DIM == 3) ? ct.PSI3[q * 8 + m] : ct.PSI2[q * 4 + m]) * sX[s * Cfg::SX + q];
            sOp[s * NP + m] = acc;
          }
        }
        __syncthreads();
      }
      // ---- transposed value passes -> nodal output in sO
      for (int dir = 0; dir < DIM; ++dir) {
        for (int it = threadIdx.x; it < ns * NC * NL; it += blockDim.x) {
          const int s = it / (NC * NL), r = it % (NC * NL);
          const int c = r / NL, l = r % NL;
          T* gsl = sG + s * Cfg::SG + (c * DIM + DIM - 1) * NQ;
          T* dst = (dir == DIM - 1) ? sO + s * Cfg::SX + c * NQ : gsl;
          line_pass<DIM, T>(gsl, dir, l, ct.Bt, dst);
        }
        __syncthreads();
      }
      if constexpr (MODE == OP_RES) {
        // ---- value terms in nodal form: M_e (-sum_j K_ij u_j + m_i v^- + tau w_i f_i)
        const T* vp = reinterpret_cast<const T*>(a.vprev);
        const T* ff = reinterpret_cast<const T*>(a.f);
        for (int it = threadIdx.x; it < nc * NC * NQ; it += blockDim.x) {
          const int ci = it / (NC * NQ), c = (it / NQ) % NC, q = it % NQ;
          const int cell = sCell[ci];
          const int ex = cell % a.n[0], ey = (cell / a.n[0]) % a.n[1], ez = (DIM == 3) ? cell / (a.n[0] * a.n[1]) : 0;
          const int qx = q % 3, qy = (q / 3) % 3, qz = (DIM == 3) ? q / 9 : 0;
          const long gn = (2L * ex + qx) + a.g2[0] * ((2L * ey + qy) + a.g2[1] * (2L * ez + qz)) + c * a.Nq2;
          T uj[K1];
#pragma unroll
          for (int j = 0; j < K1; ++j) uj[j] = in[(long)j * a.Mv + gn];
          const T v = vp ? vp[gn] : (T)0;
#pragma unroll
          for (int i = 0; i < K1; ++i) {
            T y = (T)a.mt[i] * v;
#pragma unroll
            for (int j = 0; j < K1; ++j) y -= (T)a.Kt[i * K1 + j] * uj[j];
            if (ff) y += (T)a.tw[i] * ff[(long)i * a.Mv + gn];
            sX[(ci * K1 + i) * Cfg::SX + c * NQ + q] = y;
          }
        }
        __syncthreads();
        for (int dir = 0; dir < DIM; ++dir) {
          for (int it = threadIdx.x; it < ns * NC * NL; it += blockDim.x) {
            const int s = it / (NC * NL), r = it % (NC * NL);
            T* x = sX + s * Cfg::SX + (r / NL) * NQ;
            line_pass<DIM, T>(x, dir, r % NL, sM1[dir], x);
          }
          __syncthreads();
        }
        for (int it = threadIdx.x; it < ns * NC * NQ; it += blockDim.x) {
          const int s = it / (NC * NQ), r = it % (NC * NQ);
          sO[s * Cfg::SX + r] += sX[s * Cfg::SX + r];
        }
        __syncthreads();
      }
    }

    // ---- boundary faces, in rounds of at most one face per slot
    const int nrounds = sBfaces;
    for (int round = 0; round < nrounds; ++round) {
      if (threadIdx.x == 0) {
        int na = 0;
        for (int s = 0; s < ns; ++s) {
          const int ci = s / K1;
          const int cell = sCell[ci];
          const int e3[3] = {cell % a.n[0], (cell / a.n[0]) % a.n[1], (DIM == 3) ? cell / (a.n[0] * a.n[1]) : 0};
          int r = 0, side = -1;
          for (int sd = 0; sd < 2 * DIM && side < 0; ++sd) {
            const int ax = sd >> 1, up = sd & 1;
            const bool on = up ? (e3[ax] == a.n[ax] - 1) : (e3[ax] == 0);
            if (on) {
              if (r == round) side = sd;
              ++r;
            }
          }
          sFside[s] = side;
          if (side >= 0) {
            sAct[na++] = s;
            sFid[s] = a.face_off[a.col_start + b0 + ci] + round;
          }
        }
        sNact = na;
      }
      __syncthreads();
      const int na = sNact;
      // workspace inside the slot's gradient array: PV[NC][NFQ], PN[NC][NFQ], PT[NC][DIM-1][NFQ], FQ[NFQ]
      constexpr int oPV = 0, oPN = NC * NFQ, oPT = 2 * NC * NFQ, oFQ = 2 * NC * NFQ + NC * (DIM - 1) * NFQ;
      // FA: face-plane nodal values and normal derivatives
      for (int it = threadIdx.x; it < na * NC * NFQ; it += blockDim.x) {
        const int ai = it / (NC * NFQ), c = (it / NFQ) % NC, tn = it % NFQ;
        const int s = sAct[ai], side = sFside[s], ax = side >> 1, up = side & 1;
        const int ci = s / K1, mu = s % K1;
        const int cell = sCell[ci];
        const int e3[3] = {cell % a.n[0], (cell / a.n[0]) % a.n[1], (DIM == 3) ? cell / (a.n[0] * a.n[1]) : 0};
        const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
        int pos[3] = {0, 0, 0};
        pos[t1] = tn % 3;
        if (DIM == 3) pos[t2] = tn / 3;
        T v[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          pos[ax] = i;
          const long gnode = (2L * e3[0] + pos[0]) + a.g2[0] * ((2L * e3[1] + pos[1]) + a.g2[1] * (2L * e3[2] + pos[2]));
          v[i] = in[(long)mu * a.Mv + c * a.Nq2 + gnode];
        }
        T* w = sG + s * Cfg::SG;
        w[oPV + c * NFQ + tn] = up ? v[2] : v[0];
        const T ih = (T)a.ih[ax];
        w[oPN + c * NFQ + tn] = ((T)ct.ED[up * 3 + 0] * v[0] + (T)ct.ED[up * 3 + 1] * v[1] + (T)ct.ED[up * 3 + 2] * v[2]) * ih;
      }
      __syncthreads();
      // FB: values at the face points (tangential passes on PV and PN)
      for (int td = 0; td < DIM - 1; ++td) {
        constexpr int FL = (DIM == 3) ? 3 : 1;
        for (int it = threadIdx.x; it < na * NC * 2 * FL; it += blockDim.x) {
          const int ai = it / (NC * 2 * FL), c = (it / (2 * FL)) % NC, wh = (it / FL) % 2, l = it % FL;
          const int s = sAct[ai];
          T* x = sG + s * Cfg::SG + (wh ? oPN : oPV) + c * NFQ;
          // face plane indexed tn = i1 + 3 i2: lines along i1 (td = 0) or i2 (td = 1)
          const int b = (td == 0) ? 3 * l : l, st = (td == 0) ? 1 : 3;
          T y0, y1, y2;
          apply3<T, T>(ct.B, x[b], x[b + st], x[b + 2 * st], y0, y1, y2);
          x[b] = y0;
          x[b + st] = y1;
          x[b + 2 * st] = y2;
        }
        __syncthreads();
      }
      // FC: tangential derivatives at the face points (collocation form)
      {
        constexpr int FL = (DIM == 3) ? 3 : 1;
        for (int it = threadIdx.x; it < na * NC * (DIM - 1) * FL; it += blockDim.x) {
          const int ai = it / (NC * (DIM - 1) * FL), c = (it / ((DIM - 1) * FL)) % NC, td = (it / FL) % (DIM - 1),
                    l = it % FL;
          const int s = sAct[ai], side = sFside[s], ax = side >> 1;
          const int tax = (td == 0) ? (ax == 0 ? 1 : 0) : (ax == 2 ? 1 : 2);
          const T* x = sG + s * Cfg::SG + oPV + c * NFQ;
          T* y = sG + s * Cfg::SG + oPT + (c * (DIM - 1) + td) * NFQ;
          const int b = (td == 0) ? 3 * l : l, st = (td == 0) ? 1 : 3;
          T y0, y1, y2;
          apply3<T, T>(Dd[tax], x[b], x[b + st], x[b + 2 * st], y0, y1, y2);
          y[b] = y0;
          y[b + st] = y1;
          y[b + 2 * st] = y2;
        }
        __syncthreads();
      }
      // FD: pointwise face terms
      for (int it = threadIdx.x; it < na * NFQ; it += blockDim.x) {
        const int ai = it / NFQ, fq = it % NFQ;
        const int s = sAct[ai], side = sFside[s], ax = side >> 1, up = side & 1;
        const int ci = s / K1, mu = s % K1;
        const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
        const bool isD = (a.dmask >> side) & 1u;
        T* w = sG + s * Cfg::SG;
        T u[3] = {0, 0, 0}, g[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          u[c] = w[oPV + c * NFQ + fq];
          g[c][ax] = w[oPN + c * NFQ + fq];
          g[c][t1] = w[oPT + (c * (DIM - 1) + 0) * NFQ + fq];
          if (DIM == 3) g[c][t2] = w[oPT + (c * (DIM - 1) + 1) * NFQ + fq];
        }
        const T nsg = up ? (T)1 : (T)-1;  // n = nsg e_ax
        // pressure at the face point from the face's Q1 nodes
        T pf = 0;
        {
#pragma unroll
          for (int m = 0; m < D::NFP; ++m) {
            int mm[3] = {0, 0, 0};
            mm[ax] = up;
            mm[t1] = m & 1;
            if (DIM == 3) mm[t2] = m >> 1;
            const int pm = mm[0] + 2 * mm[1] + 4 * mm[2];
            pf += ((DIM == 3) ? ct.FPSI3[fq * 4 + m] : ct.FPSI2[fq * 2 + m]) * sP[s * NP + pm];
          }
        }
        const double hD = a.h[ax];
        T V[3] = {0, 0, 0}, Gf[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Qf = 0;
        if constexpr (MODE == OP_LIN) {
          // physical point, face weight
          const int cell = sCell[ci];
          const int e3[3] = {cell % a.n[0], (cell / a.n[0]) % a.n[1], (DIM == 3) ? cell / (a.n[0] * a.n[1]) : 0};
          const double* Wg = cT.W;
          const double gpt[3] = {0.5 - 0.3872983346207417, 0.5, 0.5 + 0.3872983346207417};
          double r3[3] = {0, 0, 0};
          r3[ax] = up ? 1.0 : 0.0;
          r3[t1] = gpt[fq % 3];
          if (DIM == 3) r3[t2] = gpt[fq / 3];
          double x[3];
          for (int d = 0; d < 3; ++d) x[d] = d < DIM ? (e3[d] + r3[d]) * a.h[d] : 0.0;
          double fw = ((DIM == 3) ? cT.FW3[fq] : cT.FW2[fq]) * a.tw[mu];
          for (int d = 0; d < DIM; ++d)
            if (d != ax) fw *= a.h[d];
          (void)Wg;
          double Am[NS];
#pragma unroll
          for (int i = 0; i < DIM; ++i) Am[i] = (double)g[i][i];
          Am[DIM] = 0.5 * ((double)g[0][1] + (double)g[1][0]);
          if (DIM == 3) {
            Am[4] = 0.5 * ((double)g[0][2] + (double)g[2][0]);
            Am[5] = 0.5 * ((double)g[1][2] + (double)g[2][1]);
          }
          double a2 = 0.0;
#pragma unroll
          for (int i = 0; i < NS; ++i) a2 += (i < DIM ? 1.0 : 2.0) * Am[i] * Am[i];
          const double D2 = a.delta * a.delta + a2;
          const double mu_m = a.nu * pow(D2, 0.5 * (a.p - 2.0));
          const double eta = a.nu_inf + mu_m;
          double cfac = 0.0;
          if (a.tangent == ST_EXN) {
            cfac = (a.p - 2.0) * mu_m / D2;
          } else if (a.tangent == ST_MODN) {
            const double sig = mu_m * sqrt(a2);
            const double sc = sig > 0.0 ? fmin(1.0, a.sigma_max / sig) : 0.0;
            cfac = sc * (a.p - 2.0) * mu_m / D2;
          }
          const double un = (double)nsg * (double)u[ax];
          const double negp = 0.5 * (fabs(un) - un);
          double gl[3], ggr[9];
          lifting(a, x, gl, ggr);
          double Dg[NS];
#pragma unroll
          for (int i = 0; i < DIM; ++i) Dg[i] = ggr[i * 3 + i];
          Dg[DIM] = 0.5 * (ggr[1] + ggr[3]);
          if (DIM == 3) {
            Dg[4] = 0.5 * (ggr[2] + ggr[6]);
            Dg[5] = 0.5 * (ggr[5] + ggr[7]);
          }
          double g2n = 0.0;
#pragma unroll
          for (int i = 0; i < NS; ++i) g2n += (i < DIM ? 1.0 : 2.0) * Dg[i] * Dg[i];
          const double DgD = a.delta * a.delta + g2n;
          const double etaD = a.nu_inf + a.nu * pow(DgD, 0.5 * (a.p - 2.0));
          const double betaD = a.nu * (a.p - 2.0) * pow(DgD, 0.5 * (a.p - 4.0));
          const long fid = sFid[s];
          double* cp = a.wfcache + ((fid * K1 + mu) * (long)D::NF_FACE) * NFQ + fq;
          int o = 0;
          cp[(o++) * NFQ] = eta * fw;
          cp[(o++) * NFQ] = cfac * fw;
#pragma unroll
          for (int i = 0; i < NS; ++i) cp[(o++) * NFQ] = Am[i];
#pragma unroll
          for (int c = 0; c < NC; ++c) cp[(o++) * NFQ] = (double)u[c] * fw;
          cp[(o++) * NFQ] = negp * fw;
          cp[(o++) * NFQ] = a.gamma1 / hD * etaD * fw;
          cp[(o++) * NFQ] = a.gamma2 / hD * fw;
          cp[(o++) * NFQ] = etaD * fw;
          cp[(o++) * NFQ] = betaD * fw;
#pragma unroll
          for (int i = 0; i < NS; ++i) cp[(o++) * NFQ] = Dg[i];
          cp[(o++) * NFQ] = fw;
          (void)pf;
          (void)isD;
          continue;
        } else if constexpr (MODE == OP_JAC) {
          const T* cp = reinterpret_cast<const T*>(a.fcache) + (((long)sFid[s] * K1 + mu) * (long)D::NF_FACE) * NFQ + fq;
          constexpr int oU = 2 + NS, oN = oU + NC;
          T uw[3] = {0, 0, 0};
#pragma unroll
          for (int c = 0; c < NC; ++c) uw[c] = cp[(oU + c) * NFQ];
          const T unw = nsg * uw[ax];
          const T dun = nsg * u[ax];
#pragma unroll
          for (int c = 0; c < NC; ++c) V[c] = unw * u[c] + (TAN == 1 ? dun * uw[c] : (T)0);
          if (isD) {
            const T etaw = cp[0], cw = cp[NQ > 0 ? NFQ : 0];
            T Am[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) Am[i] = cp[(2 + i) * NFQ];
            const T negw = cp[oN * NFQ], pen1 = cp[(oN + 1) * NFQ], pen2 = cp[(oN + 2) * NFQ];
            const T etaDw = cp[(oN + 3) * NFQ], betaDw = cp[(oN + 4) * NFQ];
            T Dg[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) Dg[i] = cp[(oN + 5 + i) * NFQ];
            const T fw = cp[(oN + 5 + NS) * NFQ];
            // B = D(du) (full), (T B) n
            T Bm[3][3];
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
              for (int j = 0; j < DIM; ++j) Bm[i][j] = (T)0.5 * (g[i][j] + g[j][i]);
            T AB = 0;
            if (TAN == 1) {
#pragma unroll
              for (int i = 0; i < DIM; ++i)
#pragma unroll
                for (int j = 0; j < DIM; ++j) AB += Am[sym_idx<DIM>(i, j)] * Bm[i][j];
            }
            const T sfac = cw * AB;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              const T Tn = nsg * (etaw * Bm[c][ax] + (TAN == 1 ? sfac * Am[sym_idx<DIM>(c, ax)] : (T)0));
              V[c] += -Tn - negw * u[c] + pen1 * u[c];
            }
            V[ax] += nsg * (pf * fw) + pen2 * dun * nsg;
            // -(du, DS(Dg)(Dz) n) = -DS(Dg)(sym(du (x) n)) : grad z
            T Sd[3][3];
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
              for (int j = 0; j < DIM; ++j)
                Sd[i][j] = (T)0.5 * ((j == ax ? nsg * u[i] : (T)0) + (i == ax ? nsg * u[j] : (T)0));
            T gS = 0;
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
              for (int j = 0; j < DIM; ++j) gS += Dg[sym_idx<DIM>(i, j)] * Sd[i][j];
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
              for (int j = 0; j < DIM; ++j) Gf[i][j] = -(etaDw * Sd[i][j] + betaDw * gS * Dg[sym_idx<DIM>(i, j)]);
            Qf = (T)a.q_sign * dun * fw;
          }
        } else {  // OP_RES face terms, F = RHS - LHS
          const int cell = sCell[ci];
          const int e3[3] = {cell % a.n[0], (cell / a.n[0]) % a.n[1], (DIM == 3) ? cell / (a.n[0] * a.n[1]) : 0};
          const double gpt[3] = {0.5 - 0.3872983346207417, 0.5, 0.5 + 0.3872983346207417};
          double r3[3] = {0, 0, 0};
          r3[ax] = up ? 1.0 : 0.0;
          r3[t1] = gpt[fq % 3];
          if (DIM == 3) r3[t2] = gpt[fq / 3];
          double x[3];
          for (int d = 0; d < 3; ++d) x[d] = d < DIM ? (e3[d] + r3[d]) * a.h[d] : 0.0;
          double fwd = ((DIM == 3) ? cT.FW3[fq] : cT.FW2[fq]) * a.tw[mu];
          for (int d = 0; d < DIM; ++d)
            if (d != ax) fwd *= a.h[d];
          const T fw = (T)fwd;
          const T un = nsg * u[ax];
#pragma unroll
          for (int c = 0; c < NC; ++c) V[c] = -un * u[c] * fw;
          if (isD) {
            double gl[3], ggr[9];
            lifting(a, x, gl, ggr);
            double Dgf[3][3];
            double g2n = 0.0;
            for (int i = 0; i < 3; ++i)
              for (int j = 0; j < 3; ++j) {
                Dgf[i][j] = 0.5 * (ggr[i * 3 + j] + ggr[j * 3 + i]);
                g2n += Dgf[i][j] * Dgf[i][j];
              }
            const double DgD = a.delta * a.delta + g2n;
            const T etaD = (T)(a.nu_inf + a.nu * pow(DgD, 0.5 * (a.p - 2.0)));
            const T betaD = (T)(a.nu * (a.p - 2.0) * pow(DgD, 0.5 * (a.p - 4.0)));
            T A[3][3];
            T a2 = 0;
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
              for (int j = 0; j < DIM; ++j) {
                A[i][j] = (T)0.5 * (g[i][j] + g[j][i]);
                a2 += A[i][j] * A[i][j];
              }
            const T eta = (T)a.nu_inf + (T)a.nu * pow((T)(a.delta * a.delta) + a2, (T)(0.5 * (a.p - 2.0)));
            const T gn = nsg * (T)gl[ax];
            const T negu = (T)0.5 * (fabs(un) - un), negg = (T)0.5 * (fabs(gn) - gn);
            T dlt[3] = {0, 0, 0};
#pragma unroll
            for (int c = 0; c < NC; ++c) dlt[c] = u[c] - (T)gl[c];
            const T dn = nsg * dlt[ax];
            const T p1 = (T)(a.gamma1 / hD) * etaD, p2 = (T)(a.gamma2 / hD);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              const T Sn = nsg * eta * A[c][ax];
              V[c] += (Sn - (c == ax ? nsg * pf : (T)0) + negu * u[c] - negg * (T)gl[c] - p1 * dlt[c] -
                       (c == ax ? p2 * dn * nsg : (T)0)) * fw;
            }
            T Sd[3][3];
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
              for (int j = 0; j < DIM; ++j)
                Sd[i][j] = (T)0.5 * ((j == ax ? nsg * dlt[i] : (T)0) + (i == ax ? nsg * dlt[j] : (T)0));
            T gS = 0;
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
              for (int j = 0; j < DIM; ++j) gS += (T)Dgf[i][j] * Sd[i][j];
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
              for (int j = 0; j < DIM; ++j) Gf[i][j] = (etaD * Sd[i][j] + betaD * gS * (T)Dgf[i][j]) * fw;
            Qf = -(T)a.q_sign * dn * fw;
          }
        }
        if constexpr (MODE != OP_LIN) {
          // store fluxes in place: FV <- PV slot, FGn <- PN slot, FGt <- PT slot
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            w[oPV + c * NFQ + fq] = V[c];
            w[oPN + c * NFQ + fq] = Gf[c][ax];
            w[oPT + (c * (DIM - 1) + 0) * NFQ + fq] = Gf[c][t1];
            if (DIM == 3) w[oPT + (c * (DIM - 1) + 1) * NFQ + fq] = Gf[c][t2];
          }
          w[oFQ + fq] = Qf;
        }
      }
      __syncthreads();
      if constexpr (MODE != OP_LIN) {
        constexpr int FL = (DIM == 3) ? 3 : 1;
        // FE1: tangential derivative tests, chained into FV
        for (int td = 0; td < DIM - 1; ++td) {
          for (int it = threadIdx.x; it < na * NC * FL; it += blockDim.x) {
            const int ai = it / (NC * FL), c = (it / FL) % NC, l = it % FL;
            const int s = sAct[ai], side = sFside[s], ax = side >> 1;
            const int tax = (td == 0) ? (ax == 0 ? 1 : 0) : (ax == 2 ? 1 : 2);
            T* w = sG + s * Cfg::SG;
            const T* x = w + oPT + (c * (DIM - 1) + td) * NFQ;
            T* y = w + oPV + c * NFQ;
            const int b = (td == 0) ? 3 * l : l, st = (td == 0) ? 1 : 3;
            const T* m = Ddt[tax];
            const T x0 = x[b], x1 = x[b + st], x2 = x[b + 2 * st];
            y[b] += m[0] * x0 + m[1] * x1 + m[2] * x2;
            y[b + st] += m[3] * x0 + m[4] * x1 + m[5] * x2;
            y[b + 2 * st] += m[6] * x0 + m[7] * x1 + m[8] * x2;
          }
          __syncthreads();
        }
        // FE2: transposed tangential value passes on FV and FGn
        for (int td = 0; td < DIM - 1; ++td) {
          for (int it = threadIdx.x; it < na * NC * 2 * FL; it += blockDim.x) {
            const int ai = it / (NC * 2 * FL), c = (it / (2 * FL)) % NC, wh = (it / FL) % 2, l = it % FL;
            const int s = sAct[ai];
            T* x = sG + s * Cfg::SG + (wh ? oPN : oPV) + c * NFQ;
            const int b = (td == 0) ? 3 * l : l, st = (td == 0) ? 1 : 3;
            T y0, y1, y2;
            apply3<T, T>(ct.Bt, x[b], x[b + st], x[b + 2 * st], y0, y1, y2);
            x[b] = y0;
            x[b + st] = y1;
            x[b + 2 * st] = y2;
          }
          __syncthreads();
        }
        // FF: expand onto the cell's nodes along the normal; pressure test
        for (int it = threadIdx.x; it < na * (NC * NFQ + D::NFP); it += blockDim.x) {
          const int ai = it / (NC * NFQ + D::NFP), r = it % (NC * NFQ + D::NFP);
          const int s = sAct[ai], side = sFside[s], ax = side >> 1, up = side & 1;
          const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
          T* w = sG + s * Cfg::SG;
          if (r < NC * NFQ) {
            const int c = r / NFQ, tn = r % NFQ;
            int pos[3] = {0, 0, 0};
            pos[t1] = tn % 3;
            if (DIM == 3) pos[t2] = tn / 3;
            const T fv = w[oPV + c * NFQ + tn], fn = w[oPN + c * NFQ + tn] * (T)a.ih[ax];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              pos[ax] = i;
              const int q = pos[0] + 3 * pos[1] + 9 * pos[2];
              sO[s * Cfg::SX + c * NQ + q] += (T)ct.E[up * 3 + i] * fv + (T)ct.ED[up * 3 + i] * fn;
            }
          } else {
            const int m = r - NC * NFQ;
            int mm[3] = {0, 0, 0};
            mm[ax] = up;
            mm[t1] = m & 1;
            if (DIM == 3) mm[t2] = m >> 1;
            const int pm = mm[0] + 2 * mm[1] + 4 * mm[2];
            T acc = 0;
#pragma unroll
            for (int fq = 0; fq < NFQ; ++fq)
              acc += ((DIM == 3) ? ct.FPSI3[fq * 4 + m] : ct.FPSI2[fq * 2 + m]) * w[oFQ + fq];
            sOp[s * NP + pm] += acc;
          }
        }
        __syncthreads();
      }
    }

    // ---- scatter-add (cells of one colour class share no node)
    if constexpr (MODE != OP_LIN) {
      for (int it = threadIdx.x; it < ns * (NC * NQ + NP); it += blockDim.x) {
        const int s = it / (NC * NQ + NP), r = it % (NC * NQ + NP);
        const int ci = s / K1, mu = s % K1;
        const int cell = sCell[ci];
        const int ex = cell % a.n[0], ey = (cell / a.n[0]) % a.n[1], ez = (DIM == 3) ? cell / (a.n[0] * a.n[1]) : 0;
        if (r < NC * NQ) {
          const int c = r / NQ, q = r % NQ;
          const int qx = q % 3, qy = (q / 3) % 3, qz = (DIM == 3) ? q / 9 : 0;
          const long g = (2L * ex + qx) + a.g2[0] * ((2L * ey + qy) + a.g2[1] * (2L * ez + qz));
          const long gi = (long)mu * a.Mv + c * a.Nq2 + g;
          out[gi] += sO[s * Cfg::SX + r];
        } else {
          const int m = r - NC * NQ;
          const int mx = m & 1, my = (m >> 1) & 1, mz = (DIM == 3) ? (m >> 2) : 0;
          const long g = (ex + mx) + a.g1[0] * ((ey + my) + a.g1[1] * (ez + mz));
          out[(long)K1 * a.Mv + (long)mu * a.Mp + g] += sOp[s * NP + m];
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace st
