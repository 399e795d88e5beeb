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
// class and processes it in batches of C cells, i.e. C*(k+1) "slots" (cell,
// Radau node) held in shared memory.  Stages (separated by __syncthreads):
//   S0  gather the nodal values of every slot (coalesced over slots);
//   S1  per (slot, component), in registers: values at the 3^d Gauss points
//       (one pass of the 3x3 Q2 basis matrix per direction) and the gradient in
//       collocation form (one pass of the collocation derivative per direction);
//   S3  per (slot, quadrature point): the pointwise work (coefficient cache,
//       tangent, convection, pressure; residual stress law) -> gradient-test
//       fluxes in place, pressure-test flux;
//   S4  per (slot, component), in registers: the K_t (x) M_x value term, the
//       transposed derivative chain and transposed value passes, then the
//       scatter-add straight from registers; per (slot, pressure node): the
//       pressure test.
// All FP64 arithmetic of S1/S4 runs on register-resident 3^d blocks with
// nine independent FMA chains per pass.  Boundary-face terms are a separate
// kernel (st_face.cuh) launched after the volume kernel of the same colour.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "st_internal.h"

namespace st {

// mesh-independent reference tables in constant memory (double and float)
struct ConstTables {
  double B[9], Bt[9], Dc[9], W[3], B1[6], E[6], ED[6];
  double BS[5], BtS[5];      // even/odd form of B, Bt (see rpass_sym)
  double WQ3[27], WQ2[9];    // tensor Gauss weights on the unit cell
  double PSI3[27 * 8], PSI2[9 * 4];  // Q1 basis at the cell Gauss points
  double FW3[9], FW2[3];     // tensor Gauss weights on a unit face
  double FPSI3[9 * 4], FPSI2[3 * 2]; // face Q1 basis at face points
};
struct ConstTablesF {
  float B[9], Bt[9], Dc[9], W[3], B1[6], E[6], ED[6];
  float BS[5], BtS[5];
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

// asynchronous element copy global -> shared (Ampere+ cp.async, 4 or 8 bytes)
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gmem_src) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem_dst);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(saddr), "l"(gmem_src));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr), "l"(gmem_src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// compile-time geometry of the 3-point lines of a 3^DIM block
template <int DIM, int DIR>
__device__ __forceinline__ constexpr int lbase(int l) {
  return DIM == 2 ? (DIR == 0 ? 3 * l : l) : (DIR == 0 ? 3 * l : (DIR == 1 ? (l % 3) + 9 * (l / 3) : l));
}
template <int DIR>
__device__ __forceinline__ constexpr int lstride() {
  return DIR == 0 ? 1 : (DIR == 1 ? 3 : 9);
}

// in-place pass of a register array along DIR: v <- M v on every line
template <int DIM, int DIR, typename T, typename MT>
__device__ __forceinline__ void rpass(T* v, const MT* m) {
  constexpr int NL = Dims<DIM>::NL, st = lstride<DIR>();
  const T m0 = (T)m[0], m1 = (T)m[1], m2 = (T)m[2], m3 = (T)m[3], m4 = (T)m[4], m5 = (T)m[5], m6 = (T)m[6],
          m7 = (T)m[7], m8 = (T)m[8];
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    const int b = lbase<DIM, DIR>(l);
    const T x0 = v[b], x1 = v[b + st], x2 = v[b + 2 * st];
    v[b] = m0 * x0 + m1 * x1 + m2 * x2;
    v[b + st] = m3 * x0 + m4 * x1 + m5 * x2;
    v[b + 2 * st] = m6 * x0 + m7 * x1 + m8 * x2;
  }
}

// in-place pass v <- M v along DIR for a centro-symmetric M (M[2-i][2-j] =
// M[i][j]) given in even/odd form cs = {(m00+m02)/2, (m00-m02)/2, m01, m10,
// m11}: with e = x0 + x2, o = x0 - x2 every line costs 8 FP operations
// instead of 9
template <int DIM, int DIR, typename T, typename MT>
__device__ __forceinline__ void rpass_sym(T* v, const MT* cs) {
  constexpr int NL = Dims<DIM>::NL, st = lstride<DIR>();
  const T s = (T)cs[0], t = (T)cs[1], m1 = (T)cs[2], m3 = (T)cs[3], m4 = (T)cs[4];
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    const int b = lbase<DIM, DIR>(l);
    const T x0 = v[b], x1 = v[b + st], x2 = v[b + 2 * st];
    const T e = x0 + x2, o = x0 - x2;
    const T c = fma(s, e, m1 * x1);
    v[b] = fma(t, o, c);
    v[b + st] = fma(m3, e, m4 * x1);
    v[b + 2 * st] = fma(-t, o, c);
  }
}

// dst <- D v along DIR (dst in shared memory) for a centro-antisymmetric D,
// whose centre entry is zero
template <int DIM, int DIR, typename T, typename MT>
__device__ __forceinline__ void rpass_out_d(const T* v, const MT* m, T* dst) {
  constexpr int NL = Dims<DIM>::NL, st = lstride<DIR>();
  const T m0 = (T)m[0], m1 = (T)m[1], m2 = (T)m[2], m3 = (T)m[3], m5 = (T)m[5], m6 = (T)m[6], m7 = (T)m[7],
          m8 = (T)m[8];
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    const int b = lbase<DIM, DIR>(l);
    const T x0 = v[b], x1 = v[b + st], x2 = v[b + 2 * st];
    dst[b] = fma(m2, x2, fma(m1, x1, m0 * x0));
    dst[b + st] = fma(m5, x2, m3 * x0);
    dst[b + 2 * st] = fma(m8, x2, fma(m7, x1, m6 * x0));
  }
}

// acc <- acc + D g along DIR (g in shared memory), D as in rpass_out_d
template <int DIM, int DIR, typename T, typename MT>
__device__ __forceinline__ void rpass_acc_d(T* acc, const MT* m, const T* g) {
  constexpr int NL = Dims<DIM>::NL, st = lstride<DIR>();
  const T m0 = (T)m[0], m1 = (T)m[1], m2 = (T)m[2], m3 = (T)m[3], m5 = (T)m[5], m6 = (T)m[6], m7 = (T)m[7],
          m8 = (T)m[8];
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    const int b = lbase<DIM, DIR>(l);
    const T x0 = g[b], x1 = g[b + st], x2 = g[b + 2 * st];
    acc[b] = fma(m2, x2, fma(m1, x1, fma(m0, x0, acc[b])));
    acc[b + st] = fma(m5, x2, fma(m3, x0, acc[b + st]));
    acc[b + 2 * st] = fma(m8, x2, fma(m7, x1, fma(m6, x0, acc[b + 2 * st])));
  }
}

// dst <- M v along DIR (dst in shared memory)
template <int DIM, int DIR, typename T, typename MT>
__device__ __forceinline__ void rpass_out(const T* v, const MT* m, T* dst) {
  constexpr int NL = Dims<DIM>::NL, st = lstride<DIR>();
  const T m0 = (T)m[0], m1 = (T)m[1], m2 = (T)m[2], m3 = (T)m[3], m4 = (T)m[4], m5 = (T)m[5], m6 = (T)m[6],
          m7 = (T)m[7], m8 = (T)m[8];
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    const int b = lbase<DIM, DIR>(l);
    const T x0 = v[b], x1 = v[b + st], x2 = v[b + 2 * st];
    dst[b] = m0 * x0 + m1 * x1 + m2 * x2;
    dst[b + st] = m3 * x0 + m4 * x1 + m5 * x2;
    dst[b + 2 * st] = m6 * x0 + m7 * x1 + m8 * x2;
  }
}

// acc <- acc + M g along DIR (g in shared memory)
template <int DIM, int DIR, typename T, typename MT>
__device__ __forceinline__ void rpass_acc(T* acc, const MT* m, const T* g) {
  constexpr int NL = Dims<DIM>::NL, st = lstride<DIR>();
  const T m0 = (T)m[0], m1 = (T)m[1], m2 = (T)m[2], m3 = (T)m[3], m4 = (T)m[4], m5 = (T)m[5], m6 = (T)m[6],
          m7 = (T)m[7], m8 = (T)m[8];
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    const int b = lbase<DIM, DIR>(l);
    const T x0 = g[b], x1 = g[b + st], x2 = g[b + 2 * st];
    acc[b] += m0 * x0 + m1 * x1 + m2 * x2;
    acc[b + st] += m3 * x0 + m4 * x1 + m5 * x2;
    acc[b + 2 * st] += m6 * x0 + m7 * x1 + m8 * x2;
  }
}

// Q1 nodal values (m = mx + 2 my + 4 mz) -> values at the 3^DIM Gauss points
// (q = qx + 3 qy + 9 qz), one 2 -> 3 pass per direction; B1 is [q][a]
template <int DIM, typename T, typename MT>
__device__ __forceinline__ void q1_to_gauss(const T* pn, const MT* B1, T* out) {
  const T b00 = (T)B1[0], b01 = (T)B1[1], b10 = (T)B1[2], b11 = (T)B1[3], b20 = (T)B1[4], b21 = (T)B1[5];
  constexpr int NZ = DIM == 3 ? 2 : 1, QZ = DIM == 3 ? 3 : 1;
  T t1[NZ][2][3], t2[NZ][3][3];
#pragma unroll
  for (int z = 0; z < NZ; ++z)
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      const T p0 = pn[2 * y + 4 * z], p1 = pn[1 + 2 * y + 4 * z];
      t1[z][y][0] = fma(b01, p1, b00 * p0);
      t1[z][y][1] = fma(b11, p1, b10 * p0);
      t1[z][y][2] = fma(b21, p1, b20 * p0);
    }
#pragma unroll
  for (int z = 0; z < NZ; ++z)
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      t2[z][0][x] = fma(b01, t1[z][1][x], b00 * t1[z][0][x]);
      t2[z][1][x] = fma(b11, t1[z][1][x], b10 * t1[z][0][x]);
      t2[z][2][x] = fma(b21, t1[z][1][x], b20 * t1[z][0][x]);
    }
#pragma unroll
  for (int y = 0; y < 3; ++y)
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      if constexpr (DIM == 3) {
        out[x + 3 * y] = fma(b01, t2[1][y][x], b00 * t2[0][y][x]);
        out[x + 3 * y + 9] = fma(b11, t2[1][y][x], b10 * t2[0][y][x]);
        out[x + 3 * y + 18] = fma(b21, t2[1][y][x], b20 * t2[0][y][x]);
      } else {
        out[x + 3 * y] = t2[0][y][x];
      }
    }
  (void)QZ;
}

// transpose of q1_to_gauss: out_m = sum_q psi_m(q) f(q)
template <int DIM, typename T, typename MT>
__device__ __forceinline__ void gauss_to_q1(const T* f, const MT* B1, T* out) {
  const T b00 = (T)B1[0], b01 = (T)B1[1], b10 = (T)B1[2], b11 = (T)B1[3], b20 = (T)B1[4], b21 = (T)B1[5];
  constexpr int NZ = DIM == 3 ? 2 : 1;
  T t2[NZ][3][3], t1[NZ][2][3];
#pragma unroll
  for (int y = 0; y < 3; ++y)
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      if constexpr (DIM == 3) {
        const T f0 = f[x + 3 * y], f1 = f[x + 3 * y + 9], f2 = f[x + 3 * y + 18];
        t2[0][y][x] = fma(b20, f2, fma(b10, f1, b00 * f0));
        t2[1][y][x] = fma(b21, f2, fma(b11, f1, b01 * f0));
      } else {
        t2[0][y][x] = f[x + 3 * y];
      }
    }
#pragma unroll
  for (int z = 0; z < NZ; ++z)
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      t1[z][0][x] = fma(b20, t2[z][2][x], fma(b10, t2[z][1][x], b00 * t2[z][0][x]));
      t1[z][1][x] = fma(b21, t2[z][2][x], fma(b11, t2[z][1][x], b01 * t2[z][0][x]));
    }
#pragma unroll
  for (int z = 0; z < NZ; ++z)
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      out[2 * y + 4 * z] = fma(b20, t1[z][y][2], fma(b10, t1[z][y][1], b00 * t1[z][y][0]));
      out[1 + 2 * y + 4 * z] = fma(b21, t1[z][y][2], fma(b11, t1[z][y][1], b01 * t1[z][y][0]));
    }
}

// colour-ordered index of a linear cell id (the coefficient caches use it)
template <int DIM>
__device__ __forceinline__ int colour_of(int ex, int ey, int ez) {
  return (ex & 1) | ((ey & 1) << 1) | (DIM == 3 ? ((ez & 1) << 2) : 0);
}

template <int DIM>
__device__ __forceinline__ long colour_index(const OpArgs& a, int cell) {
  const int ex = cell % a.n[0], ey = (cell / a.n[0]) % a.n[1], ez = (DIM == 3) ? cell / (a.n[0] * a.n[1]) : 0;
  const int c = (ex & 1) | ((ey & 1) << 1) | ((ez & 1) << 2);
  return a.col_start_all[c] + (ex >> 1) + (long)a.cn_all[c][0] * ((ey >> 1) + (long)a.cn_all[c][1] * (ez >> 1));
}

template <int DIM, int K1, typename T>
struct OpCfg {
  using D = Dims<DIM>;
  static constexpr int NT = DIM == 3 ? 128 : 128;  // threads per CTA (2 CTAs per SM: 2 warps per scheduler)
  static constexpr int SLOTS = DIM == 3 ? 36 : 64;  // target (cell, node) slots per batch
  static constexpr int C = SLOTS / K1 > 0 ? SLOTS / K1 : 1;
  static constexpr int S = C * K1;
  // per-slot shared arrays (elements of T): qp values, gradients/fluxes, nodal pressure, pressure-test flux
  static constexpr int SX = D::NC * D::NQ;
  static constexpr int SG = D::NC * DIM * D::NQ;
  static constexpr int SP = D::NP;
  static constexpr int SQ = D::NQ;
  static constexpr int per_slot = SX + SG + SP + SQ;
  // + per item: linear cell id, Q2 and Q1 grid index of the cell's first node, colour class
  static constexpr size_t smem_bytes =
      (size_t)S * per_slot * sizeof(T) + (size_t)S * sizeof(int) + 8 + (size_t)S * (2 * sizeof(long) + sizeof(int)) + 64;
};

// One batch of the volume kernel: nc items (cells in colour order; element-
// matrix mode: (cell, column) pairs) starting at b0, in the CTA's shared
// memory; sDd/sDdt/sM1 hold the scaled 1D matrices of the mesh of `a`.
template <int DIM, int K1, typename T, int MODE, int TAN>
__device__ __forceinline__ void op_batch(const OpArgs& a, const long b0, const int nc, unsigned char* smem_raw,
                                         const T (*sDd)[9], const T (*sDdt)[9], const T (*sM1)[9]) {
  using D = Dims<DIM>;
  using Cfg = OpCfg<DIM, K1, T>;
  constexpr int NQ = D::NQ, NC = D::NC, NP = D::NP, NS = D::NS;
  constexpr int S = Cfg::S;
  const auto& ct = CT<T>::t();
  T* sX = reinterpret_cast<T*>(smem_raw);
  T* sG = sX + S * Cfg::SX;
  T* sP = sG + S * Cfg::SG;
  T* sQ = sP + S * Cfg::SP;
  int* sCell = reinterpret_cast<int*>(sQ + S * Cfg::SQ);  // linear cell id of batch cell
  // the cell's first Q2 and Q1 node (grid index) and its colour class, so that
  // the per-element gathers and stores need no division by the mesh extents
  long* sB2 = reinterpret_cast<long*>((reinterpret_cast<uintptr_t>(sCell + S) + 7) & ~(uintptr_t)7);
  long* sB1 = sB2 + S;
  int* sCl = reinterpret_cast<int*>(sB1 + S);
  const T* in = reinterpret_cast<const T*>(a.in);
  constexpr int SK = (MODE == OP_ELM) ? 1 : K1;  // slots per batch item
  const int ns = nc * SK;
  (void)NS;

  // ---- batch setup: cell ids (element-matrix mode: item = (cell, column))
  for (int ci = threadIdx.x; ci < nc; ci += blockDim.x) {
    int ex, ey, ez;
    if constexpr (MODE == OP_ELM) {
      const int cell = (int)((b0 + ci) / D::NE);
      sCell[ci] = cell;
      ex = cell % a.n[0];
      ey = (cell / a.n[0]) % a.n[1];
      ez = (DIM == 3) ? cell / (a.n[0] * a.n[1]) : 0;
    } else {
      // colour-ordered cell index -> colour class c -> cell (o + 2 i, ...)
      long li = b0 + ci;
      int c = 0;
#pragma unroll
      for (int cc = 1; cc < (1 << DIM); ++cc) c += (li >= a.col_start_all[cc]) ? 1 : 0;
      li -= a.col_start_all[c];
      const int cn0 = a.cn_all[c][0], cn1 = a.cn_all[c][1];
      const int i = (int)(li % cn0);
      const int j = (int)((li / cn0) % cn1);
      const int l = (int)(li / ((long)cn0 * cn1));
      ex = (c & 1) + 2 * i;
      ey = ((c >> 1) & 1) + 2 * j;
      ez = (DIM == 3) ? ((c >> 2) & 1) + 2 * l : 0;
      sCell[ci] = ex + a.n[0] * (ey + a.n[1] * ez);
    }
    sB2[ci] = 2L * ex + a.g2[0] * (2L * ey + a.g2[1] * 2L * ez);
    sB1[ci] = (long)ex + a.g1[0] * ((long)ey + a.g1[1] * ez);
    sCl[ci] = colour_of<DIM>(ex, ey, ez);
  }
  __syncthreads();

  // ---- S0: gather nodal values of every slot (velocity, pressure) with
  //      asynchronous global->shared copies (all loads of the batch in flight);
  //      prefetch the batch's coefficient-cache block into L2 meanwhile
  for (int it = threadIdx.x; it < ns * (NC * NQ + NP); it += blockDim.x) {
    const int s = it / (NC * NQ + NP), r = it % (NC * NQ + NP);
    if constexpr (MODE == OP_ELM) {
      // unit vector e_j of the cell's local dofs (velocity c-major, then pressure)
      const int jcol = (int)((b0 + s) % D::NE);
      const T v = (r == jcol) ? (T)1 : (T)0;
      if (r < NC * NQ) sX[s * Cfg::SX + r] = v;
      else sP[s * NP + (r - NC * NQ)] = v;
      continue;
    }
    const int ci = s / K1, mu = s % K1;
    const int cell = sCell[ci];
    const T* src;
    T* dst;
    if (r < NC * NQ) {
      const int c = r / NQ, q = r % NQ;
      const int qx = q % 3, qy = (q / 3) % 3, qz = (DIM == 3) ? q / 9 : 0;
      const long g = sB2[ci] + qx + a.g2[0] * (qy + a.g2[1] * qz);
      src = in + (long)mu * a.Mv + c * a.Nq2 + g;
      dst = sX + s * Cfg::SX + r;
    } else {
      const int m = r - NC * NQ;
      dst = sP + s * NP + m;
      if (a.pdisc) {
        // P1disc: the value at vertex m of the cell's affine pressure (pdisc_T)
        const T* pc = in + (long)K1 * a.Mv + (long)mu * a.Mp + (long)cell * (DIM + 1);
        T v = pc[0];
#pragma unroll
        for (int j = 1; j <= DIM; ++j) v += ((m >> (j - 1)) & 1) ? pc[j] : -pc[j];
        *dst = v;
        continue;
      }
      const int mx = m & 1, my = (m >> 1) & 1, mz = (DIM == 3) ? (m >> 2) : 0;
      const long g = sB1[ci] + mx + a.g1[0] * (my + a.g1[1] * mz);
      src = in + (long)K1 * a.Mv + (long)mu * a.Mp + g;
    }
    cp_async_elem<T>(dst, src);
  }
  cp_async_commit();
  if constexpr (MODE == OP_JAC) {
    const char* cb = reinterpret_cast<const char*>(a.cache) +
                     (size_t)(a.col_start + b0) * K1 * D::NF_VOL * NQ * sizeof(T);
    const size_t nbytes = (size_t)ns * D::NF_VOL * NQ * sizeof(T);
    for (size_t off = (size_t)threadIdx.x * 128; off < nbytes; off += (size_t)blockDim.x * 128)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(cb + off));
  }
  cp_async_wait_all();
  __syncthreads();

  // ---- S1: per (slot, component), in registers: values at the Gauss points
  //      (Q2 basis, one pass per direction), then the gradient in collocation
  //      form; per slot: the pressure at the Gauss points (Q1 basis) into sQ
  constexpr int NPI = (MODE == OP_LIN) ? 0 : 1;  // pressure items per slot
  for (int it = threadIdx.x; it < ns * (NC + NPI); it += blockDim.x) {
    if (it >= ns * NC) {
      const int s = it - ns * NC;
      T pn[NP], pq[NQ];
#pragma unroll
      for (int m = 0; m < NP; ++m) pn[m] = sP[s * NP + m];
      q1_to_gauss<DIM>(pn, ct.B1, pq);
#pragma unroll
      for (int q = 0; q < NQ; ++q) sQ[s * NQ + q] = pq[q];
      continue;
    }
    const int s = it / NC, c = it % NC;
    T* xs = sX + s * Cfg::SX + c * NQ;
    T v[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = xs[q];
    rpass_sym<DIM, 0>(v, ct.BS);
    rpass_sym<DIM, 1>(v, ct.BS);
    if constexpr (DIM == 3) rpass_sym<DIM, 2>(v, ct.BS);
#pragma unroll
    for (int q = 0; q < NQ; ++q) xs[q] = v[q];
    T* gs = sG + s * Cfg::SG + c * DIM * NQ;
    rpass_out_d<DIM, 0>(v, sDd[0], gs);
    rpass_out_d<DIM, 1>(v, sDd[1], gs + NQ);
    if constexpr (DIM == 3) rpass_out_d<DIM, 2>(v, sDd[2], gs + 2 * NQ);
  }
  __syncthreads();

  // ---- S3: pointwise work at every quadrature point of every slot
  for (int it = threadIdx.x; it < ns * NQ; it += blockDim.x) {
    const int s = it / NQ, q = it % NQ;
    const int ci = s / SK, mu = (MODE == OP_ELM) ? a.elm_mu : s % SK;
    const long gidx = (MODE == OP_ELM) ? colour_index<DIM>(a, sCell[ci]) : a.col_start + b0 + ci;  // colour-ordered cell index
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
    } else if constexpr (MODE == OP_JAC || MODE == OP_ELM) {
      const T* cp = reinterpret_cast<const T*>(a.cache) + ((gidx * K1 + mu) * (long)D::NF_VOL) * NQ + q;
      const T etaw = cp[0];
      T nuw[3] = {0, 0, 0};
#pragma unroll
      for (int c = 0; c < NC; ++c) nuw[c] = cp[(2 + NS + c) * NQ];
      const T dpi = sQ[s * NQ + q];  // pressure increment at q (S1)
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
      sQ[s * NQ + q] = -div * tw;  // pressure test flux
    } else {  // OP_RES: F = RHS - LHS, gradient-test flux -(S(Du) - u (x) u - pi I)
      const T pi = sQ[s * NQ + q];  // pressure at q (S1)
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
      sQ[s * NQ + q] = div * tw;
    }
  }
  __syncthreads();

  if constexpr (MODE != OP_LIN) {
    // ---- S4: per (slot, component), in registers: K_t (x) M_x value term,
    //      transposed derivative chain, transposed value passes, nodal value
    //      terms (residual), scatter-add; per (slot, pressure node): pressure test
    for (int it = threadIdx.x; it < ns * (NC + 1); it += blockDim.x) {
      if (it < ns * NC) {
        const int s = it / NC, c = it % NC;
        const int ci = s / SK, mu = (MODE == OP_ELM) ? a.elm_mu : s % SK;
        T acc[NQ];
        if constexpr (MODE == OP_JAC) {
          // tv_mu(q) = W(q) sum_j (K_t vol)_{mu j} du_j(q)
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            T t = (T)a.KtV[mu * K1] * sX[(ci * K1) * Cfg::SX + c * NQ + q];
#pragma unroll
            for (int j = 1; j < K1; ++j) t += (T)a.KtV[mu * K1 + j] * sX[(ci * K1 + j) * Cfg::SX + c * NQ + q];
            acc[q] = t * ((DIM == 3) ? ct.WQ3[q] : ct.WQ2[q]);
          }
        } else {
#pragma unroll
          for (int q = 0; q < NQ; ++q) acc[q] = 0;
        }
        const T* gs = sG + s * Cfg::SG + c * DIM * NQ;
        rpass_acc_d<DIM, 0>(acc, sDdt[0], gs);
        rpass_acc_d<DIM, 1>(acc, sDdt[1], gs + NQ);
        if constexpr (DIM == 3) rpass_acc_d<DIM, 2>(acc, sDdt[2], gs + 2 * NQ);
        rpass_sym<DIM, 0>(acc, ct.BtS);
        rpass_sym<DIM, 1>(acc, ct.BtS);
        if constexpr (DIM == 3) rpass_sym<DIM, 2>(acc, ct.BtS);
        const int cell = sCell[ci];
        if constexpr (MODE == OP_RES) {
          // value terms in nodal form: M_e (-sum_j K_ij u_j + m_i v^- + tau w_i f_i)
          const T* vp = reinterpret_cast<const T*>(a.vprev);
          const T* ff = reinterpret_cast<const T*>(a.f);
          T y[NQ];
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            const int qx = q % 3, qy = (q / 3) % 3, qz = (DIM == 3) ? q / 9 : 0;
            const long gn = sB2[ci] + qx + a.g2[0] * (qy + a.g2[1] * qz) + c * a.Nq2;
            T t = vp ? (T)a.mt[mu] * vp[gn] : (T)0;
#pragma unroll
            for (int j = 0; j < K1; ++j) t -= (T)a.Kt[mu * K1 + j] * in[(long)j * a.Mv + gn];
            if (ff) t += (T)a.tw[mu] * ff[(long)mu * a.Mv + gn];
            y[q] = t;
          }
          rpass<DIM, 0>(y, sM1[0]);
          rpass<DIM, 1>(y, sM1[1]);
          if constexpr (DIM == 3) rpass<DIM, 2>(y, sM1[2]);
#pragma unroll
          for (int q = 0; q < NQ; ++q) acc[q] += y[q];
        }
        if constexpr (MODE == OP_ELM) {
          // column j of the element matrix (rows: velocity c-major, then pressure)
          const long item = b0 + s;
          T* E = reinterpret_cast<T*>(a.out) + ((long)cell * a.elm_stride + a.elm_slot) * D::NE * D::NE + item % D::NE;
#pragma unroll
          for (int q = 0; q < NQ; ++q) E[(long)(c * NQ + q) * D::NE] = acc[q];
          continue;
        }
        // plain stores into the private buffer of the cell's colour class:
        // cells of one class share no node, so no two threads write the same
        // entry; st_cbuf_sum adds the classes' buffers afterwards
        T* ob = reinterpret_cast<T*>(a.cbuf) + (long)sCl[ci] * a.cbuf_stride + (long)mu * a.Mv + c * a.Nq2 + sB2[ci];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const int qx = q % 3, qy = (q / 3) % 3, qz = (DIM == 3) ? q / 9 : 0;
          ob[qx + a.g2[0] * (qy + a.g2[1] * qz)] = acc[q];
        }
      } else {
        // pressure test of the slot, sum-factorised (transposed Q1 passes)
        const int s = it - ns * NC;
        const int ci = s / SK, mu = (MODE == OP_ELM) ? a.elm_mu : s % SK;
        T fq[NQ], pt[NP];
#pragma unroll
        for (int q = 0; q < NQ; ++q) fq[q] = sQ[s * NQ + q];
        gauss_to_q1<DIM>(fq, ct.B1, pt);
        const int cell = sCell[ci];
        if constexpr (MODE == OP_ELM) {
          const long item = b0 + s;
          T* E = reinterpret_cast<T*>(a.out) + ((long)cell * a.elm_stride + a.elm_slot) * D::NE * D::NE + item % D::NE;
#pragma unroll
          for (int m = 0; m < NP; ++m) E[(long)(NC * NQ + m) * D::NE] = pt[m];
          continue;
        }
        T* pb = reinterpret_cast<T*>(a.cbuf) + (long)sCl[ci] * a.cbuf_stride + (long)K1 * a.Mv + (long)mu * a.Mp;
        if (a.pdisc) {
          // P1disc tests: T^T times the vertex tests, at the cell's own coefficients
#pragma unroll
          for (int j = 0; j <= DIM; ++j) {
            T t = 0;
#pragma unroll
            for (int m = 0; m < NP; ++m) t += (j == 0 || ((m >> (j - 1)) & 1)) ? pt[m] : -pt[m];
            pb[(long)cell * (DIM + 1) + j] = t;
          }
          continue;
        }
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          const int mx = m & 1, my = (m >> 1) & 1, mz = (DIM == 3) ? (m >> 2) : 0;
          pb[sB1[ci] + mx + a.g1[0] * (my + a.g1[1] * mz)] = pt[m];
        }
      }
    }
  }
  __syncthreads();
}

template <int DIM, int K1, typename T, int MODE, int TAN>
__global__ void __launch_bounds__(OpCfg<DIM, K1, T>::NT) st_op_kernel(const OpArgs a) {
  using Cfg = OpCfg<DIM, K1, T>;
  constexpr int C = Cfg::C, S = Cfg::S;
  extern __shared__ __align__(16) unsigned char smem_raw[];

  // balanced chunk of the colour-ordered cells (element-matrix mode: of the items)
  const long ncol = a.ncol;
  const long cbeg = (long)blockIdx.x * ncol / gridDim.x;
  const long cend = (long)(blockIdx.x + 1) * ncol / gridDim.x;

  // scaled derivative and mass matrices in the precision of the kernel
  __shared__ T sDd[3][9], sDdt[3][9], sM1[3][9];
  if (threadIdx.x < 27) {
    const int d = threadIdx.x / 9, e = threadIdx.x % 9;
    sDd[d][e] = (T)a.Dd[d][e];
    sDdt[d][e] = (T)a.Ddt[d][e];
    sM1[d][e] = (T)a.M1d[d][e];
  }
  __syncthreads();

  constexpr int CB = (MODE == OP_ELM) ? S : C;  // items per batch
  for (long b0 = cbeg; b0 < cend; b0 += CB)
    op_batch<DIM, K1, T, MODE, TAN>(a, b0, (int)min((long)CB, cend - b0), smem_raw, sDd, sDdt, sM1);
}

// Many independent slab problems in one persistent launch: descs[i] is the
// argument block of instance i (same dim and k, any mesh and parameters);
// item t of the work queue is cell batch t - first[i] of the instance i with
// first[i] <= t < first[i+1].  A CTA keeps the block of its current instance
// in shared memory.
template <int DIM, int K1, typename T, int MODE, int TAN>
__global__ void __launch_bounds__(OpCfg<DIM, K1, T>::NT)
    st_op_kernel_batch(const OpArgs* __restrict__ descs, const long* __restrict__ first, int ninst,
                       unsigned* __restrict__ queue) {
  using Cfg = OpCfg<DIM, K1, T>;
  constexpr int C = Cfg::C;
  static_assert(MODE != OP_ELM, "element matrices are built per instance");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ OpArgs sA;
  __shared__ T sDd[3][9], sDdt[3][9], sM1[3][9];
  __shared__ long sItem;
  __shared__ int sInst;
  const long nitems = first[ninst];
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      const long t = (long)atomicAdd(queue, 1u);
      int lo = 0, hi = ninst;  // first[lo] <= t < first[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (first[mid] <= t) lo = mid;
        else hi = mid;
      }
      sItem = t;
      sInst = lo;
    }
    __syncthreads();
    const long t = sItem;
    const int i = sInst;
    if (t >= nitems) break;
    if (i != cur) {
      const unsigned* src = reinterpret_cast<const unsigned*>(descs + i);
      unsigned* dst = reinterpret_cast<unsigned*>(&sA);
      for (int w = threadIdx.x; w < (int)(sizeof(OpArgs) / sizeof(unsigned)); w += blockDim.x) dst[w] = src[w];
      __syncthreads();
      if (threadIdx.x < 27) {
        const int d = threadIdx.x / 9, e = threadIdx.x % 9;
        sDd[d][e] = (T)sA.Dd[d][e];
        sDdt[d][e] = (T)sA.Ddt[d][e];
        sM1[d][e] = (T)sA.M1d[d][e];
      }
      __syncthreads();
      cur = i;
    }
    const long b0 = (t - first[i]) * C;
    op_batch<DIM, K1, T, MODE, TAN>(sA, b0, (int)min((long)C, sA.ncol - b0), smem_raw, sDd, sDdt, sM1);
  }
}

}  // namespace st
