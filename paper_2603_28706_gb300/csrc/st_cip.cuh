// Convection-aligned CIP stabilisation on the interior faces (eq. scip-def):
//   s(uhat; u, v) = sum_F gamma_CIP h_F^2 (|uhat.n_F| [d_n u], [d_n v])_F
// at every Radau node with the weight tau w_mu of M_t.  n_F = e_a on the faces
// normal to axis a, [w] = w on the upper cell minus w on the lower one, h_F the
// face diameter (diagonal), 3-point Gauss quadrature per tangential direction.
//
// Three kernels:
//   st_cip_weights  gamma_CIP h_F^2 |uhat_a| x face-quadrature weight x tau w_mu
//                   at the Gauss points of every interior face, from the velocity
//                   of a slab vector (the linearisation state for the lagged
//                   Jacobian, Sec. 4.2-4.4; the argument itself for the residual).
//                   Layout w[((a * ncells + upper cell) * K1 + mu) * NFQ + g],
//                   g = g1 + 3 g2 along the face's tangential axes in increasing
//                   order; entries of cells on the lower boundary stay zero.
//   st_cip_face     every interior face once: the jump of d_n u at the face
//                   Gauss points, weighted and tested against the face-plane
//                   nodes (9 values per face, component and node, into a face
//                   buffer); one thread per (cell, component, node) does the
//                   faces below its cell.
//   st_cip_apply    one thread per (cell, component, node): the jump of a test
//                   function is the difference of its one-sided traces, so the
//                   cell adds sign_K d_n phi_i|K times the face values to its own
//                   nodes (sign_K = +1 on its lower face, where it is the upper
//                   cell, -1 on its upper face), and adds the result into the
//                   private buffer of the cell's colour class after the volume
//                   kernel has stored there: cells of one class share no node.
#pragma once

#include "st_operator.cuh"

namespace st {

// local node (3^DIM block, x fastest) of index i along AX and p1, p2 along the
// tangential axes t1 < t2 of AX
template <int AX>
__device__ __forceinline__ constexpr int cip_lnode(int i, int p1, int p2) {
  return (AX == 0 ? i : p1) + 3 * (AX == 1 ? i : (AX == 0 ? p1 : p2)) + 9 * (AX == 2 ? i : p2);
}

// offset of a local node of a cell from the cell's first Q2 node
__device__ __forceinline__ long cip_goff(const OpArgs& a, int q) {
  return (q % 3) + a.g2[0] * (((q / 3) % 3) + a.g2[1] * (q / 9));
}

// tangential passes over a face's 3 x 3 (3D) or 3 (2D) values with the 3 x 3
// matrix m: t1 first (stride 1), then t2 (stride 3)
template <int DIM, typename T, typename M>
__device__ __forceinline__ void cip_tpass(T* x, const M* m) {
  if constexpr (DIM == 3) {
#pragma unroll
    for (int l = 0; l < 3; ++l) apply3<T, M>(m, x[3 * l], x[3 * l + 1], x[3 * l + 2], x[3 * l], x[3 * l + 1], x[3 * l + 2]);
#pragma unroll
    for (int l = 0; l < 3; ++l) apply3<T, M>(m, x[l], x[l + 3], x[l + 6], x[l], x[l + 3], x[l + 6]);
  } else {
    apply3<T, M>(m, x[0], x[1], x[2], x[0], x[1], x[2]);
  }
}

template <int DIM, int K1, typename T>
__global__ void st_cip_weights(const OpArgs a, const T* __restrict__ U, T* __restrict__ w) {
  constexpr int NFQ = Dims<DIM>::NFQ;
  const auto& ct = CT<T>::t();
  const long nc = (long)a.n[0] * a.n[1] * (DIM == 3 ? a.n[2] : 1);
  const long total = (long)DIM * nc * K1;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int mu = (int)(t % K1);
    const long r = t / K1;
    const long cell = r % nc;
    const int ax = (int)(r / nc);
    const int e3[3] = {(int)(cell % a.n[0]), (int)((cell / a.n[0]) % a.n[1]),
                       DIM == 3 ? (int)(cell / ((long)a.n[0] * a.n[1])) : 0};
    T* wo = w + t * NFQ;
    if ((ax == 0 ? e3[0] : (ax == 1 ? e3[1] : e3[2])) == 0) {
#pragma unroll
      for (int g = 0; g < NFQ; ++g) wo[g] = (T)0;
      continue;
    }
    // node strides along the tangential axes t1 < t2
    const long s1 = ax == 0 ? a.g2[0] : 1, s2 = ax == 2 ? a.g2[0] : a.g2[0] * a.g2[1];
    const long base = 2L * e3[0] + a.g2[0] * (2L * e3[1] + a.g2[1] * 2L * e3[2]);
    const T* ua = U + (long)mu * a.Mv + (long)ax * a.Nq2 + base;
    T v[NFQ];
#pragma unroll
    for (int tn = 0; tn < NFQ; ++tn) {
      const int p1 = tn % 3, p2 = DIM == 3 ? tn / 3 : 0;
      v[tn] = ua[p1 * s1 + (DIM == 3 ? p2 * s2 : 0)];
    }
    cip_tpass<DIM>(v, ct.B);
    double hF2 = 0.0, area = 1.0;
#pragma unroll
    for (int b = 0; b < DIM; ++b)
      if (b != ax) {
        hF2 += a.h[b] * a.h[b];
        area *= a.h[b];
      }
    const T scale = (T)(a.gcip * hF2 * area * a.tw[mu]);
#pragma unroll
    for (int g = 0; g < NFQ; ++g) {
      const T fw = (T)ct.W[g % 3] * (DIM == 3 ? (T)ct.W[g / 3] : (T)1);
      wo[g] = scale * fw * fabs(v[g]);
    }
  }
}

// Per interior face normal to AX (index = its upper cell), component c and
// node mu: the weighted jump tested against the face-plane nodes,
//   f = B^T (w o B [d_n u]),   [d_n u] = d_n u|upper - d_n u|lower at the
// face-plane nodes, B the Q2 values at the tangential Gauss points.  Both
// cells' tests are +-(d_n phi) expansions of f, formed by st_cip_apply.
// Layout fb[(((AX * K1 + mu) * DIM + c) * NFQ + tn) * ncells + upper cell].
template <int DIM, int K1, typename T, int AX>
__device__ __forceinline__ void cip_face_values(const OpArgs& a, const T* __restrict__ x, const T* __restrict__ w,
                                                T* __restrict__ fb, long cell, long nc, const int* e3, int c, int mu) {
  constexpr int NFQ = Dims<DIM>::NFQ;
  const auto& ct = CT<T>::t();
  const long s[3] = {1, a.g2[0], a.g2[0] * a.g2[1]};
  const long base = 2L * e3[0] + a.g2[0] * (2L * e3[1] + a.g2[1] * 2L * e3[2]);
  const T* xu = x + base;                // upper cell (this one)
  const T* xl = x + base - 2 * s[AX];    // lower cell
  const T ih = (T)a.ih[AX];
  T j[NFQ];
#pragma unroll
  for (int tn = 0; tn < NFQ; ++tn) {
    const int p1 = tn % 3, p2 = DIM == 3 ? tn / 3 : 0;
    T du = 0, dl = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int q = cip_lnode<AX>(i, p1, p2);
      du += (T)ct.ED[i] * xu[cip_goff(a, q)];
      dl += (T)ct.ED[3 + i] * xl[cip_goff(a, q)];
    }
    j[tn] = (du - dl) * ih;
  }
  cip_tpass<DIM>(j, ct.B);
  const T* wf = w + (((long)AX * nc + cell) * K1 + mu) * NFQ;
#pragma unroll
  for (int g = 0; g < NFQ; ++g) j[g] *= wf[g];
  cip_tpass<DIM>(j, ct.Bt);
  T* o = fb + ((((long)AX * K1 + mu) * DIM + c) * NFQ) * nc + cell;
#pragma unroll
  for (int tn = 0; tn < NFQ; ++tn) o[(long)tn * nc] = j[tn];
}

// one thread per (cell, component, node): the faces below the cell in every
// direction (the cell is their upper cell)
template <int DIM, int K1, typename T>
__global__ void __launch_bounds__(128) st_cip_face(const OpArgs a, const T* __restrict__ w, T* __restrict__ fb) {
  const long nc = (long)a.n[0] * a.n[1] * (DIM == 3 ? a.n[2] : 1);
  const long total = nc * DIM * K1;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long cell = t % nc;
    const int r = (int)(t / nc), c = r % DIM, mu = r / DIM;
    const int e3[3] = {(int)(cell % a.n[0]), (int)((cell / a.n[0]) % a.n[1]),
                       DIM == 3 ? (int)(cell / ((long)a.n[0] * a.n[1])) : 0};
    const T* x = reinterpret_cast<const T*>(a.in) + (long)mu * a.Mv + (long)c * a.Nq2;
    if (e3[0] > 0) cip_face_values<DIM, K1, T, 0>(a, x, w, fb, cell, nc, e3, c, mu);
    if (e3[1] > 0) cip_face_values<DIM, K1, T, 1>(a, x, w, fb, cell, nc, e3, c, mu);
    if constexpr (DIM == 3)
      if (e3[2] > 0) cip_face_values<DIM, K1, T, 2>(a, x, w, fb, cell, nc, e3, c, mu);
  }
}

// the cell's test of the face normal to AX on its lower (UP = 0: the cell is
// the upper cell, sign +) or upper side (sign -): y += sign d_n phi_i f
template <int DIM, int K1, typename T, int AX, int UP>
__device__ __forceinline__ void cip_expand(const OpArgs& a, const T* __restrict__ fb, T* y, long cell, long nc,
                                           const int* e3, int c, int mu) {
  constexpr int NFQ = Dims<DIM>::NFQ;
  if constexpr (AX < DIM) {
    if (UP == 0 ? e3[AX] == 0 : e3[AX] == a.n[AX] - 1) return;  // boundary face
    const auto& ct = CT<T>::t();
    const long cs[3] = {1, a.n[0], (long)a.n[0] * a.n[1]};
    const T* f = fb + ((((long)AX * K1 + mu) * DIM + c) * NFQ) * nc + (UP ? cell + cs[AX] : cell);
    const T ih = (T)a.ih[AX];
#pragma unroll
    for (int tn = 0; tn < NFQ; ++tn) {
      const int p1 = tn % 3, p2 = DIM == 3 ? tn / 3 : 0;
      const T v = UP ? -f[(long)tn * nc] : f[(long)tn * nc];
#pragma unroll
      for (int i = 0; i < 3; ++i) y[cip_lnode<AX>(i, p1, p2)] += (T)ct.ED[UP * 3 + i] * ih * v;
    }
  }
}

template <int DIM, int K1, typename T>
__global__ void __launch_bounds__(128) st_cip_apply(const OpArgs a, const T* __restrict__ fb, T sgn) {
  constexpr int NQ = Dims<DIM>::NQ;
  const long nc = (long)a.n[0] * a.n[1] * (DIM == 3 ? a.n[2] : 1);
  const long total = nc * DIM * K1;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long cell = t % nc;
    const int r = (int)(t / nc), c = r % DIM, mu = r / DIM;
    const int e3[3] = {(int)(cell % a.n[0]), (int)((cell / a.n[0]) % a.n[1]),
                       DIM == 3 ? (int)(cell / ((long)a.n[0] * a.n[1])) : 0};
    const long base = 2L * e3[0] + a.g2[0] * (2L * e3[1] + a.g2[1] * 2L * e3[2]);
    T y[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) y[q] = (T)0;
    cip_expand<DIM, K1, T, 0, 0>(a, fb, y, cell, nc, e3, c, mu);
    cip_expand<DIM, K1, T, 0, 1>(a, fb, y, cell, nc, e3, c, mu);
    cip_expand<DIM, K1, T, 1, 0>(a, fb, y, cell, nc, e3, c, mu);
    cip_expand<DIM, K1, T, 1, 1>(a, fb, y, cell, nc, e3, c, mu);
    cip_expand<DIM, K1, T, 2, 0>(a, fb, y, cell, nc, e3, c, mu);
    cip_expand<DIM, K1, T, 2, 1>(a, fb, y, cell, nc, e3, c, mu);
    T* ob = reinterpret_cast<T*>(a.cbuf) + (long)colour_of<DIM>(e3[0], e3[1], e3[2]) * a.cbuf_stride +
            (long)mu * a.Mv + (long)c * a.Nq2 + base;
#pragma unroll
    for (int q = 0; q < NQ; ++q) ob[cip_goff(a, q)] += sgn * y[q];
  }
}

}  // namespace st
