// Space-time multigrid preconditioner (Sec. 6.3): nested Q2/Q1 transfers,
// Galerkin coarse operators, exact and surrogate cell patches, batched
// Gauss-Jordan patch inverses, additive Vanka sweeps and the V-cycle.
//
// Data per level l (0 = coarsest, L = finest):
//   E_l   spatial element matrices (times tau w_mu) of every cell and node mu,
//         [ncells][K1][NE][NE]: on level L from the coefficient cache of the
//         current linearisation (volume by unit-vector probing of the
//         sum-factorised operator, faces directly), on l < L by Galerkin
//         coarsening E_l = sum_children P_c^T E_{l+1} P_c (exact for nested
//         spaces, identity in time, so A_l = P^T A_{l+1} P);
//   LU_l  explicit inverses (Gauss-Jordan, partial pivoting, column-major) of the cell patches
//         A_{l,K} = R_K A_l R_K^T (l < L) resp. the surrogate A~_{L,K}
//         (eq. surrogate-diag: every node's spatial block replaced by the one
//         at t_rep = slab midpoint, temporal matrices unchanged).
// Patch size N = (k+1) NE (all velocity and pressure dofs of the cell at all
// Radau nodes).  A Vanka step computes the defect r - A_l d once, solves all
// patches and adds omega times their corrections into d, colour class by
// colour class (cells of one class share no dof), eq. stmg-vanka-update.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "st_blas.cuh"
#include "st_coarse.cuh"
#include "st_internal.h"
#include "st_tune.h"

namespace st {

cudaError_t dispatch_elm_2d(const st_problem* h, const Level& L, const OpArgs& a, int prec, int tangent, void* E,
                            const int* bcells, int nbc);
cudaError_t dispatch_elm_3d(const st_problem* h, const Level& L, const OpArgs& a, int prec, int tangent, void* E,
                            const int* bcells, int nbc);

namespace {

constexpr int MAXN = 4 * 89;  // largest patch size (k = 3, 3D)

int ne_of(int dim) { return dim == 3 ? 3 * 27 + 8 : 2 * 9 + 4; }
// vertex-star patch dofs per time node: the 3^dim velocity nodes around the
// vertex (every component) and its pressure
int nev_of(int dim) { return dim == 3 ? 3 * 27 + 1 : 2 * 9 + 1; }
long n_vertices(const st_problem* h, const Level& L);

// ------------------------------------------------------------- transfers
// One direction of the nested prolongation on blocks of a tensor grid:
// input grid gi (coarse along dir), output grid go (fine along dir).  ORDER 2
// (Q2: 2nc+1 -> 4nc+1 points) or 1 (Q1: nc+1 -> 2nc+1).  Fine point i lies in
// coarse cell e = min(i / (2 ORDER), nc - 1) at local position r = i - 2 ORDER e.
template <typename T, int ORDER>
__global__ void prolong_pass(const T* __restrict__ x, T* __restrict__ y, int gi0, int gi1, int gi2, int dir, int nc,
                             int nblk, const double* __restrict__ P) {
  const int go[3] = {dir == 0 ? 2 * ORDER * nc + 1 : gi0, dir == 1 ? 2 * ORDER * nc + 1 : gi1,
                     dir == 2 ? 2 * ORDER * nc + 1 : gi2};
  const long nout = (long)go[0] * go[1] * go[2];
  const long nin = (long)gi0 * gi1 * gi2;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < nout * nblk; t += (long)gridDim.x * blockDim.x) {
    const long b = t / nout, r = t % nout;
    int idx[3] = {(int)(r % go[0]), (int)((r / go[0]) % go[1]), (int)(r / ((long)go[0] * go[1]))};
    const int i = idx[dir];
    int e = i / (2 * ORDER);
    if (e > nc - 1) e = nc - 1;
    const int loc = i - 2 * ORDER * e;
    T acc = 0;
    for (int aa = 0; aa <= ORDER; ++aa) {
      idx[dir] = ORDER * e + aa;
      const long src = idx[0] + (long)gi0 * (idx[1] + (long)gi1 * idx[2]);
      acc += (T)P[loc * (ORDER + 1) + aa] * x[b * nin + src];
    }
    y[t] = acc;
  }
}

// One direction of the restriction P^T (gather form): coarse point j collects
// every fine point whose coarse cell contains it.
template <typename T, int ORDER>
__global__ void restrict_pass(const T* __restrict__ x, T* __restrict__ y, int gi0, int gi1, int gi2, int dir, int nc,
                              int nblk, const double* __restrict__ P) {
  const int go[3] = {dir == 0 ? ORDER * nc + 1 : gi0, dir == 1 ? ORDER * nc + 1 : gi1, dir == 2 ? ORDER * nc + 1 : gi2};
  const long nout = (long)go[0] * go[1] * go[2];
  const long nin = (long)gi0 * gi1 * gi2;
  const int gid = dir == 0 ? gi0 : (dir == 1 ? gi1 : gi2);
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < nout * nblk; t += (long)gridDim.x * blockDim.x) {
    const long b = t / nout, r = t % nout;
    int idx[3] = {(int)(r % go[0]), (int)((r / go[0]) % go[1]), (int)(r / ((long)go[0] * go[1]))};
    const int j = idx[dir];
    T acc = 0;
    for (int i = 2 * j - 2 * ORDER; i <= 2 * j + 2 * ORDER; ++i) {
      if (i < 0 || i >= gid) continue;
      int e = i / (2 * ORDER);
      if (e > nc - 1) e = nc - 1;
      const int aa = j - ORDER * e;
      if (aa < 0 || aa > ORDER) continue;
      const int loc = i - 2 * ORDER * e;
      idx[dir] = i;
      const long src = idx[0] + (long)gi0 * (idx[1] + (long)gi1 * idx[2]);
      acc += (T)P[loc * (ORDER + 1) + aa] * x[b * nin + src];
    }
    y[t] = acc;
  }
}

// P1disc pressure transfers, cell by cell.  A child with offset o in {0,1}^d
// inside its parent holds the parent's affine pressure exactly: with the
// basis 1, 2 r_a - 1 on both cells, r_parent = (r_child + o) / 2, so
//   f_0 = c_0 + sum_a c_{1+a} (o_a - 1/2),   f_{1+a} = c_{1+a} / 2;
// the restriction is the transpose (summed over the 2^d children).
template <typename T, int DIM>
__global__ void pdisc_prolong(const T* __restrict__ xc, T* __restrict__ yf, int nfx, int nfy, int nfz, int K1) {
  const long ncf = (long)nfx * nfy * nfz, ncc = ncf >> DIM;
  const int ncx = nfx / 2, ncy = nfy / 2;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < ncf * K1; t += (long)gridDim.x * blockDim.x) {
    const int mu = (int)(t / ncf);
    const long f = t % ncf;
    const int fx = (int)(f % nfx), fy = (int)((f / nfx) % nfy), fz = (int)(f / ((long)nfx * nfy));
    const long c = (fx >> 1) + (long)ncx * ((fy >> 1) + (long)ncy * (DIM == 3 ? (fz >> 1) : 0));
    const int o[3] = {fx & 1, fy & 1, fz & 1};
    const T* cc = xc + ((long)mu * ncc + c) * (DIM + 1);
    T* ff = yf + ((long)mu * ncf + f) * (DIM + 1);
    T v = cc[0];
#pragma unroll
    for (int a = 0; a < DIM; ++a) v += cc[1 + a] * (T)(o[a] - 0.5);
    ff[0] = v;
#pragma unroll
    for (int a = 0; a < DIM; ++a) ff[1 + a] = cc[1 + a] * (T)0.5;
  }
}

template <typename T, int DIM>
__global__ void pdisc_restrict(const T* __restrict__ xf, T* __restrict__ yc, int ncx, int ncy, int ncz, int K1) {
  const long ncc = (long)ncx * ncy * ncz, ncf = ncc << DIM;
  const int nfx = 2 * ncx, nfy = 2 * ncy;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < ncc * K1; t += (long)gridDim.x * blockDim.x) {
    const int mu = (int)(t / ncc);
    const long c = t % ncc;
    const int cx = (int)(c % ncx), cy = (int)((c / ncx) % ncy), cz = (int)(c / ((long)ncx * ncy));
    T acc[DIM + 1];
#pragma unroll
    for (int j = 0; j <= DIM; ++j) acc[j] = 0;
    for (int ch = 0; ch < (1 << DIM); ++ch) {
      const int o[3] = {ch & 1, (ch >> 1) & 1, (ch >> 2) & 1};
      const long f = (2 * cx + o[0]) + (long)nfx * ((2 * cy + o[1]) + (long)nfy * (DIM == 3 ? 2 * cz + o[2] : 0));
      const T* ff = xf + ((long)mu * ncf + f) * (DIM + 1);
      acc[0] += ff[0];
#pragma unroll
      for (int a = 0; a < DIM; ++a) acc[1 + a] += ff[0] * (T)(o[a] - 0.5) + ff[1 + a] * (T)0.5;
    }
    T* cc = yc + ((long)mu * ncc + c) * (DIM + 1);
#pragma unroll
    for (int j = 0; j <= DIM; ++j) cc[j] = acc[j];
  }
}

// ------------------------------------------------------------- Galerkin
// E_c[cell][mu] = sum over the 2^d children of P_ch^T E_f[child][mu] P_ch, with
// P_ch the child-local-dof <- parent-local-dof prolongation (block diagonal:
// one tensor Q2 block per velocity component, one Q1 block for the pressure).
// Sum-factorised Galerkin coarsening.  The child prolongation is block
// diagonal with Kronecker blocks: per velocity component P2[oz] (x) P2[oy]
// (x) P2[ox] (3x3 1D blocks, rows child node, columns parent node), for the
// pressure P1[oz] (x) P1[oy] (x) P1[ox] (2x2), o the child's offset.  So
// T = E_f P applies P^T to every row segment and R += P^T T to every column
// segment, one 1D pass per direction (3^d x 3 instead of 3^d x 3^d FMA per
// segment).  One CTA per (coarse cell, node); E_f, T, R in shared memory.
template <int DIM, int N1, typename T>
__device__ __forceinline__ void kron_pass_t(T* v, const T (*m)[3][3], const int* off) {
  // v (N1^DIM, x fastest) <- (M_z (x) M_y (x) M_x)^T v, M_d = m[off[d]] (N1 x N1 used)
  constexpr int NT = DIM == 3 ? N1 * N1 * N1 : N1 * N1;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const int st = d == 0 ? 1 : (d == 1 ? N1 : N1 * N1);
    const T(*M)[3] = m[off[d]];
    T u[NT];
#pragma unroll
    for (int i = 0; i < NT; ++i) {
      const int ci = (i / st) % N1;  // output (parent) index along d
      const int base = i - ci * st;
      T acc = 0;
#pragma unroll
      for (int j = 0; j < N1; ++j) acc = fma(M[j][ci], v[base + j * st], acc);
      u[i] = acc;
    }
#pragma unroll
    for (int i = 0; i < NT; ++i) v[i] = u[i];
  }
}

// one segment of E (row r or column b) through P_seg^T; ld: stride between segment entries
template <int DIM, int N1, typename T, bool ACC>
__device__ __forceinline__ void galerkin_segment(const T* src, T* dst, int ld, const T (*m)[3][3], const int* off) {
  constexpr int NT = DIM == 3 ? N1 * N1 * N1 : N1 * N1;
  T v[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) v[j] = src[j * ld];
  kron_pass_t<DIM, N1, T>(v, m, off);
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    if (ACC) dst[j * ld] += v[j];
    else dst[j * ld] = v[j];
  }
}

template <int DIM, typename T>
__global__ void __launch_bounds__(256) galerkin_sf_kernel(const T* __restrict__ Ef, T* __restrict__ Ec, int ncx,
                                                          int ncy, int ncz, int K1, const double* __restrict__ tab) {
  constexpr int NQ = DIM == 3 ? 27 : 9, NC = DIM, NP = DIM == 3 ? 8 : 4, NE = NC * NQ + NP;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sE = reinterpret_cast<T*>(smraw);  // child matrix, row-major
  T* sT = sE + NE * NE;                  // E_f P
  T* sR = sT + NE * NE;                  // result
  __shared__ T p2[2][3][3], p1[2][3][3];  // [offset][child node][parent node] (p1 uses 2 x 2)
  if (threadIdx.x < 18) {
    const int o = threadIdx.x / 9, i = (threadIdx.x / 3) % 3, a = threadIdx.x % 3;
    p2[o][i][a] = (T)tab[(2 * o + i) * 3 + a];
    p1[o][i][a] = (i < 2 && a < 2) ? (T)tab[15 + (o + i) * 2 + a] : (T)0;
  }
  __syncthreads();
  const long ncell = (long)ncx * ncy * ncz;
  const int nfx = 2 * ncx, nfy = 2 * ncy;
  constexpr int NSEG = NC + 1;  // velocity component blocks + the pressure block
  for (long item = blockIdx.x; item < ncell * K1; item += gridDim.x) {
    const long cc = item / K1;
    const int mu = (int)(item % K1);
    const int cx = (int)(cc % ncx), cy = (int)((cc / ncx) % ncy), cz = (int)(cc / ((long)ncx * ncy));
    for (int i = threadIdx.x; i < NE * NE; i += blockDim.x) sR[i] = 0;
    for (int ch = 0; ch < (1 << DIM); ++ch) {
      const int off[3] = {ch & 1, (ch >> 1) & 1, (ch >> 2) & 1};
      const long fcell = (2 * cx + off[0]) + (long)nfx * ((2 * cy + off[1]) + (long)nfy * (DIM == 3 ? 2 * cz + off[2] : 0));
      const T* src = Ef + (fcell * K1 + mu) * NE * NE;
      for (int i = threadIdx.x; i < NE * NE; i += blockDim.x) sE[i] = src[i];
      __syncthreads();
      // T[r][seg] = P_seg^T E[r][seg]  (row segments)
      for (int t = threadIdx.x; t < NE * NSEG; t += blockDim.x) {
        const int r = t / NSEG, sg = t % NSEG;
        if (sg < NC) galerkin_segment<DIM, 3, T, false>(sE + r * NE + sg * NQ, sT + r * NE + sg * NQ, 1, p2, off);
        else galerkin_segment<DIM, 2, T, false>(sE + r * NE + NC * NQ, sT + r * NE + NC * NQ, 1, p1, off);
      }
      __syncthreads();
      // R[seg][b] += P_seg^T T[seg][b]  (column segments)
      for (int t = threadIdx.x; t < NE * NSEG; t += blockDim.x) {
        const int b = t / NSEG, sg = t % NSEG;
        if (sg < NC) galerkin_segment<DIM, 3, T, true>(sT + sg * NQ * NE + b, sR + sg * NQ * NE + b, NE, p2, off);
        else galerkin_segment<DIM, 2, T, true>(sT + NC * NQ * NE + b, sR + NC * NQ * NE + b, NE, p1, off);
      }
      __syncthreads();
    }
    T* dst = Ec + (cc * K1 + mu) * NE * NE;
    for (int i = threadIdx.x; i < NE * NE; i += blockDim.x) dst[i] = sR[i];
    __syncthreads();
  }
}

// ------------------------------------------------------- patch assembly
// A_K (N x N, column-major F[col][row]) for cell K:
//   block (mu, nu): K_t[mu][nu] M_K (velocity part) + delta_{mu nu} S_mu,
//   S_mu = sum over the neighbour cells e of K of E[e][mu] restricted to the
//   dofs of K (surrogate: S_mu = (w_mu / w_0) sum_e Erep[e]).
// Velocity dof (c, node a in {0,1,2}^d of K) is node a - 2 delta in a
// neighbour shifted by delta in {-1,0,1}^d; pressure node m is m - delta.
struct PatchArgs {
  int n[3];
  int K1;
  double Kt[16];
  double wr[4];        // w_mu / w_0 (surrogate) or 1
  double M1h[3][9];    // 1D Q2 mass matrices scaled by h
  int surrogate;
  int c13;             // surrogate patch diagonalised in time: nb complex blocks lambda_b M_v + S
  int nb;
  double lam[4][2];
  int pdisc;           // P1disc pressure: patch pressure dofs are the cell's coefficients, the
                       // element matrices' pressure part is in vertex form (pdisc_T)
};

// P1disc patch entry (row p, column q of a spatial block, one of them a
// pressure dof): the cell's own element matrix with its pressure rows and
// columns changed from vertex values to coefficients (T^T E T); local
// pressure dofs beyond the DIM+1 coefficients are unused and get an
// identity row, so the patch matrix stays invertible.  S[mu] as in
// patch_assemble (surrogate: w_mu / w_0 times the representative matrix).
template <int DIM, typename T>
__device__ void pdisc_patch_entry(const T* __restrict__ E, int estride, const PatchArgs& pa, long K, int p, int q,
                                  T* S) {
  constexpr int NQ = DIM == 3 ? 27 : 9, NC = DIM, NP = DIM == 3 ? 8 : 4, NE = NC * NQ + NP, NV = NC * NQ;
  const bool pp = p >= NV, pq = q >= NV;
  const int jp = p - NV, jq = q - NV;
  if ((pp && jp > DIM) || (pq && jq > DIM)) {
    for (int mu = 0; mu < pa.K1; ++mu) S[mu] = (p == q) ? (T)1 : (T)0;
    return;
  }
  const int nmat = pa.surrogate ? 1 : pa.K1;
  for (int s = 0; s < nmat; ++s) {
    const T* Em = E + ((K * estride) + (pa.surrogate ? 0 : s)) * (long)NE * NE;
    double v = 0.0;
    if (pp && pq) {
      for (int m = 0; m < NP; ++m)
        for (int m2 = 0; m2 < NP; ++m2)
          v += pdisc_T(m, jp) * (double)Em[(NV + m) * NE + NV + m2] * pdisc_T(m2, jq);
    } else if (pp) {
      for (int m = 0; m < NP; ++m) v += pdisc_T(m, jp) * (double)Em[(NV + m) * NE + q];
    } else {
      for (int m = 0; m < NP; ++m) v += (double)Em[p * NE + NV + m] * pdisc_T(m, jq);
    }
    if (pa.surrogate) {
      for (int mu = 0; mu < pa.K1; ++mu) S[mu] = (T)(pa.wr[mu] * v);
    } else {
      S[s] = (T)v;
    }
  }
}

template <int DIM>
__device__ __forceinline__ bool local_in(int dof, const int dl[3], int& out) {
  // dof of K -> local dof in the neighbour shifted by dl (false if not shared)
  constexpr int NQ = DIM == 3 ? 27 : 9, NC = DIM;
  if (dof < NC * NQ) {
    const int c = dof / NQ, n = dof % NQ;
    int ni[3] = {n % 3, (n / 3) % 3, n / 9};
    for (int d = 0; d < DIM; ++d) {
      ni[d] -= 2 * dl[d];
      if (ni[d] < 0 || ni[d] > 2) return false;
    }
    out = c * NQ + ni[0] + 3 * ni[1] + 9 * ni[2];
    return true;
  }
  const int m = dof - NC * NQ;
  int mi[3] = {m & 1, (m >> 1) & 1, m >> 2};
  for (int d = 0; d < DIM; ++d) {
    mi[d] -= dl[d];
    if (mi[d] < 0 || mi[d] > 1) return false;
  }
  out = NC * NQ + mi[0] + 2 * mi[1] + 4 * mi[2];
  return true;
}

template <int DIM, typename T>
__global__ void patch_assemble(const T* __restrict__ E, int estride, PatchArgs pa, T* __restrict__ F) {
  constexpr int NQ = DIM == 3 ? 27 : 9, NC = DIM, NE = NC * NQ + (DIM == 3 ? 8 : 4);
  const int K1 = pa.K1, N = K1 * NE;
  const long ncell = (long)pa.n[0] * pa.n[1] * (DIM == 3 ? pa.n[2] : 1);
  __shared__ double smass[NQ * NQ];  // element velocity mass (tensor of the 1D masses)
  for (int t = threadIdx.x; t < NQ * NQ; t += blockDim.x) {
    const int a = t / NQ, b = t % NQ;
    const int ai[3] = {a % 3, (a / 3) % 3, a / 9}, bi[3] = {b % 3, (b / 3) % 3, b / 9};
    double m = 1.0;
    for (int d = 0; d < DIM; ++d) m *= pa.M1h[d][ai[d] * 3 + bi[d]];
    smass[t] = m;
  }
  __syncthreads();
  for (long K = blockIdx.x; K < ncell; K += gridDim.x) {
    const int k3[3] = {(int)(K % pa.n[0]), (int)((K / pa.n[0]) % pa.n[1]),
                       DIM == 3 ? (int)(K / ((long)pa.n[0] * pa.n[1])) : 0};
    T* Fk = F + K * (pa.c13 ? (long)pa.nb * NE * NE * 2 : (long)N * N);
    for (int it = threadIdx.x; it < NE * NE; it += blockDim.x) {
      const int p = it / NE, q = it % NE;  // row, column within a spatial block
      // spatial block sums (per mu) and the velocity mass entry
      T S[4] = {0, 0, 0, 0};
      double mass = 0.0;
      const bool vel_pair = p < NC * NQ && q < NC * NQ && (p / NQ) == (q / NQ);
      // neighbour shifts that hold both dofs, per axis (bit delta + 1): a Q2
      // node index 0 / 1 / 2 lies in the shifts {-1, 0} / {0} / {0, 1}, a Q1
      // node index 0 / 1 in {-1, 0} / {0, 1}; the cells that do not are skipped
      // without their index arithmetic, in the same order as before
      int am[3] = {2, 2, 2};
      if (pa.pdisc && (p >= NC * NQ || q >= NC * NQ)) {
        pdisc_patch_entry<DIM, T>(E, estride, pa, K, p, q, S);
        am[0] = am[1] = am[2] = 0;  // no neighbour sums: the pressure dofs belong to K alone
      } else {
        int ip[3], iq[3];
        const bool vp = p < NC * NQ, vq = q < NC * NQ;
        const int np_ = vp ? p % NQ : p - NC * NQ, nq_ = vq ? q % NQ : q - NC * NQ;
        for (int d = 0; d < 3; ++d) {
          ip[d] = vp ? (d == 0 ? np_ % 3 : d == 1 ? (np_ / 3) % 3 : np_ / 9) : ((np_ >> d) & 1);
          iq[d] = vq ? (d == 0 ? nq_ % 3 : d == 1 ? (nq_ / 3) % 3 : nq_ / 9) : ((nq_ >> d) & 1);
        }
        for (int d = 0; d < DIM; ++d) {
          const int mp = vp ? (ip[d] == 0 ? 3 : ip[d] == 1 ? 2 : 6) : (ip[d] == 0 ? 3 : 6);
          const int mq = vq ? (iq[d] == 0 ? 3 : iq[d] == 1 ? 2 : 6) : (iq[d] == 0 ? 3 : 6);
          am[d] = mp & mq;
        }
      }
      for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz) {
        if (!((am[2] >> (dz + 1)) & 1)) continue;
        for (int dy = -1; dy <= 1; ++dy) {
          if (!((am[1] >> (dy + 1)) & 1)) continue;
          for (int dx = -1; dx <= 1; ++dx) {
            if (!((am[0] >> (dx + 1)) & 1)) continue;
            const int dl[3] = {dx, dy, dz};
            const int e3[3] = {k3[0] + dx, k3[1] + dy, k3[2] + dz};
            bool inside = true;
            for (int d = 0; d < DIM; ++d) inside = inside && e3[d] >= 0 && e3[d] < pa.n[d];
            if (!inside) continue;
            int lp, lq;
            if (!local_in<DIM>(p, dl, lp) || !local_in<DIM>(q, dl, lq)) continue;
            const long ecell = e3[0] + (long)pa.n[0] * (e3[1] + (long)pa.n[1] * e3[2]);
            if (pa.surrogate) {
              const T v = E[(ecell * estride) * NE * NE + (long)lp * NE + lq];
              for (int mu = 0; mu < K1; ++mu) S[mu] += (T)pa.wr[mu] * v;
            } else {
              for (int mu = 0; mu < K1; ++mu) S[mu] += E[(ecell * estride + mu) * NE * NE + (long)lp * NE + lq];
            }
            if (vel_pair) mass += smass[(lp % NQ) * NQ + (lq % NQ)];
          }
        }
      }
      if (pa.c13) {
        // block b: lambda_b M_v + S_0 (S_0: the surrogate block of node 0), complex, column-major
        for (int b = 0; b < pa.nb; ++b) {
          T* g = Fk + ((long)(b * NE + q) * NE + p) * 2;
          g[0] = S[0] + (vel_pair ? (T)(pa.lam[b][0] * mass) : (T)0);
          g[1] = vel_pair ? (T)(pa.lam[b][1] * mass) : (T)0;
        }
        continue;
      }
      for (int mu = 0; mu < K1; ++mu)
        for (int nu = 0; nu < K1; ++nu) {
          T v = (mu == nu) ? S[mu] : (T)0;
          if (vel_pair) v += (T)(pa.Kt[mu * K1 + nu] * mass);
          // column-major: F[col][row]
          Fk[(long)(nu * NE + q) * N + (mu * NE + p)] = v;
        }
    }
    __syncthreads();
  }
}

// Vertex-star patch of vertex v (patch_type = 1, exact patches only): per
// time node the velocity nodes with Q2 indices 2 v_a - 1 + j_a, j in {0,1,2}^d,
// that lie in the mesh (every component), then the pressure at v.  The spatial
// block sums the element matrices E[e][mu] of the 2^d cells e = v - 1 + o,
// o in {0,1}^d, around v; patch node j is local node j_a + 1 - 2 o_a of cell e
// and the vertex is local Q1 node 1 - o_a.  Dofs outside the mesh get an
// identity row and column.  Column-major F[col][row] as for cell patches.
template <int DIM>
__device__ __forceinline__ bool vertex_local(int dof, const int o[3], int& out) {
  constexpr int NQ = DIM == 3 ? 27 : 9, NC = DIM;
  if (dof == NC * NQ) {
    out = NC * NQ + (1 - o[0]) + 2 * (1 - o[1]) + (DIM == 3 ? 4 * (1 - o[2]) : 0);
    return true;
  }
  const int c = dof / NQ, n = dof % NQ;
  const int j[3] = {n % 3, (n / 3) % 3, n / 9};
  int l[3] = {0, 0, 0};
  for (int d = 0; d < DIM; ++d) {
    l[d] = j[d] + 1 - 2 * o[d];
    if (l[d] < 0 || l[d] > 2) return false;
  }
  out = c * NQ + l[0] + 3 * l[1] + 9 * l[2];
  return true;
}

template <int DIM>
__device__ __forceinline__ bool vertex_dof_in_mesh(int dof, const int v[3], const int n[3]) {
  constexpr int NQ = DIM == 3 ? 27 : 9, NC = DIM;
  if (dof == NC * NQ) return true;
  const int q = dof % NQ;
  const int j[3] = {q % 3, (q / 3) % 3, q / 9};
  for (int d = 0; d < DIM; ++d) {
    const int gi = 2 * v[d] - 1 + j[d];
    if (gi < 0 || gi > 2 * n[d]) return false;
  }
  return true;
}

template <int DIM, typename T>
__global__ void patch_assemble_vertex(const T* __restrict__ E, int estride, PatchArgs pa, T* __restrict__ F) {
  constexpr int NQ = DIM == 3 ? 27 : 9, NC = DIM, NE = NC * NQ + (DIM == 3 ? 8 : 4), NEV = NC * NQ + 1;
  const int K1 = pa.K1, N = K1 * NEV;
  const int nv0 = pa.n[0] + 1, nv1 = pa.n[1] + 1;
  const long nvert = (long)nv0 * nv1 * (DIM == 3 ? pa.n[2] + 1 : 1);
  __shared__ double smass[NQ * NQ];
  for (int t = threadIdx.x; t < NQ * NQ; t += blockDim.x) {
    const int a = t / NQ, b = t % NQ;
    const int ai[3] = {a % 3, (a / 3) % 3, a / 9}, bi[3] = {b % 3, (b / 3) % 3, b / 9};
    double m = 1.0;
    for (int d = 0; d < DIM; ++d) m *= pa.M1h[d][ai[d] * 3 + bi[d]];
    smass[t] = m;
  }
  __syncthreads();
  for (long V = blockIdx.x; V < nvert; V += gridDim.x) {
    const int v[3] = {(int)(V % nv0), (int)((V / nv0) % nv1), DIM == 3 ? (int)(V / ((long)nv0 * nv1)) : 0};
    T* Fv = F + V * (long)N * N;
    for (int it = threadIdx.x; it < NEV * NEV; it += blockDim.x) {
      const int p = it / NEV, q = it % NEV;  // row, column within a spatial block
      const bool inp = vertex_dof_in_mesh<DIM>(p, v, pa.n), inq = vertex_dof_in_mesh<DIM>(q, v, pa.n);
      const bool vel_pair = p < NC * NQ && q < NC * NQ && (p / NQ) == (q / NQ);
      T S[4] = {0, 0, 0, 0};
      double mass = 0.0;
      if (inp && inq) {
        for (int oc = 0; oc < (1 << DIM); ++oc) {
          const int o[3] = {oc & 1, (oc >> 1) & 1, (oc >> 2) & 1};
          int e3[3] = {0, 0, 0};
          bool inside = true;
          for (int d = 0; d < DIM; ++d) {
            e3[d] = v[d] - 1 + o[d];
            inside = inside && e3[d] >= 0 && e3[d] < pa.n[d];
          }
          int lp, lq;
          if (!inside || !vertex_local<DIM>(p, o, lp) || !vertex_local<DIM>(q, o, lq)) continue;
          const long ecell = e3[0] + (long)pa.n[0] * (e3[1] + (long)pa.n[1] * e3[2]);
          for (int mu = 0; mu < K1; ++mu) S[mu] += E[(ecell * estride + mu) * NE * NE + (long)lp * NE + lq];
          if (vel_pair) mass += smass[(lp % NQ) * NQ + (lq % NQ)];
        }
      }
      for (int mu = 0; mu < K1; ++mu)
        for (int nu = 0; nu < K1; ++nu) {
          T val;
          if (inp && inq) {
            val = (mu == nu) ? S[mu] : (T)0;
            if (vel_pair) val += (T)(pa.Kt[mu * K1 + nu] * mass);
          } else {
            val = (mu == nu && p == q) ? (T)1 : (T)0;
          }
          Fv[(long)(nu * NEV + q) * N + (mu * NEV + p)] = val;
        }
    }
    __syncthreads();
  }
}

// CIP restricted to the finest-level surrogate patches (eq. scip-def at the
// representative state): C_K = R_K S R_K^T with
//   S = sum_F sum_q w_{F,q} c_{F,q} c_{F,q}^T,
//   c_{F,q}[i] = d_n phi_i|upper cell(x_q) - d_n phi_i|lower cell(x_q),
// w the face weights at Radau node 0 (they carry tau w_0, as the surrogate
// element matrices do).  The faces whose cells share a node with K are the
// ones normal to axis a on the planes k_a - 1 .. k_a + 2 with tangential cell
// indices within one of K's.  C_K is the same for every velocity component;
// it is added to S_mu with the factor w_mu / w_0, or to S_0 of every
// time-diagonalised block.  One CTA per patch: the jump coefficients of the
// face's quadrature points at K's nodes go to shared memory, each thread
// accumulates up to three entries of C_K.
struct CipPatchArgs {
  int n[3];
  int K1, nb, c13;
  double ih[3];
  double ED[6], B[9];
  double wr[4];
};

template <int DIM, typename T>
__global__ void __launch_bounds__(256) cip_patch_add(CipPatchArgs ca, const double* __restrict__ w,
                                                     T* __restrict__ F) {
  constexpr int NQ = DIM == 3 ? 27 : 9, NC = DIM, NE = NC * NQ + (DIM == 3 ? 8 : 4), NFQ = DIM == 3 ? 9 : 3;
  constexpr int R = (NQ * NQ + 255) / 256;
  const int K1 = ca.K1, N = K1 * NE;
  const long ncell = (long)ca.n[0] * ca.n[1] * (DIM == 3 ? ca.n[2] : 1);
  __shared__ double sc[NFQ][NQ];
  __shared__ double sw[NFQ];
  for (long K = blockIdx.x; K < ncell; K += gridDim.x) {
    const int k3[3] = {(int)(K % ca.n[0]), (int)((K / ca.n[0]) % ca.n[1]),
                       DIM == 3 ? (int)(K / ((long)ca.n[0] * ca.n[1])) : 0};
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    for (int ax = 0; ax < DIM; ++ax) {
      const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
      for (int P = k3[ax] - 1; P <= k3[ax] + 2; ++P) {
        if (P < 1 || P > ca.n[ax] - 1) continue;  // boundary planes carry no CIP
        for (int d2 = (DIM == 3 ? -1 : 0); d2 <= (DIM == 3 ? 1 : 0); ++d2)
          for (int d1 = -1; d1 <= 1; ++d1) {
            int u3[3] = {0, 0, 0};
            u3[ax] = P;
            u3[t1] = k3[t1] + d1;
            if (DIM == 3) u3[t2] = k3[t2] + d2;
            if (u3[t1] < 0 || u3[t1] >= ca.n[t1]) continue;
            if (DIM == 3 && (u3[t2] < 0 || u3[t2] >= ca.n[t2])) continue;
            __syncthreads();  // the previous face's coefficients are consumed
            for (int it = threadIdx.x; it < NFQ * NQ; it += blockDim.x) {
              const int q = it / NQ, i = it % NQ;
              const int g1 = q % 3, g2 = DIM == 3 ? q / 3 : 0;
              const int li[3] = {i % 3, (i / 3) % 3, i / 9};
              int lu[3], ll[3];
              bool in_u = true, in_l = true;
              for (int d = 0; d < 3; ++d) {
                const int G = 2 * k3[d] + li[d];
                lu[d] = d < DIM ? G - 2 * u3[d] : 0;
                ll[d] = d < DIM ? G - 2 * (u3[d] - (d == ax ? 1 : 0)) : 0;
                in_u = in_u && lu[d] >= 0 && lu[d] <= 2;
                in_l = in_l && ll[d] >= 0 && ll[d] <= 2;
              }
              double c = 0.0;
              if (in_u) c += ca.ED[lu[ax]] * ca.B[g1 * 3 + lu[t1]] * (DIM == 3 ? ca.B[g2 * 3 + lu[t2]] : 1.0);
              if (in_l) c -= ca.ED[3 + ll[ax]] * ca.B[g1 * 3 + ll[t1]] * (DIM == 3 ? ca.B[g2 * 3 + ll[t2]] : 1.0);
              sc[q][i] = c * ca.ih[ax];
            }
            if (threadIdx.x < NFQ) {
              const long up = u3[0] + (long)ca.n[0] * (u3[1] + (long)ca.n[1] * u3[2]);
              sw[threadIdx.x] = w[(((long)ax * ncell + up) * K1) * NFQ + threadIdx.x];
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const int e = threadIdx.x + 256 * r;
              if (e < NQ * NQ) {
                const int a = e / NQ, b = e % NQ;
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < NFQ; ++q) s += sw[q] * sc[q][a] * sc[q][b];
                acc[r] += s;
              }
            }
          }
      }
    }
    T* Fk = F + K * (ca.c13 ? (long)ca.nb * NE * NE * 2 : (long)N * N);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = threadIdx.x + 256 * r;
      if (e >= NQ * NQ) continue;
      const int a = e / NQ, b = e % NQ;
      for (int c = 0; c < NC; ++c) {
        const int pr = c * NQ + a, pc = c * NQ + b;
        if (ca.c13) {
          for (int blk = 0; blk < ca.nb; ++blk) Fk[((long)(blk * NE + pc) * NE + pr) * 2] += (T)acc[r];
        } else {
          for (int mu = 0; mu < K1; ++mu) Fk[(long)(mu * NE + pc) * N + (mu * NE + pr)] += (T)(ca.wr[mu] * acc[r]);
        }
      }
    }
  }
}

// Colour classes of a level for one launch over all its cells in colour
// order: class c holds the cells (c_x + 2 i, c_y + 2 j, c_z + 2 l); cells of
// one class share no dof, so each class writes its own buffer (cb + c*stride)
// with plain stores and colour_sum adds the buffers afterwards.
struct ColourMap {
  long start[9];
  int cn[8][3];
  int nclass;
};

__device__ __forceinline__ void colour_cell(const ColourMap& cm, long li, int& c, int& ex, int& ey, int& ez) {
  c = 0;
  for (int cc = 1; cc < cm.nclass; ++cc) c += (li >= cm.start[cc]) ? 1 : 0;
  const long r = li - cm.start[c];
  ex = (c & 1) + 2 * (int)(r % cm.cn[c][0]);
  ey = ((c >> 1) & 1) + 2 * (int)((r / cm.cn[c][0]) % cm.cn[c][1]);
  ez = ((c >> 2) & 1) + 2 * (int)(r / ((long)cm.cn[c][0] * cm.cn[c][1]));
}

// y = (accumulate ? y : 0) + alpha sum_c cb[c * stride + i]
template <typename T>
__global__ void colour_sum(const T* __restrict__ cb, long stride, int ncls, T* __restrict__ y, long n, T alpha,
                           int accumulate) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    T acc = cb[i];
    for (int c = 1; c < ncls; ++c) acc += cb[c * stride + i];
    y[i] = (accumulate ? y[i] : (T)0) + alpha * acc;
  }
}

// ------------------------------------------------------- batched inverse
// In-place Gauss-Jordan inversion with partial (row) pivoting of `count`
// matrices of size N stored column-major (F[col][row]); one CTA per matrix.
// Step k: pivot row p = argmax_{i>=k} |a_ik| (lowest index on ties), swap rows
// k and p, scale row k by 1/a_kk with the pivot entry replaced by 1, and
// subtract multiples of it from every other row, with column k replaced by
// zero first.  After the last step the columns are permuted back in reverse
// pivot order, which leaves A^{-1}.  A zero pivot sets err[0].
template <typename T>
__global__ void gj_invert_kernel(T* __restrict__ F, int* __restrict__ piv, int N, long count,
                                 int* __restrict__ err) {
  __shared__ int s_piv;
  __shared__ T s_val[256];
  __shared__ int s_idx[256];
  __shared__ T s_row[MAXN], s_col[MAXN];
  for (long m = blockIdx.x; m < count; m += gridDim.x) {
    T* A = F + m * (long)N * N;
    int* pv = piv + m * N;
    for (int k = 0; k < N; ++k) {
      T best = -1;
      int bi = k;
      for (int i = k + threadIdx.x; i < N; i += blockDim.x) {
        const T v = fabs(A[(long)k * N + i]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
      s_val[threadIdx.x] = best;
      s_idx[threadIdx.x] = bi;
      __syncthreads();
      for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
          const T o = s_val[threadIdx.x + w];
          const int oi = s_idx[threadIdx.x + w];
          if (o > s_val[threadIdx.x] || (o == s_val[threadIdx.x] && oi < s_idx[threadIdx.x])) {
            s_val[threadIdx.x] = o;
            s_idx[threadIdx.x] = oi;
          }
        }
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        s_piv = s_idx[0];
        pv[k] = s_piv;
        if (!(s_val[0] > 0)) atomicExch(err, 1);
      }
      __syncthreads();
      const int p = s_piv;
      const T d = A[(long)k * N + p];
      const T inv = d != (T)0 ? (T)1 / d : (T)0;
      // pivot row (swapped into k) scaled, pivot entry -> 1/d; multipliers of column k
      for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const T rk = A[(long)j * N + p];
        if (p != k) A[(long)j * N + p] = A[(long)j * N + k];
        s_row[j] = (j == k ? (T)1 : rk) * inv;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < N; i += blockDim.x) s_col[i] = (i == k) ? (T)0 : A[(long)k * N + i];
      __syncthreads();
      for (long t = threadIdx.x; t < (long)N * N; t += blockDim.x) {
        const int j = (int)(t / N), i = (int)(t % N);
        T* aij = A + t;
        if (i == k) *aij = s_row[j];
        else *aij = (j == k ? (T)0 : *aij) - s_col[i] * s_row[j];
      }
      __syncthreads();
    }
    for (int k = N - 1; k >= 0; --k) {
      const int p = pv[k];
      if (p != k)
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
          const T t = A[(long)k * N + i];
          A[(long)k * N + i] = A[(long)p * N + i];
          A[(long)p * N + i] = t;
        }
      __syncthreads();
    }
  }
}

// Register-resident Gauss-Jordan inversion (FP32, N <= 32 RPL and N <= NW CPW)
// with partial pivoting done implicitly: step k picks the pivot row p_k of
// largest |a_ik| among the rows not yet used (lowest index on ties) and
// applies the exchange step on (p_k, k) without moving rows,
//   a_pj <- a_pj / d (j != k),  a_pk <- 1/d,
//   a_ij <- a_ij - a_ik a_pj / d (i != p, j != k),  a_ik <- -a_ik / d,
// d = a_pk.  After all N steps the stored M satisfies
// (A^{-1})[k][p_j] = M[p_k][j], which the write-out applies through shared
// memory.  Thread (lane, warp) holds rows lane + 32 r and columns
// warp + NW c, so column k lies in one warp (warp-local pivot search) and the
// pivot row is a shared-memory broadcast.  One CTA of 32 NW threads per matrix.
template <int RPL, int CPW, int NW, typename R, bool STAGE>
__global__ void __launch_bounds__(32 * NW) gj_invert_reg_kernel(R* __restrict__ F, int* __restrict__ piv, int N,
                                                                long count, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char gr_raw[];
  R* S = reinterpret_cast<R*>(gr_raw);                    // N x N staging of the result (STAGE)
  R* s_col = S + (STAGE ? (size_t)N * N : 0);             // column k before the step
  R* s_row = s_col + 32 * RPL;                            // pivot row before the step
  int* s_used = reinterpret_cast<int*>(s_row + NW * CPW); // row already a pivot
  int* s_kinv = s_used + 32 * RPL;                        // step whose pivot row is i
  int* s_pv = s_kinv + 32 * RPL;                          // pivot row of step k
  __shared__ int s_p;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (long m = blockIdx.x; m < count; m += gridDim.x) {
    const R* G = F + m * (long)N * N;
    R a[RPL][CPW];
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      const int j = w + NW * c;
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int i = lane + 32 * r;
        a[r][c] = (i < N && j < N) ? G[(long)j * N + i] : (R)0;
      }
    }
    for (int i = threadIdx.x; i < 32 * RPL; i += blockDim.x) s_used[i] = (i < N) ? 0 : 1;
    __syncthreads();
    for (int k = 0; k < N; ++k) {
      const int wk = k % NW, ck = k / NW;
      if (w == wk) {
        // pivot search over the unused rows of column k; column k to shared memory
        R best = (R)-1;
        int bi = 0x7fffffff;
#pragma unroll
        for (int c = 0; c < CPW; ++c)
          if (c == ck) {
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
              const int i = lane + 32 * r;
              const R v = a[r][c];
              s_col[i] = v;
              if (i < N && !s_used[i]) {
                if (bi == 0x7fffffff) bi = i;  // a valid row even if every candidate is NaN
                if (fabs(v) > best) {
                  best = fabs(v);
                  bi = i;
                }
              }
            }
          }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const R ov = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ov > best || (ov == best && oi < bi)) {
            best = ov;
            bi = oi;
          }
        }
        if (lane == 0) {
          s_p = bi;
          s_used[bi] = 1;
          s_kinv[bi] = k;
          s_pv[k] = bi;
          if (!(best > (R)0)) atomicExch(err, 1);
        }
      }
      __syncthreads();
      const int p = s_p, lp = p & 31, rp = p >> 5;
      if (lane == lp) {
#pragma unroll
        for (int r = 0; r < RPL; ++r)
          if (r == rp) {
#pragma unroll
            for (int c = 0; c < CPW; ++c) s_row[w + NW * c] = a[r][c];
          }
      }
      __syncthreads();
      const R inv = (R)1 / s_row[k];
      R rj[CPW], f[RPL];
#pragma unroll
      for (int c = 0; c < CPW; ++c) rj[c] = s_row[w + NW * c] * inv;
#pragma unroll
      for (int r = 0; r < RPL; ++r) f[r] = s_col[lane + 32 * r];
      if (lane == lp) {
#pragma unroll
        for (int r = 0; r < RPL; ++r)
          if (r == rp) f[r] = (R)0;  // the pivot row is set below
      }
      if (w == wk) {
#pragma unroll
        for (int c = 0; c < CPW; ++c)
          if (c == ck) {
            rj[c] = inv;
#pragma unroll
            for (int r = 0; r < RPL; ++r) a[r][c] = (R)0;  // new column k: -a_ik / d
          }
      }
#pragma unroll
      for (int r = 0; r < RPL; ++r)
#pragma unroll
        for (int c = 0; c < CPW; ++c) a[r][c] = fma(-f[r], rj[c], a[r][c]);
      if (lane == lp) {
#pragma unroll
        for (int r = 0; r < RPL; ++r)
          if (r == rp) {
#pragma unroll
            for (int c = 0; c < CPW; ++c) a[r][c] = rj[c];  // pivot row a_pj / d, a_pk = 1/d
          }
      }
      __syncthreads();
    }
    // (A^{-1})[s_kinv[i]][s_pv[j]] = M[i][j]: staged column-major in S, or
    // written in place (every thread has read its entries before the steps)
    R* Go = F + m * (long)N * N;
    R* D = STAGE ? S : Go;
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      const int j = w + NW * c;
      if (j < N) {
        const int dc = s_pv[j];
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          const int i = lane + 32 * r;
          if (i < N) D[(long)dc * N + s_kinv[i]] = a[r][c];
        }
      }
    }
    __syncthreads();
    if (STAGE)
      for (long t = threadIdx.x; t < (long)N * N; t += blockDim.x) Go[t] = S[t];
    for (int k = threadIdx.x; k < N; k += blockDim.x) piv[m * N + k] = s_pv[k];
    __syncthreads();
  }
}

template <int RPL, int CPW, typename R, bool STAGE>
cudaError_t launch_gj_reg_t(R* F, int* piv, int N, long count, int* err, int nsm, cudaStream_t st) {
  constexpr int NW = 16;
  const size_t sm = (STAGE ? (size_t)N * N * sizeof(R) : 0) + (32 * RPL + NW * CPW) * sizeof(R) +
                    3 * 32 * RPL * sizeof(int);
  auto kern = gj_invert_reg_kernel<RPL, CPW, NW, R, STAGE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int occ = 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * NW, sm);
  if (e != cudaSuccess) return e;
  const long cap = (long)(occ > 0 ? occ : 1) * nsm;
  const unsigned g = (unsigned)(count < cap ? count : cap);
  kern<<<g, 32 * NW, sm, st>>>(F, piv, N, count, err);
  return cudaGetLastError();
}

// staged write-out when the N x N result fits in shared memory, else in place
template <int RPL, int CPW, typename R>
cudaError_t launch_gj_reg(R* F, int* piv, int N, long count, int* err, int nsm, cudaStream_t st) {
  if ((size_t)N * N * sizeof(R) + 8192 <= 227 * 1024)
    return launch_gj_reg_t<RPL, CPW, R, true>(F, piv, N, count, err, nsm, st);
  return launch_gj_reg_t<RPL, CPW, R, false>(F, piv, N, count, err, nsm, st);
}

// patches of the sizes that occur (3D k = 0, 1; 2D k = 0..2) go to the
// register kernel; true if it was launched
template <typename R>
inline bool try_gj_reg(R* F, int* piv, int N, long count, int* err, int nsm, cudaStream_t st, cudaError_t& e) {
  if (N <= 64 && N <= 16 * 4) { e = launch_gj_reg<2, 4>(F, piv, N, count, err, nsm, st); return true; }
  if (N <= 96) { e = launch_gj_reg<3, 6>(F, piv, N, count, err, nsm, st); return true; }
  if (N <= 192) { e = launch_gj_reg<6, 12>(F, piv, N, count, err, nsm, st); return true; }
  return false;
}

// The register Gauss-Jordan inversion (implicit pivoting, see
// gj_invert_reg_kernel) for complex matrices stored as interleaved (re, im)
// pairs, column-major; R = float or double; pivot: largest |a_ik|^2 (lowest
// row on ties).  Two barriers per elimination step: the warp that owns
// column k+1 updates it first and then searches the next pivot while the
// other warps finish their updates; pivot column, pivot row and pivot index
// are double-buffered by step parity.
template <int RPL, int CPW, int NW, typename R>
__device__ __forceinline__ void gj_cplx_search(const R (&ar)[RPL][CPW], const R (&ai)[RPL][CPW], int c_own, int N,
                                               int lane, int k, int* s_used, int* s_kinv, int* s_pv, R* s_col,
                                               int* s_pb, int* err) {
  R best = (R)-1;
  int bi = 0x7fffffff;
#pragma unroll
  for (int c = 0; c < CPW; ++c)
    if (c == c_own) {
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int i = lane + 32 * r;
        s_col[2 * i] = ar[r][c];
        s_col[2 * i + 1] = ai[r][c];
        if (i < N && !s_used[i]) {
          if (bi == 0x7fffffff) bi = i;
          const R v = ar[r][c] * ar[r][c] + ai[r][c] * ai[r][c];
          if (v > best) {
            best = v;
            bi = i;
          }
        }
      }
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const R ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  if (lane == 0) {
    *s_pb = bi;
    s_used[bi] = 1;
    s_kinv[bi] = k;
    s_pv[k] = bi;
    if (!(best > (R)0)) atomicExch(err, 1);
  }
}

template <int RPL, int CPW, int NW, typename R, int MINB = 1>
__global__ void __launch_bounds__(32 * NW, MINB) gj_invert_reg_cplx(R* __restrict__ F, int N, long count,
                                                                    int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char gc_raw[];
  R* S = reinterpret_cast<R*>(gc_raw);                          // 2 N^2 staging of the result
  R* s_col = S + 2 * (size_t)N * N;                              // column k, two buffers of 2 x 32 RPL
  R* s_row = s_col + 4 * 32 * RPL;                               // pivot row, two buffers of 2 x NW CPW
  int* s_used = reinterpret_cast<int*>(s_row + 4 * NW * CPW);
  int* s_kinv = s_used + 32 * RPL;
  int* s_pv = s_kinv + 32 * RPL;
  __shared__ int s_p[2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (long m = blockIdx.x; m < count; m += gridDim.x) {
    const R* G = F + m * 2 * (long)N * N;
    R ar[RPL][CPW], ai[RPL][CPW];
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      const int j = w + NW * c;
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int i = lane + 32 * r;
        const bool in = i < N && j < N;
        ar[r][c] = in ? G[((long)j * N + i) * 2] : (R)0;
        ai[r][c] = in ? G[((long)j * N + i) * 2 + 1] : (R)0;
      }
    }
    for (int i = threadIdx.x; i < 32 * RPL; i += blockDim.x) s_used[i] = (i < N) ? 0 : 1;
    __syncthreads();
    if (w == 0) gj_cplx_search<RPL, CPW, NW, R>(ar, ai, 0, N, lane, 0, s_used, s_kinv, s_pv, s_col, &s_p[0], err);
    __syncthreads();
    for (int k = 0; k < N; ++k) {
      const int b = k & 1, wk = k % NW, ck = k / NW;
      R* colb = s_col + b * 2 * 32 * RPL;
      R* rowb = s_row + b * 2 * NW * CPW;
      const int p = s_p[b], lp = p & 31, rp = p >> 5;
      if (lane == lp) {
#pragma unroll
        for (int r = 0; r < RPL; ++r)
          if (r == rp) {
#pragma unroll
            for (int c = 0; c < CPW; ++c) {
              rowb[2 * (w + NW * c)] = ar[r][c];
              rowb[2 * (w + NW * c) + 1] = ai[r][c];
            }
          }
      }
      __syncthreads();
      const R dr = rowb[2 * k], di = rowb[2 * k + 1], dn = dr * dr + di * di;
      const R ir = dr / dn, ii = -di / dn;  // 1 / d
      R fr[RPL], fi[RPL];
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        fr[r] = colb[2 * (lane + 32 * r)];
        fi[r] = colb[2 * (lane + 32 * r) + 1];
      }
      if (lane == lp) {
#pragma unroll
        for (int r = 0; r < RPL; ++r)
          if (r == rp) {
            fr[r] = 0;
            fi[r] = 0;
          }
      }
      if (w == wk) {
#pragma unroll
        for (int c = 0; c < CPW; ++c)
          if (c == ck) {
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
              ar[r][c] = 0;
              ai[r][c] = 0;
            }
          }
      }
#pragma unroll
      for (int c = 0; c < CPW; ++c) {
        const int j = w + NW * c;
        R xr = rowb[2 * j], xi = rowb[2 * j + 1];
        if (j == k) {
          xr = 1;
          xi = 0;
        }
        const R rr = xr * ir - xi * ii, ri = xr * ii + xi * ir;  // a_pj / d (1/d at j = k)
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          ar[r][c] = fma(-fr[r], rr, fma(fi[r], ri, ar[r][c]));
          ai[r][c] = fma(-fr[r], ri, fma(-fi[r], rr, ai[r][c]));
        }
        if (lane == lp) {
#pragma unroll
          for (int r = 0; r < RPL; ++r)
            if (r == rp) {
              ar[r][c] = rr;
              ai[r][c] = ri;
            }
        }
      }
      // the owner of column k+1 searches the next pivot on its updated column
      if (k + 1 < N && w == (k + 1) % NW)
        gj_cplx_search<RPL, CPW, NW, R>(ar, ai, (k + 1) / NW, N, lane, k + 1, s_used, s_kinv, s_pv,
                                        s_col + (b ^ 1) * 2 * 32 * RPL, &s_p[b ^ 1], err);
      __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      const int j = w + NW * c;
      if (j < N) {
        const int dc = s_pv[j];
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          const int i = lane + 32 * r;
          if (i < N) {
            S[((long)dc * N + s_kinv[i]) * 2] = ar[r][c];
            S[((long)dc * N + s_kinv[i]) * 2 + 1] = ai[r][c];
          }
        }
      }
    }
    __syncthreads();
    R* Go = F + m * 2 * (long)N * N;
    for (long t = threadIdx.x; t < 2 * (long)N * N; t += blockDim.x) Go[t] = S[t];
    __syncthreads();
  }
}

template <int RPL, int CPW, int NW, int MINB, typename R>
cudaError_t launch_gj_cplx(R* F, int N, long count, int* err, int nsm, cudaStream_t st) {
  auto kern = gj_invert_reg_cplx<RPL, CPW, NW, R, MINB>;
  const size_t sm = 2 * (size_t)N * N * sizeof(R) + 4 * (32 * RPL + NW * CPW) * sizeof(R) + 3 * 32 * RPL * sizeof(int);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int occ = 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * NW, sm);
  if (e != cudaSuccess) return e;
  const long cap = (long)(occ > 0 ? occ : 1) * nsm;
  const unsigned g = (unsigned)(count < cap ? count : cap);
  kern<<<g, 32 * NW, sm, st>>>(F, N, count, err);
  return cudaGetLastError();
}

// complex patches of the time-diagonalised surrogate (N = NE: 22 in 2D, 89 in
// 3D).  3D FP32: 8 warps per matrix with the registers capped for two CTAs per
// SM (122 registers, no spills), so that one CTA's pivot search and barriers
// overlap the other's updates; FP64 keeps 16 warps per matrix (its 8-warp
// form would spill).
template <typename R>
cudaError_t invert_patches_cplx(R* F, int N, long count, int* err, int nsm, cudaStream_t st) {
  if (N <= 32) return launch_gj_cplx<1, 2, 16, 1, R>(F, N, count, err, nsm, st);
  if (N > 96) return cudaErrorInvalidValue;
  if constexpr (sizeof(R) == 4) return launch_gj_cplx<3, 12, 8, 2, R>(F, N, count, err, nsm, st);
  else return launch_gj_cplx<3, 6, 16, 1, R>(F, N, count, err, nsm, st);
}

// Time-diagonalised surrogate patch solve (see TimeEig), all patches in one
// launch: s_b = sum_mu tin[b][mu] r_mu, z_b = G_b^{-1} s_b (complex, explicit
// inverse), x_mu = sum_b Re(tout[b][mu] z_b) into the cell's colour buffer.
struct VankaC13 {
  int nb;
  double tin[MAX_K1][MAX_K1][2], tout[MAX_K1][MAX_K1][2];
};

template <int DIM, typename T>
__global__ void vanka_patch_solve_c13(const T* __restrict__ G, VankaC13 vc, int K1, const T* __restrict__ defect,
                                      T* __restrict__ cb, long cstride, int n0, int n1, int n2, ColourMap cm,
                                      long li0, long nli, long Nq2, long Nq1, long Mv, long Mp, int pdisc,
                                      T* __restrict__ dd, T omega) {
  constexpr int NQ = DIM == 3 ? 27 : 9, NC = DIM, NP = DIM == 3 ? 8 : 4, NE = NC * NQ + NP;
  const int N = K1 * NE, nb = vc.nb;
  __shared__ T sx[MAXN];
  __shared__ long sg[MAXN];
  __shared__ T ss[MAX_K1][NE][2], sz[MAX_K1][NE][2];
  const long g2x = 2L * n0 + 1, g2y = 2L * n1 + 1, g1x = (long)n0 + 1, g1y = (long)n1 + 1;
  for (long li = li0 + blockIdx.x; li < li0 + nli; li += gridDim.x) {
    int col, ex, ey, ez;
    colour_cell(cm, li, col, ex, ey, ez);
    const long cell = ex + (long)n0 * (ey + (long)n1 * ez);
    T* ob = cb + col * cstride;
    const T* Gk = G + cell * (long)nb * NE * NE * 2;
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      const int mu = r / NE, loc = r % NE;
      long g;
      if (loc < NC * NQ) {
        const int c = loc / NQ, q = loc % NQ;
        g = (long)mu * Mv + c * Nq2 + (2L * ex + q % 3) + g2x * ((2L * ey + (q / 3) % 3) + g2y * (2L * ez + q / 9));
      } else {
        const int m = loc - NC * NQ;
        if (pdisc) {  // the cell's P1disc coefficients; patch dofs beyond them are unused
          g = m <= DIM ? (long)K1 * Mv + (long)mu * Mp + cell * (DIM + 1) + m : -1;
        } else {
          g = (long)K1 * Mv + (long)mu * Mp + (ex + (m & 1)) + g1x * ((ey + ((m >> 1) & 1)) + g1y * (ez + (m >> 2)));
        }
      }
      sg[r] = g;
      sx[r] = g >= 0 ? defect[g] : (T)0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nb * NE; t += blockDim.x) {
      const int b = t / NE, q = t % NE;
      T re = 0, im = 0;
      for (int mu = 0; mu < K1; ++mu) {
        const T x = sx[mu * NE + q];
        re += (T)vc.tin[b][mu][0] * x;
        im += (T)vc.tin[b][mu][1] * x;
      }
      ss[b][q][0] = re;
      ss[b][q][1] = im;
    }
    __syncthreads();
    // two threads (adjacent lanes) per output row, each over every other
    // column; the loop runs over whole warps (blockDim is a multiple of 32) so
    // that every lane takes part in the pair shuffle
    const int total = 2 * nb * NE, padded = (total + 31) & ~31;
    for (int t = threadIdx.x; t < padded; t += blockDim.x) {
      const bool act = t < total;
      const int row = act ? t >> 1 : 0, half = t & 1;
      const int b = row / NE, p = row % NE;
      const T* gb = Gk + (long)b * NE * NE * 2 + 2 * p;
      T re = 0, im = 0;
      if (act) {
#pragma unroll 4
        for (int q = half; q < NE; q += 2) {
          const T gr = gb[(long)q * NE * 2], gi = gb[(long)q * NE * 2 + 1];
          const T sr = ss[b][q][0], si = ss[b][q][1];
          re = fma(gr, sr, fma(-gi, si, re));
          im = fma(gr, si, fma(gi, sr, im));
        }
      }
      re += __shfl_xor_sync(0xffffffffu, re, 1);
      im += __shfl_xor_sync(0xffffffffu, im, 1);
      if (act && half == 0) {
        sz[b][p][0] = re;
        sz[b][p][1] = im;
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      const int mu = r / NE, p = r % NE;
      T x = 0;
      for (int b = 0; b < nb; ++b) x += (T)vc.tout[b][mu][0] * sz[b][p][0] - (T)vc.tout[b][mu][1] * sz[b][p][1];
      if (sg[r] >= 0) {
        if (dd) dd[sg[r]] += omega * x;
        else ob[sg[r]] = x;
      }
    }
    __syncthreads();
  }
}

// the register kernel when the patch size allows it, else the global-memory one
template <typename T>
cudaError_t invert_patches(T* F, int* piv, int N, long count, int* err, int nsm, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (try_gj_reg<T>(F, piv, N, count, err, nsm, st, e)) return e;
  // larger patches (3D, k >= 2): the global-memory kernel
  const unsigned g = (unsigned)(count < 8L * nsm ? count : 8L * nsm);
  gj_invert_kernel<T><<<g, 256, 0, st>>>(F, piv, N, count, err);
  return cudaGetLastError();
}

// ------------------------------------------------------------ Vanka solve
// The patches of colour-ordered cells li0 .. li0 + nli - 1 in one launch:
// x = A_K^{-1} defect|_K with the explicit inverse (a matrix-vector product
// streamed column by column), stored into the buffer of the cell's colour
// class (cells of one class share no dof; the caller adds omega times the
// class buffers into d), or, with dd set (the cells of one class), added as
// omega x into dd directly.
template <int DIM, typename T>
__global__ void vanka_patch_solve(const T* __restrict__ F, int K1, const T* __restrict__ defect, T* __restrict__ cb,
                                  long cstride, int n0, int n1, int n2, ColourMap cm, long li0, long nli, long Nq2,
                                  long Nq1, long Mv, long Mp, int pdisc, T* __restrict__ dd, T omega) {
  constexpr int NQ = DIM == 3 ? 27 : 9, NC = DIM, NP = DIM == 3 ? 8 : 4, NE = NC * NQ + NP;
  const int N = K1 * NE;
  __shared__ T sx[MAXN];
  __shared__ long sg[MAXN];
  const long g2x = 2L * n0 + 1, g2y = 2L * n1 + 1, g1x = (long)n0 + 1, g1y = (long)n1 + 1;
  for (long li = li0 + blockIdx.x; li < li0 + nli; li += gridDim.x) {
    int col, ex, ey, ez;
    colour_cell(cm, li, col, ex, ey, ez);
    const long cell = ex + (long)n0 * (ey + (long)n1 * ez);
    T* ob = cb + col * cstride;
    const T* A = F + cell * (long)N * N;
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      const int mu = r / NE, loc = r % NE;
      long g;
      if (loc < NC * NQ) {
        const int c = loc / NQ, q = loc % NQ;
        g = (long)mu * Mv + c * Nq2 + (2L * ex + q % 3) + g2x * ((2L * ey + (q / 3) % 3) + g2y * (2L * ez + q / 9));
      } else {
        const int m = loc - NC * NQ;
        if (pdisc) {  // the cell's P1disc coefficients; patch dofs beyond them are unused
          g = m <= DIM ? (long)K1 * Mv + (long)mu * Mp + cell * (DIM + 1) + m : -1;
        } else {
          g = (long)K1 * Mv + (long)mu * Mp + (ex + (m & 1)) + g1x * ((ey + ((m >> 1) & 1)) + g1y * (ez + (m >> 2)));
        }
      }
      sg[r] = g;
      sx[r] = g >= 0 ? defect[g] : (T)0;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      T acc = 0;
#pragma unroll 8
      for (int j = 0; j < N; ++j) acc = fma(A[(long)j * N + r], sx[j], acc);
      if (sg[r] >= 0) {
        if (dd) dd[sg[r]] += omega * acc;
        else ob[sg[r]] = acc;
      }
    }
    __syncthreads();
  }
}

// Vertex-star patch solves of the colour-ordered vertices li0 .. li0 + nli - 1
// (vm: classes of vertex parities over the (n + 1)^d vertex grid), as
// vanka_patch_solve: into the class buffers, or omega x added into dd.
template <int DIM, typename T>
__global__ void vanka_patch_solve_vertex(const T* __restrict__ F, int K1, const T* __restrict__ defect,
                                         T* __restrict__ cb, long cstride, int n0, int n1, int n2, ColourMap vm,
                                         long li0, long nli, long Nq2, long Mv, long Mp, T* __restrict__ dd,
                                         T omega) {
  constexpr int NQ = DIM == 3 ? 27 : 9, NC = DIM, NEV = NC * NQ + 1;
  const int N = K1 * NEV;
  __shared__ T sx[MAXN];
  __shared__ long sg[MAXN];
  const long g2x = 2L * n0 + 1, g2y = 2L * n1 + 1, g1x = (long)n0 + 1, g1y = (long)n1 + 1;
  const int nn[3] = {n0, n1, n2};
  for (long li = li0 + blockIdx.x; li < li0 + nli; li += gridDim.x) {
    int col, vx, vy, vz;
    colour_cell(vm, li, col, vx, vy, vz);
    const long V = vx + g1x * (vy + g1y * (long)vz);
    T* ob = cb + col * cstride;
    const T* A = F + V * (long)N * N;
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      const int mu = r / NEV, loc = r % NEV;
      long g;
      if (loc < NC * NQ) {
        const int c = loc / NQ, q = loc % NQ;
        const int v3[3] = {vx, vy, vz};
        const int j[3] = {q % 3, (q / 3) % 3, q / 9};
        long gi[3] = {0, 0, 0};
        bool in = true;
        for (int d = 0; d < DIM; ++d) {
          gi[d] = 2L * v3[d] - 1 + j[d];
          in = in && gi[d] >= 0 && gi[d] <= 2L * nn[d];
        }
        g = in ? (long)mu * Mv + c * Nq2 + gi[0] + g2x * (gi[1] + g2y * gi[2]) : -1;
      } else {
        g = (long)K1 * Mv + (long)mu * Mp + vx + g1x * (vy + g1y * (long)vz);
      }
      sg[r] = g;
      sx[r] = g >= 0 ? defect[g] : (T)0;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      T acc = 0;
#pragma unroll 8
      for (int j = 0; j < N; ++j) acc = fma(A[(long)j * N + r], sx[j], acc);
      if (sg[r] >= 0) {
        if (dd) dd[sg[r]] += omega * acc;
        else ob[sg[r]] = acc;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------- coarse-level apply
// (A_l x)|_K for all cells in one launch, into the buffer of the cell's
// colour class: per cell and node mu the element matrix E[cell][mu] (spatial
// part, times tau w_mu) and the temporal mass coupling sum_nu K_t[mu][nu]
// M_e x_nu on the velocity; colour_sum forms A_l x.  split = 0: one work item
// per cell; split = 1: one per (cell, mu), each computing that node's rows
// (more parallel work on the small coarse levels).
template <int DIM, typename T>
__global__ void coarse_apply(const T* __restrict__ E, int K1, PatchArgs pa, const T* __restrict__ x, T* __restrict__ cb,
                             long cstride, ColourMap cm, long ncells, long Nq2, long Nq1, long Mv, long Mp,
                             int split) {
  constexpr int NQ = DIM == 3 ? 27 : 9, NC = DIM, NP = DIM == 3 ? 8 : 4, NE = NC * NQ + NP;
  __shared__ T sx[MAXN];
  __shared__ long sg[MAXN];
  __shared__ T smass[NQ * NQ];             // velocity mass of one cell (tensor of the 1D masses)
  __shared__ T skt[MAX_K1][NC * NQ];       // sum_nu K_t[mu][nu] x_nu (velocity part)
  __shared__ T sy[MAX_K1 * NP];            // P1disc: vertex-form pressure rows of the product
  const int N = K1 * NE;
  const int n0 = pa.n[0], n1 = pa.n[1];
  const long g2x = 2L * n0 + 1, g2y = 2L * n1 + 1, g1x = (long)n0 + 1, g1y = (long)n1 + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int t = threadIdx.x; t < NQ * NQ; t += blockDim.x) {
    const int a = t / NQ, b = t % NQ;
    const int ai[3] = {a % 3, (a / 3) % 3, a / 9}, bi[3] = {b % 3, (b / 3) % 3, b / 9};
    double m = 1.0;
    for (int d = 0; d < DIM; ++d) m *= pa.M1h[d][ai[d] * 3 + bi[d]];
    smass[t] = (T)m;
  }
  const int P = split ? K1 : 1;
  for (long it = blockIdx.x; it < ncells * P; it += gridDim.x) {
    const long li = it / P;
    const int mlo = split ? (int)(it % P) : 0, mhi = split ? mlo + 1 : K1;  // nodes whose rows this item computes
    int col, ex, ey, ez;
    colour_cell(cm, li, col, ex, ey, ez);
    const long cell = ex + (long)n0 * (ey + (long)n1 * ez);
    T* ob = cb + col * cstride;
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      const int mu = r / NE, loc = r % NE;
      long g;
      if (loc < NC * NQ) {
        const int c = loc / NQ, q = loc % NQ;
        g = (long)mu * Mv + c * Nq2 + (2L * ex + q % 3) + g2x * ((2L * ey + (q / 3) % 3) + g2y * (2L * ez + q / 9));
      } else {
        const int m = loc - NC * NQ;
        if (pa.pdisc) {
          // vertex value of the cell's affine pressure; the outputs are the coefficients' tests
          const T* pc = x + (long)K1 * Mv + (long)mu * Mp + cell * (DIM + 1);
          T v = pc[0];
          for (int j = 1; j <= DIM; ++j) v += ((m >> (j - 1)) & 1) ? pc[j] : -pc[j];
          sg[r] = -1;
          sx[r] = v;
          continue;
        }
        g = (long)K1 * Mv + (long)mu * Mp + (ex + (m & 1)) + g1x * ((ey + ((m >> 1) & 1)) + g1y * (ez + (m >> 2)));
      }
      sg[r] = g;
      sx[r] = x[g];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < (mhi - mlo) * NC * NQ; t += blockDim.x) {
      const int mu = mlo + t / (NC * NQ), v = t % (NC * NQ);
      T acc = 0;
      for (int nu = 0; nu < K1; ++nu) acc += (T)pa.Kt[mu * K1 + nu] * sx[nu * NE + v];
      skt[mu][v] = acc;
    }
    __syncthreads();
    // one half-warp per row (two rows per warp): coalesced row of E, then the
    // temporal mass coupling; the loop runs over whole warps so that every
    // lane takes part in the half-warp shuffles
    const int hl = lane & 15, half = lane >> 4;
    const int rlo = mlo * NE, rhi = mhi * NE;
    for (int r0 = rlo + 2 * warp; r0 < rhi; r0 += 2 * nwarp) {
      const int r = r0 + half;
      const bool act = r < rhi;
      const int mu = act ? r / NE : 0, i = act ? r % NE : 0;
      const T* Er = E + (cell * K1 + mu) * NE * NE + (long)i * NE;
      T acc = 0;
      if (act) {
#pragma unroll
        for (int j = hl; j < NE; j += 16) acc = fma(Er[j], sx[mu * NE + j], acc);
        if (i < NC * NQ) {
          const int c = i / NQ, a = i % NQ;
          for (int bq = hl; bq < NQ; bq += 16) acc = fma(smass[a * NQ + bq], skt[mu][c * NQ + bq], acc);
        }
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (act && hl == 0) {
        if (sg[r] >= 0) ob[sg[r]] = acc;
        else sy[mu * NP + (i - NC * NQ)] = acc;
      }
    }
    if (pa.pdisc) {
      __syncthreads();
      for (int t = threadIdx.x; t < (mhi - mlo) * (DIM + 1); t += blockDim.x) {
        const int mu = mlo + t / (DIM + 1), j = t % (DIM + 1);
        T v = 0;
        for (int m = 0; m < NP; ++m) v += (T)pdisc_T(m, j) * sy[mu * NP + m];
        ob[(long)K1 * Mv + (long)mu * Mp + cell * (DIM + 1) + j] = v;
      }
    }
    __syncthreads();
  }
}

template <typename A, typename B>
__global__ void axpy_conv(const A* __restrict__ x, B* __restrict__ y, size_t n, double a, double b) {
  // y = a * x + b * y  (b == 0: y = a * x)
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = b == 0.0 ? (B)(a * (double)x[i]) : (B)(a * (double)x[i] + b * (double)y[i]);
}

template <typename T>
__global__ void sub_kernel(const T* __restrict__ r, const T* __restrict__ Ad, T* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = r[i] - Ad[i];
}

// U_rep: every node's velocity replaced by sum_mu lrep_mu V_mu; pressure copied
__global__ void rep_state_kernel(const double* __restrict__ U, double* __restrict__ Ur, int K1, long Mv, long Np,
                                 double l0, double l1, double l2, double l3) {
  const double l[4] = {l0, l1, l2, l3};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < Mv + Np; i += (long)gridDim.x * blockDim.x) {
    if (i < Mv) {
      double v = 0.0;
      for (int mu = 0; mu < K1; ++mu) v += l[mu] * U[(long)mu * Mv + i];
      for (int mu = 0; mu < K1; ++mu) Ur[(long)mu * Mv + i] = v;
    } else {
      const long j = i - Mv;
      Ur[(long)K1 * Mv + j] = U[(long)K1 * Mv + j];
    }
  }
}

std::string shape_label(const LaunchShape& c, int nsm) {
  return std::to_string(c.threads) + " threads x " + std::to_string(c.grid / (nsm > 0 ? nsm : 1)) + "/SM";
}

unsigned gridn(size_t n, int nsm) {
  size_t g = (n + 255) / 256;
  const size_t cap = 16 * (size_t)nsm;
  if (g > cap) g = cap;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

// ------------------------------------------------------------------ state
struct MgLevelData {
  void* E = nullptr;    // [ncells][K1][NE][NE]
  void* LU = nullptr;   // [ncells][N][N]
  int* piv = nullptr;   // [ncells][N]
  void* r = nullptr;    // level vectors (precision of the hierarchy)
  void* d = nullptr;
  void* t = nullptr;
  void* t2 = nullptr;
  void* t3 = nullptr;
  void* cbuf = nullptr;  // 2^d colour-private level vectors (zero outside each class's dofs)
  void* vbuf = nullptr;  // the same for the vertex-star patches' classes (patch_type = 1)
};

struct MgState {
  int prec = -1;
  bool allocated = false;
  std::vector<MgLevelData> L;
  void* Erep = nullptr;          // finest surrogate matrices [ncells][NE][NE]
  double* Urep = nullptr;        // representative state (slab vector)
  double* cache_rep64 = nullptr;
  double* fcache_rep64 = nullptr;
  float* cache_rep32 = nullptr;
  float* fcache_rep32 = nullptr;
  int* bcells = nullptr;         // boundary cells (linear) of the finest level
  int nbc = 0;
  double* d_tab = nullptr;       // 1D transfer tables on the device (P2, P1)
  // the V-cycle as a CUDA graph, for the (r, d, precision, tangent) it was captured with
  cudaGraphExec_t gexec = nullptr;
  const void* g_r = nullptr;
  void* g_d = nullptr;
  int g_prec = -1, g_tangent = -1;
  bool g_seen = false;           // the key was run once eagerly (all lazy initialisation done)
  bool g_failed = false;         // capture failed for this key: eager
  bool c13 = false;              // finest surrogate patches diagonalised in time (TimeEig)
  TimeEig te;
  CoarseDirect cd;               // direct solve of the coarsest level (coarse_solve = 1)
};

namespace {

size_t esz(int prec) { return prec == ST_FP64 ? sizeof(double) : sizeof(float); }

void drop_graph(MgState* m) {
  if (m->gexec) cudaGraphExecDestroy(m->gexec);
  m->gexec = nullptr;
  m->g_seen = false;
  m->g_failed = false;
  m->g_r = nullptr;
  m->g_d = nullptr;
}

void free_mg(MgState* m) {
  drop_graph(m);
  for (auto& l : m->L) {
    cudaFree(l.E);
    cudaFree(l.LU);
    cudaFree(l.piv);
    cudaFree(l.r);
    cudaFree(l.d);
    cudaFree(l.t);
    cudaFree(l.t2);
    cudaFree(l.t3);
    cudaFree(l.cbuf);
    cudaFree(l.vbuf);
  }
  m->L.clear();
  cudaFree(m->Erep);
  cudaFree(m->Urep);
  cudaFree(m->cache_rep64);
  cudaFree(m->fcache_rep64);
  cudaFree(m->cache_rep32);
  cudaFree(m->fcache_rep32);
  cudaFree(m->bcells);
  cudaFree(m->d_tab);
  coarse_direct_free(m->cd);
  m->Erep = nullptr;
  m->Urep = nullptr;
  m->cache_rep64 = m->fcache_rep64 = nullptr;
  m->cache_rep32 = m->fcache_rep32 = nullptr;
  m->bcells = nullptr;
  m->d_tab = nullptr;
  m->allocated = false;
}

cudaError_t alloc_mg(st_problem* h, MgState* m, int prec) {
  m->c13 = h->P.finest_patches == 0 && make_time_eig(h->T, m->te) && m->te.nb <= MAX_K1;
  const int nl = (int)h->lev.size();
  const int NE = ne_of(h->dim), K1 = h->K1, N = K1 * NE;
  const size_t es = esz(prec);
  m->L.resize(nl);
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < nl && e == cudaSuccess; ++l) {
    const Level& Lv = h->lev[l];
    MgLevelData& d = m->L[l];
    e = cudaMalloc(&d.E, (size_t)Lv.ncells * K1 * NE * NE * es);
    // finest level with the time-diagonalised surrogate: nb complex NE x NE inverses per patch
    const bool c13 = (l == nl - 1) && m->c13;
    const size_t nlu = c13 ? (size_t)m->te.nb * NE * NE * 2 : (size_t)N * N;
    // vertex-star patches: one K1 * nev_of(dim) patch per vertex
    const bool vtx = h->P.patch_type == 1;
    const size_t Nv = (size_t)K1 * nev_of(h->dim);
    const size_t npat = vtx ? (size_t)n_vertices(h, Lv) : (size_t)Lv.ncells;
    if (e == cudaSuccess) e = cudaMalloc(&d.LU, npat * (vtx ? Nv * Nv : nlu) * es);
    if (e == cudaSuccess) e = cudaMalloc(&d.piv, npat * (vtx ? Nv : (size_t)N) * sizeof(int));
    if (e == cudaSuccess && vtx) e = cudaMalloc(&d.vbuf, (size_t)(1 << h->dim) * Lv.Nst * es);
    if (e == cudaSuccess && vtx) e = cudaMemset(d.vbuf, 0, (size_t)(1 << h->dim) * Lv.Nst * es);
    if (e == cudaSuccess) e = cudaMalloc(&d.r, (size_t)Lv.Nst * es);
    if (e == cudaSuccess) e = cudaMalloc(&d.d, (size_t)Lv.Nst * es);
    if (e == cudaSuccess) e = cudaMalloc(&d.t, (size_t)Lv.Nst * es);
    if (e == cudaSuccess) e = cudaMalloc(&d.t2, (size_t)Lv.Nst * es);
    if (e == cudaSuccess) e = cudaMalloc(&d.t3, (size_t)Lv.Nst * es);
    if (e == cudaSuccess) e = cudaMalloc(&d.cbuf, (size_t)(1 << h->dim) * Lv.Nst * es);
    if (e == cudaSuccess) e = cudaMemset(d.cbuf, 0, (size_t)(1 << h->dim) * Lv.Nst * es);
  }
  const Level& F = h->lev.back();
  if (e == cudaSuccess) e = cudaMalloc(&m->Erep, (size_t)F.ncells * NE * NE * es);
  if (e == cudaSuccess) e = cudaMalloc(&m->Urep, (size_t)F.Nst * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&m->cache_rep64, h->cache_len * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&m->fcache_rep64, h->fcache_len * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&m->cache_rep32, h->cache_len * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->fcache_rep32, h->fcache_len * sizeof(float));
  if (e == cudaSuccess) {
    std::vector<int> bc;
    for (long c = 0; c < F.ncells; ++c) {
      const int e3[3] = {(int)(c % F.n[0]), (int)((c / F.n[0]) % F.n[1]), (int)(c / ((long)F.n[0] * F.n[1]))};
      bool on = false;
      for (int ax = 0; ax < h->dim; ++ax) on = on || e3[ax] == 0 || e3[ax] == F.n[ax] - 1;
      if (on) bc.push_back((int)c);
    }
    m->nbc = (int)bc.size();
    if (bc.empty()) bc.push_back(0);
    e = cudaMalloc(&m->bcells, bc.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(m->bcells, bc.data(), bc.size() * sizeof(int), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    double tab[21];
    memcpy(tab, h->R.P2, sizeof(h->R.P2));
    memcpy(tab + 15, h->R.P1, sizeof(h->R.P1));
    e = cudaMalloc(&m->d_tab, sizeof(tab));
    if (e == cudaSuccess) e = cudaMemcpy(m->d_tab, tab, sizeof(tab), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && h->P.coarse_solve == 1) e = coarse_direct_alloc(m->cd, h->lev[0].Nst);
  m->prec = prec;
  m->allocated = e == cudaSuccess;
  return e;
}

CoarseGeom coarse_geom(const st_problem* h) {
  CoarseGeom g;
  memset(&g, 0, sizeof(g));
  const Level& L = h->lev[0];
  g.dim = h->dim;
  g.K1 = h->K1;
  g.pdisc = h->P.pressure_space == 1 ? 1 : 0;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = L.n[d];
    g.g2[d] = L.g2[d];
    g.g1[d] = L.g1[d];
    for (int i = 0; i < 9; ++i) g.M1h[d][i] = h->R.M1[i] * (d < h->dim ? L.h[d] : 1.0);
  }
  g.Nq2 = L.Nq2;
  g.Mv = L.Mv;
  g.Mp = L.Mp;
  for (int i = 0; i < h->K1 * h->K1; ++i) g.Kt[i] = h->T.Kt[i];
  return g;
}

// refinement steps and relative tolerance of the coarsest-level direct solve
constexpr int COARSE_REFINE_STEPS = 10;
constexpr double COARSE_RTOL = 1e-12;

PatchArgs patch_args(const st_problem* h, int level, bool surrogate) {
  PatchArgs pa;
  memset(&pa, 0, sizeof(pa));
  const Level& L = h->lev[level];
  for (int d = 0; d < 3; ++d) pa.n[d] = L.n[d];
  pa.K1 = h->K1;
  for (int i = 0; i < h->K1 * h->K1; ++i) pa.Kt[i] = h->T.Kt[i];
  for (int mu = 0; mu < h->K1; ++mu) pa.wr[mu] = surrogate ? h->T.w[mu] / h->T.w[0] : 1.0;
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < 9; ++i) pa.M1h[d][i] = h->R.M1[i] * (d < h->dim ? L.h[d] : 1.0);
  pa.surrogate = surrogate ? 1 : 0;
  pa.pdisc = h->P.pressure_space == 1 ? 1 : 0;
  return pa;
}

template <typename T>
cudaError_t elm_dispatch(st_problem* h, int level, int prec, int tangent, const void* cache, const void* fcache, int mu,
                         int stride, int slot, void* E, const int* bcells, int nbc) {
  OpArgs a;
  fill_op_args(h, level, a);
  a.tangent = tangent;
  a.cache = cache;
  a.fcache = fcache;
  a.elm_mu = mu;
  a.elm_stride = stride;
  a.elm_slot = slot;
  const Level& L = h->lev[level];
  return h->dim == 2 ? dispatch_elm_2d(h, L, a, prec, tangent, E, bcells, nbc)
                     : dispatch_elm_3d(h, L, a, prec, tangent, E, bcells, nbc);
}

ColourMap colour_map(const st_problem* h, const Level& L) {
  ColourMap cm;
  cm.nclass = 1 << h->dim;
  for (int c = 0; c < 9; ++c) cm.start[c] = L.col_start[c];
  for (int c = 0; c < 8; ++c)
    for (int d = 0; d < 3; ++d) cm.cn[c][d] = L.cn[c][d];
  return cm;
}

long n_vertices(const st_problem* h, const Level& L) {
  return (long)(L.n[0] + 1) * (L.n[1] + 1) * (h->dim == 3 ? L.n[2] + 1 : 1);
}

// classes of the vertex grid by vertex-coordinate parity (px + 2 py + 4 pz),
// in the ColourMap form the patch kernels read
ColourMap vertex_map(const st_problem* h, const Level& L) {
  ColourMap cm;
  cm.nclass = 1 << h->dim;
  long start = 0;
  for (int c = 0; c < 8; ++c) {
    cm.start[c] = start;
    for (int a = 0; a < 3; ++a) {
      const int nv = a < h->dim ? L.n[a] + 1 : 1, bit = a < h->dim ? (c >> a) & 1 : 0;
      cm.cn[c][a] = (nv + 1 - bit) / 2;
    }
    if (c < cm.nclass) start += (long)cm.cn[c][0] * cm.cn[c][1] * cm.cn[c][2];
  }
  cm.start[8] = start;
  for (int c = cm.nclass; c < 8; ++c) cm.start[c] = start;
  return cm;
}

template <typename T>
cudaError_t level_apply(st_problem* h, MgState* m, int l, const T* x, T* y) {
  // y = A_l x
  const Level& L = h->lev[l];
  const int prec = sizeof(T) == 8 ? ST_FP64 : ST_FP32;
  if (l == (int)h->lev.size() - 1) return launch_op(h, l, OP_JAC, prec, h->lin_tangent, x, y, nullptr, nullptr);
  PatchArgs pa = patch_args(h, l, false);
  const ColourMap cm = colour_map(h, L);
  T* cb = (T*)m->L[l].cbuf;
  // autotuned launch shape (threads per CTA, CTAs per SM, one work item per
  // cell or per (cell, node))
  const LaunchShape cand[7] = {{128, 8L * h->nsm},  {256, 8L * h->nsm},  {128, 16L * h->nsm}, {256, 4L * h->nsm},
                               {128, 16L * h->nsm}, {256, 8L * h->nsm},  {512, 4L * h->nsm}};
  const int csplit[7] = {0, 0, 0, 0, 1, 1, 1};
  auto run = [&](int i) {
    const long items = L.ncells * (csplit[i] ? h->K1 : 1);
    const unsigned g = (unsigned)(items < cand[i].grid ? items : cand[i].grid);
    if (h->dim == 2)
      coarse_apply<2, T><<<g, cand[i].threads, 0, h->stream>>>((const T*)m->L[l].E, h->K1, pa, x, cb, L.Nst, cm,
                                                               L.ncells, L.Nq2, L.Nq1, L.Mv, L.Mp, csplit[i]);
    else
      coarse_apply<3, T><<<g, cand[i].threads, 0, h->stream>>>((const T*)m->L[l].E, h->K1, pa, x, cb, L.Nst, cm,
                                                               L.ncells, L.Nq2, L.Nq1, L.Mv, L.Mp, csplit[i]);
    return cudaGetLastError();
  };
  const int pick = tune_pick(
      "coarse_apply<" + std::to_string(h->dim) + "," + (sizeof(T) == 8 ? "double" : "float") + "> K1=" +
          std::to_string(h->K1) + " cells=" + std::to_string(L.ncells),
      h->K1 > 1 ? 7 : 4, run,
      [&](int i) { return shape_label(cand[i], h->nsm) + (csplit[i] ? " per (cell, node)" : " per cell"); },
      h->stream);
  cudaError_t e = run(pick);
  if (e != cudaSuccess) return e;
  colour_sum<T><<<gridn(L.Nst, h->nsm), 256, 0, h->stream>>>(cb, L.Nst, cm.nclass, y, L.Nst, (T)1, 0);
  return cudaGetLastError();
}

// d_zero: d is zero on entry (the V-cycle's pre-smoothing and coarse sweeps),
// so the first defect is r itself and its apply is skipped
template <typename T>
cudaError_t vanka_steps(st_problem* h, MgState* m, int l, int sweeps, const T* r, T* d, bool d_zero = false) {
  const Level& L = h->lev[l];
  MgLevelData& D = m->L[l];
  const int N = h->K1 * ne_of(h->dim);
  const ColourMap cm = colour_map(h, L);
  T* cb = (T*)D.cbuf;
  const bool c13 = m->c13 && l == (int)h->lev.size() - 1;
  const int pdisc = h->P.pressure_space == 1 ? 1 : 0;
  VankaC13 vc;
  memset(&vc, 0, sizeof(vc));
  if (c13) {
    vc.nb = m->te.nb;
    memcpy(vc.tin, m->te.tin, sizeof(vc.tin));
    memcpy(vc.tout, m->te.tout, sizeof(vc.tout));
  }
  // smoother 0: one pass over all cells into the class buffers, then
  // d += omega sum of the buffers; smoother 1: one pass per colour class,
  // each after a fresh defect, adding omega x into d directly
  const bool finest = l == (int)h->lev.size() - 1;
  const bool mult = h->P.smoother == 1 || (h->P.smoother == 2 && finest);
  const int npass = mult ? cm.nclass : 1;
  // vertex-star patches (patch_type = 1): their own classes and buffers
  const bool vtx = h->P.patch_type == 1;
  const ColourMap pm = vtx ? vertex_map(h, L) : cm;
  const long npatch = vtx ? n_vertices(h, L) : L.ncells;
  T* pbuf = vtx ? (T*)D.vbuf : cb;
  const int Np = vtx ? h->K1 * nev_of(h->dim) : N;
  const int nt0 = Np <= 128 ? 128 : 256;
  const LaunchShape cand[5] = {{nt0, 16L * h->nsm}, {128, 16L * h->nsm}, {256, 8L * h->nsm}, {512, 4L * h->nsm},
                               {128, 32L * h->nsm}};
  const T om = (T)(h->P.smoother == 2 && !finest && h->P.omega_coarse > 0 ? h->P.omega_coarse : h->P.omega);
  for (int s = 0; s < sweeps; ++s) {
    for (int c = 0; c < npass; ++c) {
      const long li0 = mult ? pm.start[c] : 0, nli = mult ? pm.start[c + 1] - pm.start[c] : npatch;
      if (nli == 0) continue;
      cudaError_t e = cudaSuccess;
      const T* defect = (const T*)D.t;
      if (d_zero) {
        defect = r;  // r - A 0
        d_zero = false;
      } else {
        e = level_apply<T>(h, m, l, d, (T*)D.t2);
        if (e != cudaSuccess) return e;
        sub_kernel<T><<<gridn(L.Nst, h->nsm), 256, 0, h->stream>>>(r, (const T*)D.t2, (T*)D.t, L.Nst);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
      }
      // the launch shape (threads per patch CTA, CTAs per SM) is autotuned;
      // trial launches store into the class buffers (dd = nullptr), so they
      // leave d alone
      auto run = [&](int i, T* dd) {
        const unsigned g = (unsigned)(nli < cand[i].grid ? nli : cand[i].grid);
        const int nt = cand[i].threads;
        if (vtx) {
          if (h->dim == 2)
            vanka_patch_solve_vertex<2, T><<<g, nt, 0, h->stream>>>((const T*)D.LU, h->K1, defect, pbuf, L.Nst,
                                                                    L.n[0], L.n[1], L.n[2], pm, li0, nli, L.Nq2,
                                                                    L.Mv, L.Mp, dd, om);
          else
            vanka_patch_solve_vertex<3, T><<<g, nt, 0, h->stream>>>((const T*)D.LU, h->K1, defect, pbuf, L.Nst,
                                                                    L.n[0], L.n[1], L.n[2], pm, li0, nli, L.Nq2,
                                                                    L.Mv, L.Mp, dd, om);
        } else if (c13) {
          if (h->dim == 2)
            vanka_patch_solve_c13<2, T><<<g, nt, 0, h->stream>>>((const T*)D.LU, vc, h->K1, defect, cb, L.Nst,
                                                                 L.n[0], L.n[1], L.n[2], cm, li0, nli, L.Nq2, L.Nq1,
                                                                 L.Mv, L.Mp, pdisc, dd, om);
          else
            vanka_patch_solve_c13<3, T><<<g, nt, 0, h->stream>>>((const T*)D.LU, vc, h->K1, defect, cb, L.Nst,
                                                                 L.n[0], L.n[1], L.n[2], cm, li0, nli, L.Nq2, L.Nq1,
                                                                 L.Mv, L.Mp, pdisc, dd, om);
        } else if (h->dim == 2) {
          vanka_patch_solve<2, T><<<g, nt, 0, h->stream>>>((const T*)D.LU, h->K1, defect, cb, L.Nst, L.n[0],
                                                           L.n[1], L.n[2], cm, li0, nli, L.Nq2, L.Nq1, L.Mv, L.Mp,
                                                           pdisc, dd, om);
        } else {
          vanka_patch_solve<3, T><<<g, nt, 0, h->stream>>>((const T*)D.LU, h->K1, defect, cb, L.Nst, L.n[0],
                                                           L.n[1], L.n[2], cm, li0, nli, L.Nq2, L.Nq1, L.Mv, L.Mp,
                                                           pdisc, dd, om);
        }
        return cudaGetLastError();
      };
      const int pick = tune_pick(std::string(vtx ? "vanka_patch_solve_vertex<"
                                                 : c13 ? "vanka_patch_solve_c13<" : "vanka_patch_solve<") +
                                     std::to_string(h->dim) + "," + (sizeof(T) == 8 ? "double" : "float") +
                                     "> N=" + std::to_string(Np) + (vtx ? " vertices=" : " cells=") +
                                     std::to_string(nli),
                                 5, [&](int i) { return run(i, nullptr); },
                                 [&](int i) { return shape_label(cand[i], h->nsm); }, h->stream);
      e = run(pick, mult ? d : nullptr);
      if (e != cudaSuccess) return e;
      if (!mult) {
        colour_sum<T><<<gridn(L.Nst, h->nsm), 256, 0, h->stream>>>(pbuf, L.Nst, cm.nclass, d, L.Nst, om, 1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
      }
    }
  }
  return cudaSuccess;
}

// slab restriction y = P^T x (fine level l -> l-1) or prolongation-add
// y += P x (l-1 -> l), one 1D pass per direction; w1, w2: fine-size work
template <typename T>
cudaError_t transfer(st_problem* h, MgState* m, int l, bool restrict_, const T* x, T* y, T* w1, T* w2) {
  const Level& F = h->lev[l];
  const Level& C = h->lev[l - 1];
  const int d = h->dim, K1 = h->K1;
  const double* P2 = m->d_tab;
  const double* P1 = m->d_tab + 15;
  T* last = nullptr;
  for (int part = 0; part < 2; ++part) {
    const int nblk = part == 0 ? K1 * d : K1;
    const size_t offF = part == 0 ? 0 : (size_t)K1 * F.Mv, offC = part == 0 ? 0 : (size_t)K1 * C.Mv;
    if (part == 1 && h->P.pressure_space == 1) {
      // P1disc pressure: cell-wise transfer (into y, or beside the velocity in the last work buffer)
      cudaError_t e = cudaSuccess;
      if (restrict_) {
        const unsigned gr = gridn((size_t)C.ncells * K1, h->nsm);
        if (d == 2) pdisc_restrict<T, 2><<<gr, 256, 0, h->stream>>>(x + offF, y + offC, C.n[0], C.n[1], 1, K1);
        else pdisc_restrict<T, 3><<<gr, 256, 0, h->stream>>>(x + offF, y + offC, C.n[0], C.n[1], C.n[2], K1);
      } else {
        T* work = ((d - 1) & 1) ? w2 : w1;
        const unsigned gr = gridn((size_t)F.ncells * K1, h->nsm);
        if (d == 2) pdisc_prolong<T, 2><<<gr, 256, 0, h->stream>>>(x + offC, work + offF, F.n[0], F.n[1], 1, K1);
        else pdisc_prolong<T, 3><<<gr, 256, 0, h->stream>>>(x + offC, work + offF, F.n[0], F.n[1], F.n[2], K1);
      }
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      continue;
    }
    int g[3];
    for (int a = 0; a < 3; ++a) g[a] = (int)(restrict_ ? (part == 0 ? F.g2[a] : F.g1[a]) : (part == 0 ? C.g2[a] : C.g1[a]));
    const T* src = x + (restrict_ ? offF : offC);
    for (int dir = 0; dir < d; ++dir) {
      T* work = (dir & 1) ? w2 : w1;
      T* dst = (restrict_ && dir == d - 1) ? y + offC : work + offF;
      const int nc = C.n[dir];
      int go[3] = {g[0], g[1], g[2]};
      go[dir] = restrict_ ? (part == 0 ? 2 * nc + 1 : nc + 1) : (part == 0 ? 4 * nc + 1 : 2 * nc + 1);
      const size_t nout = (size_t)go[0] * go[1] * go[2] * nblk;
      const unsigned gr = gridn(nout, h->nsm);
      if (restrict_) {
        if (part == 0) restrict_pass<T, 2><<<gr, 256, 0, h->stream>>>(src, dst, g[0], g[1], g[2], dir, nc, nblk, P2);
        else restrict_pass<T, 1><<<gr, 256, 0, h->stream>>>(src, dst, g[0], g[1], g[2], dir, nc, nblk, P1);
      } else {
        if (part == 0) prolong_pass<T, 2><<<gr, 256, 0, h->stream>>>(src, dst, g[0], g[1], g[2], dir, nc, nblk, P2);
        else prolong_pass<T, 1><<<gr, 256, 0, h->stream>>>(src, dst, g[0], g[1], g[2], dir, nc, nblk, P1);
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      g[dir] = go[dir];
      src = dst;
      if (dir == d - 1) last = work;
    }
  }
  if (!restrict_) {  // y += P x  (the prolongation sits in `last`)
    axpy_conv<T, T><<<gridn(F.Nst, h->nsm), 256, 0, h->stream>>>(last, y, F.Nst, 1.0, 1.0);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t vcycle_rec(st_problem* h, MgState* m, int l, const T* r, T* d) {
  const Level& L = h->lev[l];
  cudaError_t e = cudaMemsetAsync(d, 0, L.Nst * sizeof(T), h->stream);
  if (e != cudaSuccess) return e;
  if (l == 0)
    return h->P.coarse_solve == 1
               ? coarse_direct_solve<T>(m->cd, r, d, COARSE_REFINE_STEPS, COARSE_RTOL, h->nsm, h->stream)
               : vanka_steps<T>(h, m, 0, h->P.coarse_sweeps, r, d, true);
  e = vanka_steps<T>(h, m, l, h->P.pre_smooth, r, d, true);
  if (e != cudaSuccess) return e;
  MgLevelData& D = m->L[l];
  MgLevelData& Cd = m->L[l - 1];
  // defect and restriction: r_c = P^T (r - A d)
  e = level_apply<T>(h, m, l, d, (T*)D.t2);
  if (e != cudaSuccess) return e;
  sub_kernel<T><<<gridn(L.Nst, h->nsm), 256, 0, h->stream>>>(r, (const T*)D.t2, (T*)D.t, L.Nst);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = transfer<T>(h, m, l, true, (const T*)D.t, (T*)Cd.r, (T*)D.t2, (T*)D.t3);
  if (e != cudaSuccess) return e;
  e = vcycle_rec<T>(h, m, l - 1, (const T*)Cd.r, (T*)Cd.d);
  if (e != cudaSuccess) return e;
  e = transfer<T>(h, m, l, false, (const T*)Cd.d, d, (T*)D.t, (T*)D.t2);
  if (e != cudaSuccess) return e;
  return vanka_steps<T>(h, m, l, h->P.post_smooth, r, d);
}

}  // namespace

st_status mg_destroy(st_problem* h) {
  if (h && h->mg) {
    MgState* m = (MgState*)h->mg;
    free_mg(m);
    delete m;
    h->mg = nullptr;
  }
  return ST_OK;
}

st_status mg_setup(st_problem* h, st_prec prec, bool rebuild_finest) {
  if (!h->lin_valid) return set_error(h, ST_EINVAL, "st_precond_setup: no linearisation (call st_linearize)");
  if (h->d_Ulin == nullptr) return set_error(h, ST_EINVAL, "st_precond_setup: no linearisation state");
  MgState* m = (MgState*)h->mg;
  if (!m) {
    m = new MgState();
    h->mg = m;
  }
  cudaError_t e = cudaSuccess;
  if (!m->allocated || m->prec != prec) {
    free_mg(m);
    e = alloc_mg(h, m, prec);
    if (e != cudaSuccess) return cuda_check(h, e, "st_precond_setup alloc");
    rebuild_finest = true;
  }
  if (!h->precond_valid) rebuild_finest = true;
  const int nl = (int)h->lev.size(), L = nl - 1;
  const Level& F = h->lev[L];
  const int NE = ne_of(h->dim), K1 = h->K1, N = K1 * NE;
  const size_t es = esz(prec);
  const int tangent = h->lin_tangent;
  const void* cache = prec == ST_FP64 ? (const void*)h->d_cache64 : (const void*)h->d_cache32;
  const void* fcache = prec == ST_FP64 ? (const void*)h->d_fcache64 : (const void*)h->d_fcache32;
  // finest level: exact element matrices per node (for the Galerkin operators
  // and the exact finest patches)
  const bool exact_finest = h->P.finest_patches == 1;
  const bool direct = h->P.coarse_solve == 1;
  if (nl > 1 || exact_finest || direct)
    for (int mu = 0; mu < K1 && e == cudaSuccess; ++mu)
      e = prec == ST_FP64 ? elm_dispatch<double>(h, L, prec, tangent, cache, fcache, mu, K1, mu, m->L[L].E, m->bcells, m->nbc)
                          : elm_dispatch<float>(h, L, prec, tangent, cache, fcache, mu, K1, mu, m->L[L].E, m->bcells, m->nbc);
  if (e != cudaSuccess) return cuda_check(h, e, "st_precond_setup element matrices");
  // representative state and its coefficients -> surrogate matrices
  if (rebuild_finest && !exact_finest) {
    const double* lr = h->T.lrep;
    rep_state_kernel<<<gridn(F.Mv + F.Mp, h->nsm), 256, 0, h->stream>>>(
        h->d_Ulin, m->Urep, K1, F.Mv, (long)K1 * F.Mp, lr[0], K1 > 1 ? lr[1] : 0.0, K1 > 2 ? lr[2] : 0.0,
        K1 > 3 ? lr[3] : 0.0);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
      // linearise at U_rep into the representative caches
      double* c64 = h->d_cache64;
      double* f64 = h->d_fcache64;
      h->d_cache64 = m->cache_rep64;
      h->d_fcache64 = m->fcache_rep64;
      e = launch_op(h, L, OP_LIN, ST_FP64, tangent, m->Urep, nullptr, nullptr, nullptr);
      h->d_cache64 = c64;
      h->d_fcache64 = f64;
    }
    if (e == cudaSuccess && prec == ST_FP32) {
      e = cast_f64_f32(m->cache_rep64, m->cache_rep32, h->cache_len, h->stream);
      if (e == cudaSuccess) e = cast_f64_f32(m->fcache_rep64, m->fcache_rep32, h->fcache_len, h->stream);
    }
    const void* rc = prec == ST_FP64 ? (const void*)m->cache_rep64 : (const void*)m->cache_rep32;
    const void* rf = prec == ST_FP64 ? (const void*)m->fcache_rep64 : (const void*)m->fcache_rep32;
    if (e == cudaSuccess) {
      e = cudaMemsetAsync(m->Erep, 0, (size_t)F.ncells * NE * NE * es, h->stream);
    }
    if (e == cudaSuccess)
      e = prec == ST_FP64 ? elm_dispatch<double>(h, L, prec, tangent, rc, rf, 0, 1, 0, m->Erep, m->bcells, m->nbc)
                          : elm_dispatch<float>(h, L, prec, tangent, rc, rf, 0, 1, 0, m->Erep, m->bcells, m->nbc);
  }
  if (e != cudaSuccess) return cuda_check(h, e, "st_precond_setup surrogate matrices");
  // Galerkin coarse operators
  for (int l = L - 1; l >= 0 && e == cudaSuccess; --l) {
    const Level& C = h->lev[l];
    const size_t sm = 3 * (size_t)NE * NE * es;
    const long items = C.ncells * K1;
    const unsigned g = (unsigned)(items < 4L * h->nsm ? items : 4L * h->nsm);
    if (prec == ST_FP64) {
      if (h->dim == 2) {
        cudaFuncSetAttribute(galerkin_sf_kernel<2, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        galerkin_sf_kernel<2, double><<<g, 256, sm, h->stream>>>((const double*)m->L[l + 1].E, (double*)m->L[l].E,
                                                                 C.n[0], C.n[1], 1, K1, m->d_tab);
      } else {
        cudaFuncSetAttribute(galerkin_sf_kernel<3, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        galerkin_sf_kernel<3, double><<<g, 256, sm, h->stream>>>((const double*)m->L[l + 1].E, (double*)m->L[l].E,
                                                                 C.n[0], C.n[1], C.n[2], K1, m->d_tab);
      }
    } else {
      if (h->dim == 2) {
        cudaFuncSetAttribute(galerkin_sf_kernel<2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        galerkin_sf_kernel<2, float><<<g, 256, sm, h->stream>>>((const float*)m->L[l + 1].E, (float*)m->L[l].E,
                                                                C.n[0], C.n[1], 1, K1, m->d_tab);
      } else {
        cudaFuncSetAttribute(galerkin_sf_kernel<3, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        galerkin_sf_kernel<3, float><<<g, 256, sm, h->stream>>>((const float*)m->L[l + 1].E, (float*)m->L[l].E,
                                                                C.n[0], C.n[1], C.n[2], K1, m->d_tab);
      }
    }
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_check(h, e, "st_precond_setup Galerkin");
  // the coarsest level's direct solve: dense A_0 and its inverse
  e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
  if (e == cudaSuccess && direct) {
    const CoarseGeom cg = coarse_geom(h);
    e = prec == ST_FP64 ? coarse_direct_setup<double>(cg, (const double*)m->L[0].E, m->cd, h->d_err, h->nsm, h->stream)
                        : coarse_direct_setup<float>(cg, (const float*)m->L[0].E, m->cd, h->d_err, h->nsm, h->stream);
  }
  if (e != cudaSuccess) return cuda_check(h, e, "st_precond_setup coarse direct solve");
  // patches: assemble + factorise (the error flag also carries the coarse inversion's zero pivots)
  for (int l = 0; l < nl && e == cudaSuccess; ++l) {
    const Level& Lv = h->lev[l];
    const bool sur = (l == L) && !exact_finest;
    if (l == L && !rebuild_finest) continue;  // refresh rule: keep the finest factorisations
    if (h->P.patch_type == 1) {
      // vertex-star patches from the level's exact element matrices
      const long nvx = n_vertices(h, Lv);
      const int Nv = K1 * nev_of(h->dim);
      const unsigned gv = (unsigned)(nvx < 8L * h->nsm ? nvx : 8L * h->nsm);
      const PatchArgs pv = patch_args(h, l, false);
      if (prec == ST_FP64) {
        if (h->dim == 2)
          patch_assemble_vertex<2, double><<<gv, 256, 0, h->stream>>>((const double*)m->L[l].E, K1, pv,
                                                                      (double*)m->L[l].LU);
        else
          patch_assemble_vertex<3, double><<<gv, 256, 0, h->stream>>>((const double*)m->L[l].E, K1, pv,
                                                                      (double*)m->L[l].LU);
        e = cudaGetLastError();
        if (e == cudaSuccess)
          e = invert_patches<double>((double*)m->L[l].LU, m->L[l].piv, Nv, nvx, h->d_err, h->nsm, h->stream);
      } else {
        if (h->dim == 2)
          patch_assemble_vertex<2, float><<<gv, 256, 0, h->stream>>>((const float*)m->L[l].E, K1, pv,
                                                                     (float*)m->L[l].LU);
        else
          patch_assemble_vertex<3, float><<<gv, 256, 0, h->stream>>>((const float*)m->L[l].E, K1, pv,
                                                                     (float*)m->L[l].LU);
        e = cudaGetLastError();
        if (e == cudaSuccess)
          e = invert_patches<float>((float*)m->L[l].LU, m->L[l].piv, Nv, nvx, h->d_err, h->nsm, h->stream);
      }
      continue;
    }
    PatchArgs pa = patch_args(h, l, sur);
    const bool c13 = sur && m->c13;
    if (c13) {
      pa.c13 = 1;
      pa.nb = m->te.nb;
      for (int b = 0; b < m->te.nb; ++b) {
        pa.lam[b][0] = m->te.lam[b][0];
        pa.lam[b][1] = m->te.lam[b][1];
      }
    }
    const void* Esrc = sur ? m->Erep : m->L[l].E;
    const int estride = sur ? 1 : K1;
    const unsigned g = (unsigned)(Lv.ncells < 8L * h->nsm ? Lv.ncells : 8L * h->nsm);
    const long nblk = Lv.ncells * (long)m->te.nb;
    // CIP in the surrogate patches: face weights at the representative state
    const bool cip = sur && h->P.gamma_cip > 0 && h->d_cipw_res;
    CipPatchArgs ca;
    memset(&ca, 0, sizeof(ca));
    if (cip) {
      for (int d = 0; d < 3; ++d) {
        ca.n[d] = Lv.n[d];
        ca.ih[d] = 1.0 / Lv.h[d];
      }
      ca.K1 = K1;
      ca.nb = pa.nb;
      ca.c13 = pa.c13;
      for (int i = 0; i < 6; ++i) ca.ED[i] = h->R.ED[i];
      for (int i = 0; i < 9; ++i) ca.B[i] = h->R.B[i];
      for (int mu = 0; mu < K1; ++mu) ca.wr[mu] = pa.wr[mu];
      OpArgs wa;
      fill_op_args(h, l, wa);
      e = h->dim == 2 ? dispatch_cip_weights_2d(h, wa, m->Urep, h->d_cipw_res, h->stream)
                      : dispatch_cip_weights_3d(h, wa, m->Urep, h->d_cipw_res, h->stream);
      if (e != cudaSuccess) break;
    }
    if (prec == ST_FP64) {
      if (h->dim == 2) patch_assemble<2, double><<<g, 256, 0, h->stream>>>((const double*)Esrc, estride, pa, (double*)m->L[l].LU);
      else patch_assemble<3, double><<<g, 256, 0, h->stream>>>((const double*)Esrc, estride, pa, (double*)m->L[l].LU);
      e = cudaGetLastError();
      if (e == cudaSuccess && cip) {
        if (h->dim == 2) cip_patch_add<2, double><<<g, 256, 0, h->stream>>>(ca, h->d_cipw_res, (double*)m->L[l].LU);
        else cip_patch_add<3, double><<<g, 256, 0, h->stream>>>(ca, h->d_cipw_res, (double*)m->L[l].LU);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess)
        e = c13 ? invert_patches_cplx<double>((double*)m->L[l].LU, NE, nblk, h->d_err, h->nsm, h->stream)
                : invert_patches<double>((double*)m->L[l].LU, m->L[l].piv, N, Lv.ncells, h->d_err, h->nsm, h->stream);
    } else {
      if (h->dim == 2) patch_assemble<2, float><<<g, 256, 0, h->stream>>>((const float*)Esrc, estride, pa, (float*)m->L[l].LU);
      else patch_assemble<3, float><<<g, 256, 0, h->stream>>>((const float*)Esrc, estride, pa, (float*)m->L[l].LU);
      e = cudaGetLastError();
      if (e == cudaSuccess && cip) {
        if (h->dim == 2) cip_patch_add<2, float><<<g, 256, 0, h->stream>>>(ca, h->d_cipw_res, (float*)m->L[l].LU);
        else cip_patch_add<3, float><<<g, 256, 0, h->stream>>>(ca, h->d_cipw_res, (float*)m->L[l].LU);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess)
        e = c13 ? invert_patches_cplx<float>((float*)m->L[l].LU, NE, nblk, h->d_err, h->nsm, h->stream)
                : invert_patches<float>((float*)m->L[l].LU, m->L[l].piv, N, Lv.ncells, h->d_err, h->nsm, h->stream);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_check(h, e, "st_precond_setup patches");
  int flag = 0;
  e = cudaMemcpyAsync(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_check(h, e, "st_precond_setup");
  if (flag) return set_error(h, ST_SINGULAR_PATCH, "st_precond_setup: a patch matrix (or the coarsest-level matrix) "
                                                   "has a zero pivot");
  h->precond_valid = true;
  h->precond_prec = prec;
  return ST_OK;
}

st_status mg_vanka(st_problem* h, int level, int sweeps, st_prec prec, const void* r, void* d) {
  MgState* m = (MgState*)h->mg;
  cudaError_t e = prec == ST_FP64 ? vanka_steps<double>(h, m, level, sweeps, (const double*)r, (double*)d)
                                  : vanka_steps<float>(h, m, level, sweeps, (const float*)r, (float*)d);
  return cuda_check(h, e, "st_vanka_smooth");
}

// One V-cycle.  The launch sequence depends only on the buffers, the
// precision and the tangent (the hierarchy's contents change between calls,
// its storage does not), so it is captured once as a CUDA graph and replayed:
// the first call with a new (r, d, precision, tangent) runs eagerly, the
// second captures, later ones launch the graph.
// The V-cycle runs on the problem's internal capture stream (the caller's
// stream may be the legacy default stream, which cannot be captured),
// ordered after and before the caller's stream by events.
cudaError_t vcycle_on_cap(st_problem* h, MgState* m, st_prec prec, const void* r, void* d) {
  const int L = (int)h->lev.size() - 1;
  auto run = [&]() {
    return prec == ST_FP64 ? vcycle_rec<double>(h, m, L, (const double*)r, (double*)d)
                           : vcycle_rec<float>(h, m, L, (const float*)r, (float*)d);
  };
  const bool same = m->g_seen && m->g_r == r && m->g_d == d && m->g_prec == (int)prec &&
                    m->g_tangent == h->lin_tangent;
  if (same && m->gexec) return cudaGraphLaunch(m->gexec, h->stream);
  if (!same || m->g_failed) {
    if (!same) {
      drop_graph(m);
      m->g_r = r;
      m->g_d = d;
      m->g_prec = (int)prec;
      m->g_tangent = h->lin_tangent;
      m->g_seen = true;
    }
    return run();
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const cudaError_t er = run();
    e = cudaStreamEndCapture(h->stream, &g);
    if (er != cudaSuccess) e = er;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&m->gexec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {  // capture unavailable: stay eager for this key
    m->gexec = nullptr;
    m->g_failed = true;
    cudaGetLastError();
    return run();
  }
  return cudaGraphLaunch(m->gexec, h->stream);
}

st_status mg_vcycle(st_problem* h, st_prec prec, const void* r, void* d) {
  MgState* m = (MgState*)h->mg;
  cudaStream_t user = h->stream;
  cudaError_t e = cudaEventRecord(h->ev_cap0, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_cap, h->ev_cap0, 0);
  if (e != cudaSuccess) return cuda_check(h, e, "st_vcycle");
  h->stream = h->s_cap;
  e = vcycle_on_cap(h, m, prec, r, d);
  h->stream = user;
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_cap1, h->s_cap);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, h->ev_cap1, 0);
  return cuda_check(h, e, "st_vcycle");
}

}  // namespace st

using namespace st;

extern "C" {

st_status st_precond_setup(st_problem* h, st_prec prec) {
  if (!h) return ST_EINVAL;
  if (prec != ST_FP64 && prec != ST_FP32) return set_error(h, ST_EINVAL, "st_precond_setup: bad precision");
  return mg_setup(h, prec, true);
}

st_status st_vanka_smooth(st_problem* h, int level, int sweeps, st_prec prec, const void* r, void* d) {
  if (!h) return ST_EINVAL;
  if (level < 0 || level >= (int)h->lev.size()) return set_error(h, ST_EINVAL, "st_vanka_smooth: bad level");
  if (sweeps < 0 || !r || !d) return set_error(h, ST_EINVAL, "st_vanka_smooth: bad arguments");
  if (prec != ST_FP64 && prec != ST_FP32) return set_error(h, ST_EINVAL, "st_vanka_smooth: bad precision");
  if (!h->precond_valid || h->precond_prec != prec) {
    st_status s = mg_setup(h, prec, true);
    if (s != ST_OK) return s;
  }
  return mg_vanka(h, level, sweeps, prec, r, d);
}

st_status st_vcycle(st_problem* h, st_prec prec, const void* r, void* d) {
  if (!h) return ST_EINVAL;
  if (!r || !d) return set_error(h, ST_EINVAL, "st_vcycle: r and d are required");
  if (prec != ST_FP64 && prec != ST_FP32) return set_error(h, ST_EINVAL, "st_vcycle: bad precision");
  if (!h->precond_valid || h->precond_prec != prec) {
    st_status s = mg_setup(h, prec, true);
    if (s != ST_OK) return s;
  }
  return mg_vcycle(h, prec, r, d);
}

}  // extern "C"
