// Coarsest-level direct solve (see st_coarse.cuh).
#include <climits>
#include <cstdio>

#include "st_coarse.cuh"

namespace st {

namespace {

constexpr int CB = 16;                      // panel width of the blocked Gauss-Jordan inversion
constexpr int PT = 1024;                    // threads of the panel kernel
constexpr size_t PANEL_SMEM_MAX = 200 * 1024;
constexpr int RT = 1024;                    // threads of the single-CTA refinement kernels

// ----------------------------------------------------------------- assembly
// A += the space-time element matrices of the cells of parity class `cls`
// (cells (c_x + 2i, c_y + 2j, c_z + 2l)); cells of one class share no dof, so
// the read-modify-write adds do not race.  One CTA per cell.
template <int DIM, typename T>
__global__ void __launch_bounds__(256) coarse_dense_add(const T* __restrict__ E, CoarseGeom g, int cls,
                                                        double* __restrict__ A, long n) {
  constexpr int NQ = DIM == 3 ? 27 : 9, NC = DIM, NP = DIM == 3 ? 8 : 4, NE = NC * NQ + NP;
  __shared__ long sg[MAX_K1 * NE];
  __shared__ double smass[NQ * NQ];
  const int K1 = g.K1, N = K1 * NE;
  const int c3[3] = {cls & 1, (cls >> 1) & 1, (cls >> 2) & 1};
  int m[3];
  for (int d = 0; d < 3; ++d) m[d] = d < DIM ? (g.n[d] - c3[d] + 1) / 2 : 1;
  const long ncls = (long)m[0] * m[1] * m[2];
  for (int t = threadIdx.x; t < NQ * NQ; t += blockDim.x) {
    const int a = t / NQ, b = t % NQ;
    const int ai[3] = {a % 3, (a / 3) % 3, a / 9}, bi[3] = {b % 3, (b / 3) % 3, b / 9};
    double v = 1.0;
    for (int d = 0; d < DIM; ++d) v *= g.M1h[d][ai[d] * 3 + bi[d]];
    smass[t] = v;
  }
  for (long li = blockIdx.x; li < ncls; li += gridDim.x) {
    const int ex = c3[0] + 2 * (int)(li % m[0]);
    const int ey = c3[1] + 2 * (int)((li / m[0]) % m[1]);
    const int ez = DIM == 3 ? c3[2] + 2 * (int)(li / ((long)m[0] * m[1])) : 0;
    const long cell = ex + (long)g.n[0] * (ey + (long)g.n[1] * ez);
    __syncthreads();  // smass ready; the previous cell's indices are no longer read
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      const int mu = r / NE, loc = r % NE;
      long gi;
      if (loc < NC * NQ) {
        const int c = loc / NQ, q = loc % NQ;
        gi = (long)mu * g.Mv + c * g.Nq2 + (2L * ex + q % 3) +
             g.g2[0] * ((2L * ey + (q / 3) % 3) + g.g2[1] * (2L * ez + q / 9));
      } else {
        const int mm = loc - NC * NQ;
        if (g.pdisc)  // the cell's coefficients; local pressure dofs beyond them are unused
          gi = mm <= DIM ? (long)K1 * g.Mv + (long)mu * g.Mp + cell * (DIM + 1) + mm : -1;
        else
          gi = (long)K1 * g.Mv + (long)mu * g.Mp + (ex + (mm & 1)) +
               g.g1[0] * ((ey + ((mm >> 1) & 1)) + g.g1[1] * (ez + (mm >> 2)));
      }
      sg[r] = gi;
    }
    __syncthreads();
    for (long t = threadIdx.x; t < (long)N * N; t += blockDim.x) {
      const int rr = (int)(t / N), cc = (int)(t % N);
      if (sg[rr] < 0 || sg[cc] < 0) continue;
      const int mu = rr / NE, i = rr % NE, nu = cc / NE, j = cc % NE;
      double v = 0.0;
      constexpr int NV = NC * NQ;
      if (mu == nu) {
        const T* Em = E + (cell * K1 + mu) * (long)NE * NE;
        if (g.pdisc && i >= NV && j >= NV) {
          for (int m = 0; m < NP; ++m)
            for (int m2 = 0; m2 < NP; ++m2)
              v += pdisc_T(m, i - NV) * (double)Em[(NV + m) * NE + NV + m2] * pdisc_T(m2, j - NV);
        } else if (g.pdisc && i >= NV) {
          for (int m = 0; m < NP; ++m) v += pdisc_T(m, i - NV) * (double)Em[(NV + m) * NE + j];
        } else if (g.pdisc && j >= NV) {
          for (int m = 0; m < NP; ++m) v += (double)Em[i * NE + NV + m] * pdisc_T(m, j - NV);
        } else {
          v = (double)Em[i * NE + j];
        }
      }
      if (i < NC * NQ && j < NC * NQ && i / NQ == j / NQ) v += g.Kt[mu * K1 + nu] * smass[(i % NQ) * NQ + (j % NQ)];
      A[sg[rr] * n + sg[cc]] += v;
    }
  }
}

template <typename A_, typename B_>
__global__ void cast_copy(const A_* __restrict__ x, B_* __restrict__ y, size_t len) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (B_)x[i];
}

// ---------------------------------------------------------------- inversion
// Blocked in-place Gauss-Jordan inversion of the row-major n x n FP32 matrix A
// with partial pivoting (row swaps).  Panel K = columns kb .. kb+bw-1:
//   1. gj_panel: unblocked Gauss-Jordan on the n x bw panel (all rows): for
//      each column j of K, pivot p = argmax_{i >= j} |a_ij| (lowest index on
//      ties), swap rows j and p within the panel, scale the pivot row by 1/a_jj
//      with the pivot entry replaced by 1/a_jj, and eliminate column j from
//      every other row, the entry itself becoming -a_ij / a_jj.  Afterwards
//      the panel columns hold the columns K of the accumulated elimination
//      matrix G = G_{kb+bw-1} ... G_{kb}.
//   2. gj_swap: the same row swaps on every column outside K; the pivot rows
//      (outside K) are copied to T.
//   3. gj_update: the deferred row operations on the columns outside K,
//      A[:, J] <- G A[:, J] = A[:, J] + (A[:, K] - I[:, K]) T.
// After the last panel A holds (P A)^{-1}, P the row permutation of the
// pivots.  A zero pivot sets err[0] (the pivot is then taken as 1).
template <bool STAGED>
__global__ void __launch_bounds__(PT) gj_panel(float* __restrict__ A, long n, long kb, int bw, int* __restrict__ piv,
                                               int* __restrict__ err) {
  extern __shared__ float sp[];
  __shared__ float rv[PT / 32];
  __shared__ int ri[PT / 32];
  __shared__ int s_p;
  float* P;
  long ld;
  if (STAGED) {
    P = sp;
    ld = CB + 1;  // padded: consecutive rows fall into different banks
    for (long t = threadIdx.x; t < n * bw; t += PT) {
      const long i = t / bw;
      const int c = (int)(t % bw);
      P[i * ld + c] = A[i * n + kb + c];
    }
    __syncthreads();
  } else {
    P = A + kb;
    ld = n;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int jj = 0; jj < bw; ++jj) {
    const long j = kb + jj;
    float best = -1.0f;
    int bi = INT_MAX;
    for (long i = j + threadIdx.x; i < n; i += PT) {
      const float v = fabsf(P[i * ld + jj]);
      if (v > best) {
        best = v;
        bi = (int)i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      rv[warp] = best;
      ri[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
      best = rv[lane];
      bi = ri[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        if (!(best > 0.0f) || bi >= n) {
          err[0] = 1;
          bi = (int)j;
        }
        s_p = bi;
        piv[j] = bi;
      }
    }
    __syncthreads();
    const long p = s_p;
    if (p != j && threadIdx.x < bw) {
      const int c = threadIdx.x;
      const float t = P[j * ld + c];
      P[j * ld + c] = P[p * ld + c];
      P[p * ld + c] = t;
    }
    __syncthreads();
    float a = P[j * ld + jj];
    if (a == 0.0f) a = 1.0f;
    __syncthreads();
    if (threadIdx.x < bw) {
      const int c = threadIdx.x;
      P[j * ld + c] = (c == jj) ? 1.0f / a : P[j * ld + c] / a;
    }
    __syncthreads();
    for (long i = threadIdx.x; i < n; i += PT) {
      if (i == j) continue;
      const float f = P[i * ld + jj];
      if (f == 0.0f) continue;
      for (int c = 0; c < bw; ++c) {
        const float pj = P[j * ld + c];
        P[i * ld + c] = (c == jj) ? -f * pj : fmaf(-f, pj, P[i * ld + c]);
      }
    }
    __syncthreads();
  }
  if (STAGED) {
    for (long t = threadIdx.x; t < n * bw; t += PT) {
      const long i = t / bw;
      const int c = (int)(t % bw);
      A[i * n + kb + c] = P[i * ld + c];
    }
  }
}

__global__ void gj_swap(float* __restrict__ A, long n, long kb, int bw, const int* __restrict__ piv,
                        float* __restrict__ T) {
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    if (c >= kb && c < kb + bw) continue;
    for (int jj = 0; jj < bw; ++jj) {
      const long j = kb + jj, p = piv[j];
      if (p != j) {
        const float t = A[j * n + c];
        A[j * n + c] = A[p * n + c];
        A[p * n + c] = t;
      }
    }
    for (int jj = 0; jj < bw; ++jj) T[jj * n + c] = A[(kb + jj) * n + c];
  }
}

// 64 x 64 output tile per CTA, 256 threads with 4 x 4 outputs each
__global__ void __launch_bounds__(256) gj_update(float* __restrict__ A, long n, long kb, int bw,
                                                 const float* __restrict__ T) {
  __shared__ float sX[CB][68];
  __shared__ float sT[CB][68];
  const long r0 = (long)blockIdx.y * 64, c0 = (long)blockIdx.x * 64;
  if (c0 >= kb && c0 + 64 <= kb + bw) return;  // the tile lies inside the panel columns
  for (int t = threadIdx.x; t < 64 * CB; t += 256) {
    const int i = t / CB, jj = t % CB;
    const long row = r0 + i;
    float v = 0.0f;
    if (row < n && jj < bw) v = A[row * n + kb + jj] - (row == kb + jj ? 1.0f : 0.0f);
    sX[jj][i] = v;
  }
  for (int t = threadIdx.x; t < CB * 64; t += 256) {
    const int jj = t / 64, cc = t % 64;
    const long col = c0 + cc;
    sT[jj][cc] = (col < n && jj < bw) ? T[jj * n + col] : 0.0f;
  }
  __syncthreads();
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
#pragma unroll
  for (int jj = 0; jj < CB; ++jj) {
    float x[4], t[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) x[a] = sX[jj][ty * 4 + a];
#pragma unroll
    for (int b = 0; b < 4; ++b) t[b] = sT[jj][tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(x[a], t[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const long row = r0 + ty * 4 + a;
    if (row >= n) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const long col = c0 + tx + 16 * b;
      if (col >= n || (col >= kb && col < kb + bw)) continue;
      A[row * n + col] += acc[a][b];
    }
  }
}

// composed row permutation of the pivots: (P v)_j = v[perm[j]]
__global__ void gj_perm(const int* __restrict__ piv, int* __restrict__ perm, long n) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (long i = 0; i < n; ++i) perm[i] = (int)i;
  for (long j = 0; j < n; ++j) {
    const int p = piv[j];
    const int t = perm[j];
    perm[j] = perm[p];
    perm[p] = t;
  }
}

// --------------------------------------------------------------- refinement
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  return red[0];
}

template <typename T>
__global__ void __launch_bounds__(RT) cd_init(const T* __restrict__ rin, CoarseDirect cd) {
  __shared__ double red[RT / 32];
  double s = 0.0;
  for (long i = threadIdx.x; i < cd.n; i += RT) {
    const double v = (double)rin[i];
    cd.b[i] = v;
    cd.r[i] = v;
    cd.x[i] = 0.0;
    s += v * v;
  }
  __syncthreads();
  for (long j = threadIdx.x; j < cd.n; j += RT) cd.rp[j] = (float)cd.b[cd.perm[j]];
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    cd.st->b2 = s;
    cd.st->r2 = s;
    cd.st->done = s > 0.0 ? 0 : 1;
    cd.st->steps = 0;
    cd.st->diverged = 0;
    cd.st->accept = 0;
  }
}

// xn = x + R (P r): FP32 product with the FP32 inverse, FP64 sum; one warp per row
__global__ void cd_gemv32(CoarseDirect cd) {
  if (cd.st->done) return;
  const int lane = threadIdx.x & 31;
  const long w0 = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
  const long nw = ((long)gridDim.x * blockDim.x) >> 5;
  for (long i = w0; i < cd.n; i += nw) {
    const float* Ri = cd.R + i * cd.n;
    float s = 0.0f;
    for (long j = lane; j < cd.n; j += 32) s = fmaf(Ri[j], cd.rp[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) cd.xn[i] = cd.x[i] + (double)s;
  }
}

// rn = b - A xn in FP64; one warp per row
__global__ void cd_gemv64(CoarseDirect cd) {
  if (cd.st->done) return;
  const int lane = threadIdx.x & 31;
  const long w0 = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
  const long nw = ((long)gridDim.x * blockDim.x) >> 5;
  for (long i = w0; i < cd.n; i += nw) {
    const double* Ai = cd.A + i * cd.n;
    double s = 0.0;
    for (long j = lane; j < cd.n; j += 32) s = fma(Ai[j], cd.xn[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) cd.rn[i] = cd.b[i] - s;
  }
}

// accept the trial iterate when its residual decreased; stop at the
// tolerance, or when the residual no longer decreases (keep the best iterate)
__global__ void __launch_bounds__(RT) cd_decide(CoarseDirect cd, double rtol2) {
  __shared__ double red[RT / 32];
  __shared__ int acc;
  if (cd.st->done) return;
  double s = 0.0;
  for (long i = threadIdx.x; i < cd.n; i += RT) s += cd.rn[i] * cd.rn[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    if (s < cd.st->r2) {
      acc = 1;
      cd.st->r2 = s;
      cd.st->steps += 1;
      if (s <= rtol2 * cd.st->b2) cd.st->done = 1;
    } else {
      acc = 0;
      cd.st->diverged = 1;
      cd.st->done = 1;
    }
  }
  __syncthreads();
  if (!acc) return;
  for (long i = threadIdx.x; i < cd.n; i += RT) {
    cd.x[i] = cd.xn[i];
    cd.r[i] = cd.rn[i];
  }
  __syncthreads();
  for (long j = threadIdx.x; j < cd.n; j += RT) cd.rp[j] = (float)cd.r[cd.perm[j]];
}

template <typename T>
__global__ void cd_final(CoarseDirect cd, T* __restrict__ d) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < cd.n; i += (long)gridDim.x * blockDim.x)
    d[i] = (T)cd.x[i];
}

unsigned grid_of(size_t n, int threads, int nsm) {
  size_t g = (n + threads - 1) / threads;
  const size_t cap = 16 * (size_t)(nsm > 0 ? nsm : 1);
  if (g > cap) g = cap;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t coarse_direct_alloc(CoarseDirect& cd, long n) {
  coarse_direct_free(cd);
  cd.n = n;
  cudaError_t e = cudaMalloc(&cd.A, (size_t)n * n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&cd.R, (size_t)n * n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&cd.T, (size_t)CB * n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&cd.piv, (size_t)n * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&cd.perm, (size_t)n * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&cd.b, (size_t)5 * n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&cd.rp, (size_t)n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&cd.st, sizeof(CoarseState));
  if (e == cudaSuccess) {
    cd.x = cd.b + n;
    cd.r = cd.b + 2 * n;
    cd.xn = cd.b + 3 * n;
    cd.rn = cd.b + 4 * n;
  }
  return e;
}

void coarse_direct_free(CoarseDirect& cd) {
  cudaFree(cd.A);
  cudaFree(cd.R);
  cudaFree(cd.T);
  cudaFree(cd.piv);
  cudaFree(cd.perm);
  cudaFree(cd.b);
  cudaFree(cd.rp);
  cudaFree(cd.st);
  cd = CoarseDirect();
}

template <typename T>
cudaError_t coarse_direct_setup(const CoarseGeom& g, const T* E, CoarseDirect& cd, int* err, int nsm,
                                cudaStream_t s) {
  const long n = cd.n;
  cudaError_t e = cudaMemsetAsync(cd.A, 0, (size_t)n * n * sizeof(double), s);
  const int ncls = 1 << g.dim;
  for (int c = 0; c < ncls && e == cudaSuccess; ++c) {
    long m = 1;
    for (int d = 0; d < g.dim; ++d) m *= (g.n[d] - ((c >> d) & 1) + 1) / 2;
    if (m <= 0) continue;
    const unsigned grid = (unsigned)(m < 8L * nsm ? m : 8L * nsm);
    if (g.dim == 2) coarse_dense_add<2, T><<<grid, 256, 0, s>>>(E, g, c, cd.A, n);
    else coarse_dense_add<3, T><<<grid, 256, 0, s>>>(E, g, c, cd.A, n);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  cast_copy<double, float><<<grid_of((size_t)n * n, 256, nsm), 256, 0, s>>>(cd.A, cd.R, (size_t)n * n);
  e = cudaGetLastError();
  const size_t smem = (size_t)n * (CB + 1) * sizeof(float);
  const bool staged = smem <= PANEL_SMEM_MAX;
  if (e == cudaSuccess && staged)
    e = cudaFuncSetAttribute(gj_panel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const dim3 ug((unsigned)((n + 63) / 64), (unsigned)((n + 63) / 64));
  for (long kb = 0; kb < n && e == cudaSuccess; kb += CB) {
    const int bw = (int)(n - kb < CB ? n - kb : CB);
    if (staged) gj_panel<true><<<1, PT, smem, s>>>(cd.R, n, kb, bw, cd.piv, err);
    else gj_panel<false><<<1, PT, 0, s>>>(cd.R, n, kb, bw, cd.piv, err);
    gj_swap<<<grid_of((size_t)n, 256, nsm), 256, 0, s>>>(cd.R, n, kb, bw, cd.piv, cd.T);
    gj_update<<<ug, 256, 0, s>>>(cd.R, n, kb, bw, cd.T);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    gj_perm<<<1, 1, 0, s>>>(cd.piv, cd.perm, n);
    e = cudaGetLastError();
  }
  return e;
}

template <typename T>
cudaError_t coarse_direct_solve(CoarseDirect& cd, const T* r, T* d, int max_steps, double rtol, int nsm,
                                cudaStream_t s) {
  cd_init<T><<<1, RT, 0, s>>>(r, cd);
  cudaError_t e = cudaGetLastError();
  const unsigned gw = grid_of((size_t)cd.n * 32, 256, nsm);
  for (int it = 0; it < max_steps && e == cudaSuccess; ++it) {
    cd_gemv32<<<gw, 256, 0, s>>>(cd);
    cd_gemv64<<<gw, 256, 0, s>>>(cd);
    cd_decide<<<1, RT, 0, s>>>(cd, rtol * rtol);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    cd_final<T><<<grid_of((size_t)cd.n, 256, nsm), 256, 0, s>>>(cd, d);
    e = cudaGetLastError();
  }
  return e;
}

template cudaError_t coarse_direct_setup<double>(const CoarseGeom&, const double*, CoarseDirect&, int*, int,
                                                 cudaStream_t);
template cudaError_t coarse_direct_setup<float>(const CoarseGeom&, const float*, CoarseDirect&, int*, int,
                                                cudaStream_t);
template cudaError_t coarse_direct_solve<double>(CoarseDirect&, const double*, double*, int, double, int,
                                                 cudaStream_t);
template cudaError_t coarse_direct_solve<float>(CoarseDirect&, const float*, float*, int, double, int,
                                                cudaStream_t);

}  // namespace st
