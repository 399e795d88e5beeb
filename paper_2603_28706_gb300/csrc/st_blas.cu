// Vector kernels (see st_blas.cuh).
#include <cmath>
#include <cstdio>
#include <mutex>
#include <vector>

#include "st_blas.cuh"

namespace st {

namespace {

constexpr int BT = 256;
constexpr int NPART = 512;  // partial sums of the two-stage reductions

template <typename A, typename B>
__global__ void cast_kernel(const A* __restrict__ x, B* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (B)x[i];
}

// multiprocessor count of the current device, read once per device
int sm_count() {
  static std::mutex mu;
  static int cached[256] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return 1;
  std::lock_guard<std::mutex> lock(mu);
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    cached[dev] = n;
  }
  return cached[dev];
}

// grid-stride launches: at most 16 CTAs of BT threads per SM
size_t grid_cap() { return 16 * (size_t)sm_count(); }

unsigned grid_for(size_t n) {
  size_t g = (n + BT - 1) / BT;
  const size_t cap = grid_cap();
  if (g > cap) g = cap;
  return (unsigned)(g < 1 ? 1 : g);
}

// One direction of the global 1D mass operator on a tensor grid of
// g[0] x g[1] x g[2] points, applied to `nblk` consecutive blocks:
//   Q2 (order 2): cells [2e, 2e+2], local matrix h * M1 (3x3)
//   Q1 (order 1): cells [e, e+1], local matrix h * [[1/3, 1/6], [1/6, 1/3]]
// y_i = scale_b * sum over cells containing i of sum_b M_loc[i - start][b] x[start + b]
template <typename T, int ORDER>
__global__ void mass_pass(const T* __restrict__ x, T* __restrict__ y, long g0, long g1, long g2, int dir, double hd,
                          int nblk, const double* __restrict__ bscale,
                          int comps_per_node, T m00, T m01, T m02, T m11, T m12, T m22) {
  const long npt = g0 * g1 * g2;
  const long total = npt * nblk;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long b = t / npt, r = t % npt;
    const long ix = r % g0, iy = (r / g0) % g1, iz = r / (g0 * g1);
    const long gd = dir == 0 ? g0 : (dir == 1 ? g1 : g2);
    const long id = dir == 0 ? ix : (dir == 1 ? iy : iz);
    const long st = dir == 0 ? 1 : (dir == 1 ? g0 : g0 * g1);
    const T* xb = x + b * npt + (r - id * st);
    T acc = 0;
    // local symmetric matrix entries
    auto M = [&](int i, int j) -> T {
      if (ORDER == 2) {
        const int a = i < j ? i : j, c = i < j ? j : i;
        if (a == 0) return c == 0 ? m00 : (c == 1 ? m01 : m02);
        if (a == 1) return c == 1 ? m11 : m12;
        return m22;
      } else {
        return i == j ? m00 : m01;
      }
    };
    const long ncell = (gd - 1) / ORDER;
    // cells whose node range contains id
    long e_lo = (id - 1) / ORDER, e_hi = id / ORDER;
    if (id == 0) e_lo = 0;
    if (e_hi > ncell - 1) e_hi = ncell - 1;
    if (e_lo < 0) e_lo = 0;
    for (long e = e_lo; e <= e_hi; ++e) {
      const long s0 = e * ORDER;
      const int a = (int)(id - s0);
      if (a < 0 || a > ORDER) continue;
      for (int c = 0; c <= ORDER; ++c) acc += M(a, c) * xb[(s0 + c) * st];
    }
    const double sc = bscale ? bscale[b / comps_per_node] : 1.0;
    y[t] = acc * (T)(hd * sc);
  }
}

__global__ void partial_dot(const double* __restrict__ x, const double* __restrict__ y, size_t n,
                            double* __restrict__ part) {
  __shared__ double sh[BT];
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)BT + threadIdx.x; i < n; i += (size_t)gridDim.x * BT) acc += x[i] * y[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = BT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void partial_multidot(const double* __restrict__ V, size_t ld, int nv, const double* __restrict__ w,
                                 size_t n, double* __restrict__ part) {
  __shared__ double sh[BT];
  const int j = blockIdx.y;
  const double* v = V + j * ld;
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)BT + threadIdx.x; i < n; i += (size_t)gridDim.x * BT) acc += v[i] * w[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = BT / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)j * gridDim.x + blockIdx.x] = sh[0];
}

// fixed-order final sum of np partials per output
__global__ void finish_sum(const double* __restrict__ part, int np, int nout, double* __restrict__ res) {
  __shared__ double sh[BT];
  for (int j = 0; j < nout; ++j) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += BT) acc += part[(size_t)j * np + i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = BT / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) res[j] = sh[0];
    __syncthreads();
  }
}

__global__ void multiaxpy_kernel(const double* __restrict__ V, size_t ld, int nv, const double* __restrict__ c,
                                 double* __restrict__ w, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int j = 0; j < nv; ++j) acc -= c[j] * V[j * ld + i];
    w[i] = acc;
  }
}

__global__ void lincomb_kernel(const double* __restrict__ Z, size_t ld, int nv, const double* __restrict__ c,
                               double* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < nv; ++j) acc += c[j] * Z[j * ld + i];
    y[i] = acc;
  }
}

__global__ void axpby_kernel(double a, const double* __restrict__ x, double b, double* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

__global__ void scale_inv_kernel(const double* __restrict__ x, const double* __restrict__ s, double* __restrict__ y,
                                 size_t n) {
  const double inv = 1.0 / s[0];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = x[i] * inv;
}

}  // namespace

cudaError_t cast_f64_f32(const double* x, float* y, size_t n, cudaStream_t s) {
  cast_kernel<double, float><<<grid_for(n), BT, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t cast_f32_f64(const float* x, double* y, size_t n, cudaStream_t s) {
  cast_kernel<float, double><<<grid_for(n), BT, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

// P1disc pressure mass (block diagonal): on a cell of volume |K| the basis
// 1, 2 r_a - 1 is orthogonal with integrals |K| and |K|/3, so
// y = tau w_mu |K| diag(1, 1/3, .., 1/3) x per cell and time node.
template <typename T>
__global__ void pdisc_mass(const T* __restrict__ x, T* __restrict__ y, long ncells, int nl, int K1,
                           const double* __restrict__ bscale, double vol) {
  const long per = ncells * nl, total = per * K1;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int mu = (int)(i / per), j = (int)((i % per) % nl);
    y[i] = (T)(bscale[mu] * vol * (j == 0 ? 1.0 : 1.0 / 3.0) * (double)x[i]);
  }
}

template <typename T>
cudaError_t mass_apply(const st_problem* h, int level, const T* x, T* y, T* work) {
  const Level& L = h->lev[level];
  const int d = h->dim, K1 = h->K1;
  double* bs = h->d_scratch + 2048;  // tau*w_mu per time node (set below)
  double tw[MAX_K1];
  for (int i = 0; i < K1; ++i) tw[i] = h->P.dt * h->T.w[i];
  cudaError_t e = cudaMemcpyAsync(bs, tw, K1 * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return e;
  const double* M = h->R.M1;
  T* t1 = work;
  T* t2 = work + L.Nst;
  // velocity: K1*d blocks of Nq2 on the Q2 grid; pressure: K1 blocks on the Q1 grid
  for (int part = 0; part < 2; ++part) {
    if (part == 1 && h->P.pressure_space == 1) {
      const size_t off = (size_t)K1 * L.Mv;
      const double vol = L.h[0] * L.h[1] * (d == 3 ? L.h[2] : 1.0);
      pdisc_mass<T><<<grid_for((size_t)K1 * L.Mp), BT, 0, h->stream>>>(x + off, y + off, L.ncells, d + 1, K1, bs,
                                                                        vol);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      continue;
    }
    const long* g = part == 0 ? L.g2 : L.g1;
    const long npt = g[0] * g[1] * g[2];
    const int nblk = part == 0 ? K1 * d : K1;
    const size_t off = part == 0 ? 0 : (size_t)K1 * L.Mv;
    const T* src = x + off;
    T* bufs[2] = {t1 + off, t2 + off};
    for (int dir = 0; dir < d; ++dir) {
      T* dst = (dir == d - 1) ? y + off : bufs[dir & 1];
      const double* sc = (dir == d - 1) ? bs : nullptr;
      const int cpn = part == 0 ? d : 1;
      const long total = npt * nblk;
      unsigned grid = (unsigned)((total + BT - 1) / BT);
      if (grid > grid_cap()) grid = (unsigned)grid_cap();
      if (part == 0)
        mass_pass<T, 2><<<grid, BT, 0, h->stream>>>(src, dst, g[0], g[1], g[2], dir, L.h[dir], nblk, sc, cpn,
                                                     (T)M[0], (T)M[1], (T)M[2], (T)M[4], (T)M[5], (T)M[8]);
      else
        mass_pass<T, 1><<<grid, BT, 0, h->stream>>>(src, dst, g[0], g[1], g[2], dir, L.h[dir], nblk, sc, cpn,
                                                     (T)(1.0 / 3.0), (T)(1.0 / 6.0), (T)0, (T)0, (T)0, (T)0);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      src = dst;
    }
  }
  return cudaSuccess;
}

template cudaError_t mass_apply<double>(const st_problem*, int, const double*, double*, double*);
template cudaError_t mass_apply<float>(const st_problem*, int, const float*, float*, float*);

cudaError_t dot_f64(const double* x, const double* y, size_t n, double* dres, double* partial, cudaStream_t s) {
  partial_dot<<<NPART, BT, 0, s>>>(x, y, n, partial);
  finish_sum<<<1, BT, 0, s>>>(partial, NPART, 1, dres);
  return cudaGetLastError();
}

cudaError_t multidot_f64(const double* V, size_t ld, int nv, const double* w, size_t n, double* dres, double* partial,
                         cudaStream_t s) {
  if (nv <= 0) return cudaSuccess;
  const int np = 128;
  partial_multidot<<<dim3(np, nv), BT, 0, s>>>(V, ld, nv, w, n, partial);
  finish_sum<<<1, BT, 0, s>>>(partial, np, nv, dres);
  return cudaGetLastError();
}

cudaError_t multiaxpy_f64(const double* V, size_t ld, int nv, const double* c, double* w, size_t n, cudaStream_t s) {
  multiaxpy_kernel<<<grid_for(n), BT, 0, s>>>(V, ld, nv, c, w, n);
  return cudaGetLastError();
}

cudaError_t lincomb_f64(const double* Z, size_t ld, int nv, const double* c, double* y, size_t n, cudaStream_t s) {
  lincomb_kernel<<<grid_for(n), BT, 0, s>>>(Z, ld, nv, c, y, n);
  return cudaGetLastError();
}

cudaError_t axpby_f64(double a, const double* x, double b, double* y, size_t n, cudaStream_t s) {
  axpby_kernel<<<grid_for(n), BT, 0, s>>>(a, x, b, y, n);
  return cudaGetLastError();
}

cudaError_t scale_inv_f64(const double* x, const double* sdev, double* y, size_t n, cudaStream_t s) {
  scale_inv_kernel<<<grid_for(n), BT, 0, s>>>(x, sdev, y, n);
  return cudaGetLastError();
}

cudaError_t mnorm2_f64(st_problem* h, int level, const double* r, double* out) {
  const Level& L = h->lev[level];
  double* Mr = h->d_work;
  double* work = h->d_work + L.Nst;
  cudaError_t e = mass_apply<double>(h, level, r, Mr, work);
  if (e == cudaSuccess) e = dot_f64(r, Mr, L.Nst, h->d_scratch, h->d_scratch + 8, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, h->d_scratch, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e;
}

}  // namespace st

// ----------------------------------------------------------------------------
// Allocation-free block mass norm (st_mnorm_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs while another framework
// owns the device memory pool with a hard cap, plugins whose host forbids
// device allocations, or latency-critical paths that must not touch the
// allocator.  For them this entry point computes |r|_M without a handle and
// without any allocation: its work vectors and reduction partial sums live in
// the file-scope array below, which every GPU that loads the library keeps
// until the process exits.
//   scratch[0 .. 8)           tau * w_mu per Radau node (mass scaling)
//   scratch[8 .. 8 + 512)     partial sums of the dot product
//   scratch[1024]             the result
//   scratch[2048 ..)          two work vectors of the slab size
// The slab size is therefore limited to (ST_NOALLOC_DOUBLES - 2048) / 2.
// Every entry that a call reads is written earlier in that call, so nothing
// has to start at zero.  All calls share the array: calls that overlap on the
// GPU (two streams, or two host threads) race and must be serialised by the
// caller.
constexpr size_t ST_NOALLOC_DOUBLES = (size_t)1 << 21;  // 16 MiB
static __device__ __align__(256) double g_noalloc_scratch[ST_NOALLOC_DOUBLES];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[256] = {};  // device address of the array, per device
}  // namespace

extern "C" st_status st_mnorm_noalloc(const st_params* P, void* cuda_stream, const double* r, double* out) {
  using namespace st;
  if (!P) return ST_EINVAL;
  const int d = P->dim;
  if ((d != 2 && d != 3) || P->nx < 1 || P->ny < 1 || (d == 3 && P->nz < 1) || P->k < 0 || P->k >= MAX_K1 ||
      !(P->dt > 0) || !(P->Lx > 0) || !(P->Ly > 0) || (d == 3 && !(P->Lz > 0)) || P->pressure_space != 0) {
    fprintf(stderr, "st_mnorm_noalloc: invalid parameters\n");
    return ST_EINVAL;
  }
  const int K1 = P->k + 1;
  long g2[3], g1[3];
  double hh[3];
  const int nn[3] = {P->nx, P->ny, d == 3 ? P->nz : 1};
  const double Ls[3] = {P->Lx, P->Ly, d == 3 ? P->Lz : 1.0};
  long Nq2 = 1, Nq1 = 1;
  for (int a = 0; a < 3; ++a) {
    const bool act = a < d;
    g2[a] = act ? 2L * nn[a] + 1 : 1;
    g1[a] = act ? (long)nn[a] + 1 : 1;
    hh[a] = act ? Ls[a] / nn[a] : 1.0;
    Nq2 *= g2[a];
    Nq1 *= g1[a];
  }
  const size_t Mv = (size_t)d * Nq2, Nst = (size_t)K1 * (Mv + Nq1);
  if (2048 + 2 * Nst > ST_NOALLOC_DOUBLES) {
    fprintf(stderr,
            "st_mnorm_noalloc: the slab has %zu dofs; the static scratch holds at most %zu "
            "(use st_mnorm with a handle)\n",
            Nst, (ST_NOALLOC_DOUBLES - 2048) / 2);
    return ST_EINVAL;
  }
  if (!r || !out) return ST_EINVAL;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  // set-up: once per device, with that device current
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256) return ST_ECUDA;
  double* scr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) {
        fprintf(stderr, "st_mnorm_noalloc: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
        return ST_ECUDA;
      }
      g_noalloc_ptr[dev] = (double*)ptr;
    }
    scr = g_noalloc_ptr[dev];
  }
  TimeTab T;
  if (!make_time_tables(P->k, T)) return ST_EINVAL;
  RefTables R;
  make_ref_tables(R);
  double tw[MAX_K1];
  for (int i = 0; i < K1; ++i) tw[i] = P->dt * T.w[i];
  double* bs = scr;
  double* part = scr + 8;
  double* res = scr + 1024;
  double* w1 = scr + 2048;
  double* w2 = w1 + Nst;
  e = cudaMemcpyAsync(bs, tw, K1 * sizeof(double), cudaMemcpyHostToDevice, stream);
  // M r by one 1D mass pass per direction; the result ends in w1 (3D) or w2 (2D)
  const double* M = R.M1;
  double* Mr = nullptr;
  for (int partv = 0; partv < 2 && e == cudaSuccess; ++partv) {
    const long* g = partv == 0 ? g2 : g1;
    const long npt = g[0] * g[1] * g[2];
    const int nblk = partv == 0 ? K1 * d : K1;
    const size_t off = partv == 0 ? 0 : (size_t)K1 * Mv;
    const double* src = r + off;
    for (int dir = 0; dir < d && e == cudaSuccess; ++dir) {
      double* dst = ((dir & 1) ? w2 : w1) + off;
      const double* sc = (dir == d - 1) ? bs : nullptr;
      const int cpn = partv == 0 ? d : 1;
      const long total = npt * nblk;
      unsigned grid = (unsigned)((total + BT - 1) / BT);
      if (grid > grid_cap()) grid = (unsigned)grid_cap();
      if (partv == 0)
        mass_pass<double, 2><<<grid, BT, 0, stream>>>(src, dst, g[0], g[1], g[2], dir, hh[dir], nblk, sc, cpn, M[0],
                                                       M[1], M[2], M[4], M[5], M[8]);
      else
        mass_pass<double, 1><<<grid, BT, 0, stream>>>(src, dst, g[0], g[1], g[2], dir, hh[dir], nblk, sc, cpn,
                                                       1.0 / 3.0, 1.0 / 6.0, 0.0, 0.0, 0.0, 0.0);
      e = cudaGetLastError();
      src = dst;
    }
    Mr = (d == 3) ? w1 : w2;
  }
  if (e == cudaSuccess) {
    partial_dot<<<NPART, BT, 0, stream>>>(r, Mr, Nst, part);
    finish_sum<<<1, BT, 0, stream>>>(part, NPART, 1, res);
    e = cudaGetLastError();
  }
  double v = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, res, sizeof(double), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    fprintf(stderr, "st_mnorm_noalloc: %s\n", cudaGetErrorString(e));
    return ST_ECUDA;
  }
  *out = std::sqrt(v > 0.0 ? v : 0.0);
  return ST_OK;
}
