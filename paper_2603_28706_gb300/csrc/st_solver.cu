// Outer solvers (Sec. 6.1-6.3): right-preconditioned FGMRES in the block
// mass inner product and the globalised Newton-type step on one slab.
//
// FGMRES: Arnoldi with classical Gram-Schmidt applied twice, all vector work
// in FP64 on the device (mass operator, multi-dots, multi-axpys); the small
// Hessenberg least-squares problem (Givens rotations) on the host.  The
// preconditioner is one V-cycle in FP32 (mixed) or FP64.
// Newton: R = R_n(U); stop by eq. nk-stop; linearise; rebuild the finest-level
// surrogate patches only by the refresh rule of Sec. 6.3 (coarse operators and
// the matrix-free operator always follow the iterate; a solve with kept
// patches that passes twice the preceding solve's iteration count is stopped,
// the patches are rebuilt and the solve restarts); solve J dU = R to the
// Eisenstat-Walker forcing (choice 2; Picard: lin_rtol); Armijo backtracking
// on phi = 1/2 |R|_M^2 (exN, modN; Picard takes lambda = 1); U += lambda dU.
#include <cmath>
#include <cstring>
#include <vector>

#include "st_blas.cuh"
#include "st_internal.h"

namespace st {

namespace {

struct KrylovWs {
  int m = 0;
  size_t n = 0;
  double* V = nullptr;   // (m+1) x n
  double* Z = nullptr;   // m x n
  double* w = nullptr;
  double* Mw = nullptr;
  double* mwork = nullptr;  // 2n, mass operator work
  double* x = nullptr;
  double* r = nullptr;
  double* R = nullptr;
  double* Ut = nullptr;
  double* Rt = nullptr;
  double* dU = nullptr;
  float* r32 = nullptr;
  float* d32 = nullptr;
  double* vr64 = nullptr;   // FP64 V-cycle input / output (fixed buffers)
  double* vd64 = nullptr;
  double* dots = nullptr;   // 2(m+1) + 2
  double* part = nullptr;   // 128 (m+1)
  double* coef = nullptr;   // m + 1
};

void free_ws(KrylovWs* k) {
  cudaFree(k->V);
  cudaFree(k->Z);
  cudaFree(k->w);
  cudaFree(k->Mw);
  cudaFree(k->mwork);
  cudaFree(k->x);
  cudaFree(k->r);
  cudaFree(k->R);
  cudaFree(k->Ut);
  cudaFree(k->Rt);
  cudaFree(k->dU);
  cudaFree(k->r32);
  cudaFree(k->vr64);
  cudaFree(k->vd64);
  cudaFree(k->d32);
  cudaFree(k->dots);
  cudaFree(k->part);
  cudaFree(k->coef);
  *k = KrylovWs();
}

cudaError_t get_ws(st_problem* h, KrylovWs*& k) {
  const size_t n = h->lev.back().Nst;
  const int m = h->P.fgmres_restart > 0 ? h->P.fgmres_restart : 50;
  if (!h->kry) h->kry = new KrylovWs();
  k = (KrylovWs*)h->kry;
  if (k->n == n && k->m == m) return cudaSuccess;
  free_ws(k);
  cudaError_t e = cudaMalloc(&k->V, (size_t)(m + 1) * n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&k->Z, (size_t)m * n * sizeof(double));
  double** v1[] = {&k->w, &k->Mw, &k->x, &k->r, &k->R, &k->Ut, &k->Rt, &k->dU};
  for (double** p : v1)
    if (e == cudaSuccess) e = cudaMalloc(p, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&k->mwork, 2 * n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&k->r32, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&k->vr64, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&k->vd64, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&k->d32, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&k->dots, (2 * (m + 1) + 2) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&k->part, 128 * (size_t)(m + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&k->coef, (m + 1) * sizeof(double));
  if (e != cudaSuccess) {
    free_ws(k);
    return e;
  }
  k->n = n;
  k->m = m;
  return cudaSuccess;
}

// |v|_M on the finest level (synchronises)
cudaError_t mnorm(st_problem* h, KrylovWs* k, const double* v, double& out) {
  const int L = (int)h->lev.size() - 1;
  cudaError_t e = mass_apply<double>(h, L, v, k->Mw, k->mwork);
  if (e == cudaSuccess) e = dot_f64(v, k->Mw, k->n, k->dots, k->part, h->stream);
  double v2 = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v2, k->dots, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  out = std::sqrt(v2 > 0.0 ? v2 : 0.0);
  return e;
}

cudaError_t japply(st_problem* h, const double* x, double* y) {
  const int L = (int)h->lev.size() - 1;
  return launch_op(h, L, OP_JAC, ST_FP64, h->lin_tangent, x, y, nullptr, nullptr);
}

st_status precond(st_problem* h, KrylovWs* k, st_prec prec, const double* v, double* z) {
  // the V-cycle runs on fixed buffers (so that its captured graph is reused)
  if (prec == ST_FP64) {
    cudaError_t e = cudaMemcpyAsync(k->vr64, v, k->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "fgmres copy");
    st_status s = mg_vcycle(h, ST_FP64, k->vr64, k->vd64);
    if (s != ST_OK) return s;
    return cuda_check(h, cudaMemcpyAsync(z, k->vd64, k->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream),
                      "fgmres copy");
  }
  cudaError_t e = cast_f64_f32(v, k->r32, k->n, h->stream);
  if (e != cudaSuccess) return cuda_check(h, e, "fgmres cast");
  st_status s = mg_vcycle(h, ST_FP32, k->r32, k->d32);
  if (s != ST_OK) return s;
  return cuda_check(h, cast_f32_f64(k->d32, z, k->n, h->stream), "fgmres cast");
}

// Solve J x = b to |b - J x|_M <= rtol |b|_M; x written to k->x.
st_status fgmres(st_problem* h, KrylovWs* k, st_prec prec, const double* b, double rtol, int maxit, int& its,
                 double& res_out, double& bnorm_out) {
  const size_t n = k->n;
  const int mmax = k->m;
  cudaStream_t s = h->stream;
  cudaError_t e = cudaMemsetAsync(k->x, 0, n * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(k->r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  double beta = 0.0;
  if (e == cudaSuccess) e = mnorm(h, k, k->r, beta);
  if (e != cudaSuccess) return cuda_check(h, e, "fgmres");
  bnorm_out = beta;
  const double target = rtol * beta;
  its = 0;
  std::vector<double> H((size_t)(mmax + 1) * mmax), g(mmax + 1), cs(mmax), sn(mmax), y(mmax);
  std::vector<double> h1(mmax + 1), h2(mmax + 1);
  while (its < maxit && beta > target) {
    const int m = std::min(mmax, maxit - its);
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    e = axpby_f64(1.0 / beta, k->r, 0.0, k->V, n, s);
    if (e != cudaSuccess) return cuda_check(h, e, "fgmres");
    int used = 0;
    for (int j = 0; j < m; ++j) {
      double* Vj = k->V + (size_t)j * n;
      double* Zj = k->Z + (size_t)j * n;
      st_status st = precond(h, k, prec, Vj, Zj);
      if (st != ST_OK) return st;
      e = japply(h, Zj, k->w);
      // classical Gram-Schmidt, twice, in the M-inner product
      for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
        e = mass_apply<double>(h, (int)h->lev.size() - 1, k->w, k->Mw, k->mwork);
        if (e == cudaSuccess) e = multidot_f64(k->V, n, j + 1, k->Mw, n, k->dots + pass * (mmax + 1), k->part, s);
        if (e == cudaSuccess) e = multiaxpy_f64(k->V, n, j + 1, k->dots + pass * (mmax + 1), k->w, n, s);
      }
      if (e == cudaSuccess) e = mass_apply<double>(h, (int)h->lev.size() - 1, k->w, k->Mw, k->mwork);
      if (e == cudaSuccess) e = dot_f64(k->w, k->Mw, n, k->dots + 2 * (mmax + 1), k->part, s);
      double hn2 = 0.0;
      if (e == cudaSuccess) e = cudaMemcpyAsync(h1.data(), k->dots, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h2.data(), k->dots + (mmax + 1), (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(&hn2, k->dots + 2 * (mmax + 1), sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_check(h, e, "fgmres arnoldi");
      const double hn = std::sqrt(hn2 > 0.0 ? hn2 : 0.0);
      for (int i = 0; i <= j; ++i) H[(size_t)i * mmax + j] = h1[i] + h2[i];
      H[(size_t)(j + 1) * mmax + j] = hn;
      if (hn > 0.0) {
        e = axpby_f64(1.0 / hn, k->w, 0.0, k->V + (size_t)(j + 1) * n, n, s);
        if (e != cudaSuccess) return cuda_check(h, e, "fgmres");
      }
      // Givens rotations on column j
      for (int i = 0; i < j; ++i) {
        const double a = H[(size_t)i * mmax + j], bb = H[(size_t)(i + 1) * mmax + j];
        H[(size_t)i * mmax + j] = cs[i] * a + sn[i] * bb;
        H[(size_t)(i + 1) * mmax + j] = -sn[i] * a + cs[i] * bb;
      }
      const double a = H[(size_t)j * mmax + j], bb = H[(size_t)(j + 1) * mmax + j];
      const double rr = std::hypot(a, bb);
      cs[j] = rr > 0 ? a / rr : 1.0;
      sn[j] = rr > 0 ? bb / rr : 0.0;
      H[(size_t)j * mmax + j] = rr;
      H[(size_t)(j + 1) * mmax + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      used = j + 1;
      if (std::fabs(g[j + 1]) <= target || hn == 0.0) break;
    }
    // back substitution H(0:used,0:used) y = g
    for (int i = used - 1; i >= 0; --i) {
      double acc = g[i];
      for (int l = i + 1; l < used; ++l) acc -= H[(size_t)i * mmax + l] * y[l];
      y[i] = acc / H[(size_t)i * mmax + i];
    }
    // x += Z y; r = b - J x
    e = cudaMemcpyAsync(k->coef, y.data(), used * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = lincomb_f64(k->Z, n, used, k->coef, k->w, n, s);
    if (e == cudaSuccess) e = axpby_f64(1.0, k->w, 1.0, k->x, n, s);
    if (e == cudaSuccess) e = japply(h, k->x, k->w);
    if (e == cudaSuccess) e = cudaMemcpyAsync(k->r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = axpby_f64(-1.0, k->w, 1.0, k->r, n, s);
    if (e == cudaSuccess) e = mnorm(h, k, k->r, beta);
    if (e != cudaSuccess) return cuda_check(h, e, "fgmres update");
  }
  res_out = beta;
  return ST_OK;
}

}  // namespace

void krylov_destroy(st_problem* h) {
  if (h && h->kry) {
    KrylovWs* k = (KrylovWs*)h->kry;
    free_ws(k);
    delete k;
    h->kry = nullptr;
  }
}

}  // namespace st

using namespace st;

extern "C" st_status st_fgmres_solve(st_problem* h, st_prec vcycle_prec, const void* b, void* x, double rtol,
                                     int maxit, st_linsolve_info* info) {
  if (!h) return ST_EINVAL;
  if (!b || !x) return set_error(h, ST_EINVAL, "st_fgmres_solve: b and x are required");
  if (vcycle_prec != ST_FP64 && vcycle_prec != ST_FP32) return set_error(h, ST_EINVAL, "st_fgmres_solve: bad precision");
  if (!(rtol > 0.0) || maxit < 1) return set_error(h, ST_EINVAL, "st_fgmres_solve: need rtol > 0 and maxit >= 1");
  if (!h->lin_valid) return set_error(h, ST_EINVAL, "st_fgmres_solve: no linearisation (call st_linearize)");
  KrylovWs* k = nullptr;
  cudaError_t e = get_ws(h, k);
  if (e != cudaSuccess) return cuda_check(h, e, "st_fgmres_solve workspace");
  if (!h->precond_valid || h->precond_prec != vcycle_prec) {
    st_status s = mg_setup(h, vcycle_prec, true);
    if (s != ST_OK) return s;
  }
  int its = 0;
  double lres = 0.0, bn = 0.0;
  st_status st = fgmres(h, k, vcycle_prec, (const double*)b, rtol, maxit, its, lres, bn);
  if (st != ST_OK) return st;
  e = cudaMemcpyAsync(x, k->x, k->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_check(h, e, "st_fgmres_solve");
  if (info) {
    info->iters = its;
    info->res_norm = lres;
    info->rhs_norm = bn;
  }
  if (lres > rtol * bn * (1.0 + 1e-12))
    return set_error(h, ST_NOT_CONVERGED, "st_fgmres_solve: maxit reached before the tolerance");
  return ST_OK;
}

extern "C" st_status st_newton_step(st_problem* h, st_tangent tangent, st_prec vcycle_prec, void* U,
                                    const void* v_prev, const void* f, st_newton_info* info) {
  if (!h) return ST_EINVAL;
  if (!U || !v_prev) return set_error(h, ST_EINVAL, "st_newton_step: U and v_prev are required");
  if (tangent < ST_PIC || tangent > ST_MODN) return set_error(h, ST_EINVAL, "st_newton_step: bad tangent");
  if (vcycle_prec != ST_FP64 && vcycle_prec != ST_FP32) return set_error(h, ST_EINVAL, "st_newton_step: bad precision");
  st_newton_info inf;
  memset(&inf, 0, sizeof(inf));
  KrylovWs* k = nullptr;
  cudaError_t e = get_ws(h, k);
  if (e != cudaSuccess) return cuda_check(h, e, "st_newton_step workspace");
  const st_params& P = h->P;
  double* Ud = (double*)U;
  const size_t n = k->n;
  cudaStream_t s = h->stream;
  st_status st = st_residual(h, ST_FP64, Ud, v_prev, f, k->R);
  if (st != ST_OK) return st;
  double rn = 0.0;
  e = mnorm(h, k, k->R, rn);
  if (e != cudaSuccess) return cuda_check(h, e, "st_newton_step");
  const double r0 = rn;
  inf.res_norm_initial = r0;
  double prev_r = -1.0, eta = P.ew_max;
  double prev_ratio = -1.0;
  int lin_prev = -1, lin_last = -1;
  bool first = true;
  st_status result = ST_NOT_CONVERGED;
  for (int m = 0; m < P.newton_maxit; ++m) {
    if (!(rn == rn)) {
      result = ST_NOT_CONVERGED;
      set_error(h, ST_NOT_CONVERGED, "st_newton_step: residual is not a number");
      break;
    }
    if (rn <= P.tol_abs || rn <= P.tol_rel * r0) {
      result = ST_OK;
      break;
    }
    st = st_linearize(h, tangent, Ud);
    if (st != ST_OK) return st;
    const bool rebuild = first || (prev_ratio > P.rho_refresh) || (lin_prev >= 0 && lin_last > 2 * lin_prev);
    h->precond_valid = !first;  // keep the surrogate factorisations unless rebuilt
    st = mg_setup(h, vcycle_prec, rebuild);
    if (st != ST_OK) return st;
    inf.patch_rebuilds += rebuild ? 1 : 0;
    first = false;
    double forcing;
    if (tangent == ST_PIC) {
      forcing = P.lin_rtol;
    } else {
      if (m > 0 && prev_r > 0.0) {
        double e_new = P.ew_gamma * std::pow(rn / prev_r, P.ew_alpha);
        const double safeguard = P.ew_gamma * std::pow(eta, P.ew_alpha);
        if (safeguard > 0.1) e_new = std::max(e_new, safeguard);
        eta = std::min(P.ew_max, e_new);
      }
      forcing = eta;
    }
    int its = 0;
    double lres = 0.0, bn = 0.0;
    // refresh rule, second trigger, applied during the solve: with kept
    // surrogate patches a solve that needs more than twice the preceding
    // solve's iterations has deteriorated; rebuild them and restart the solve
    const int cap = (rebuild || lin_last < 0) ? P.fgmres_maxit : std::min(P.fgmres_maxit, 2 * lin_last);
    st = fgmres(h, k, vcycle_prec, k->R, forcing, cap, its, lres, bn);
    if (st != ST_OK) return st;
    if (lres > forcing * bn * (1.0 + 1e-12) && cap < P.fgmres_maxit) {
      inf.fgmres_iters_total += its;
      st = mg_setup(h, vcycle_prec, true);
      if (st != ST_OK) return st;
      inf.patch_rebuilds += 1;
      st = fgmres(h, k, vcycle_prec, k->R, forcing, P.fgmres_maxit, its, lres, bn);
      if (st != ST_OK) return st;
    }
    inf.fgmres_iters_total += its;
    inf.fgmres_iters_last = its;
    lin_prev = lin_last;
    lin_last = its;
    if (lres > forcing * bn * (1.0 + 1e-12)) {
      result = ST_NOT_CONVERGED;
      set_error(h, ST_NOT_CONVERGED, "st_newton_step: FGMRES missed the forcing tolerance");
      inf.newton_iters = m;
      break;
    }
    e = cudaMemcpyAsync(k->dU, k->x, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_check(h, e, "st_newton_step");
    double lam = 1.0, rt = 0.0;
    bool accepted = false;
    while (true) {
      e = cudaMemcpyAsync(k->Ut, Ud, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = axpby_f64(lam, k->dU, 1.0, k->Ut, n, s);
      if (e != cudaSuccess) return cuda_check(h, e, "st_newton_step");
      st = st_residual(h, ST_FP64, k->Ut, v_prev, f, k->Rt);
      if (st != ST_OK) return st;
      e = mnorm(h, k, k->Rt, rt);
      if (e != cudaSuccess) return cuda_check(h, e, "st_newton_step");
      if (tangent == ST_PIC || rt * rt <= (1.0 - 2.0 * P.armijo_c * lam) * rn * rn) {
        accepted = true;
        break;
      }
      lam *= 0.5;
      if (lam < P.lambda_min) break;
    }
    if (!accepted) {
      result = ST_LINESEARCH_FAILED;
      set_error(h, ST_LINESEARCH_FAILED, "st_newton_step: Armijo backtracking reached lambda_min");
      inf.newton_iters = m;
      break;
    }
    e = cudaMemcpyAsync(Ud, k->Ut, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(k->R, k->Rt, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_check(h, e, "st_newton_step");
    prev_ratio = rt / rn;
    prev_r = rn;
    rn = rt;
    inf.lambda_last = lam;
    inf.newton_iters = m + 1;
    if (m + 1 == P.newton_maxit && (rn <= P.tol_abs || rn <= P.tol_rel * r0)) result = ST_OK;
  }
  if (result == ST_NOT_CONVERGED && h->last_error.empty())
    set_error(h, ST_NOT_CONVERGED, "st_newton_step: newton_maxit reached");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_check(h, e, "st_newton_step");
  inf.res_norm_final = rn;
  inf.status = result;
  if (info) *info = inf;
  return result;
}
