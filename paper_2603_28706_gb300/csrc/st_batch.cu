// Batches of independent slab problems (st_batch_*): the operator calls of all
// instances share one persistent volume launch (work queue over (instance,
// cell batch) items); the Newton steps run concurrently, one host thread and
// one CUDA stream per instance.
#include <cstdio>
#include <string>
#include <thread>
#include <vector>

#include "st_blas.cuh"
#include "st_internal.h"

using namespace st;

struct st_batch {
  std::vector<st_problem*> inst;
  std::vector<cudaStream_t> streams;  // one per instance (its problem runs there)
  std::vector<cudaEvent_t> ev;        // one per instance
  cudaEvent_t ev_main = nullptr;
  cudaStream_t stream = nullptr;      // the caller's stream (batched launches)
  BatchDev bd;
  int dev = 0, dim = 0, K1 = 0;
  std::string last_error;
};

namespace {

st_status batch_error(st_batch* b, st_status s, const std::string& msg) {
  b->last_error = msg;
  return s;
}

st_status batch_cuda(st_batch* b, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return ST_OK;
  return batch_error(b, e == cudaErrorMemoryAllocation ? ST_ENOMEM : ST_ECUDA,
                     std::string(where) + ": " + cudaGetErrorString(e));
}

// the caller's stream waits for every instance stream
cudaError_t join_instances(st_batch* b) {
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < b->inst.size() && e == cudaSuccess; ++i) {
    e = cudaEventRecord(b->ev[i], b->streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev[i], 0);
  }
  return e;
}

// every instance stream waits for the caller's stream
cudaError_t fork_instances(st_batch* b) {
  cudaError_t e = cudaEventRecord(b->ev_main, b->stream);
  for (size_t i = 0; i < b->inst.size() && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(b->streams[i], b->ev_main, 0);
  return e;
}

cudaError_t dispatch(st_batch* b, std::vector<OpArgs>& A, int mode, int prec, int tangent) {
  return b->dim == 2 ? dispatch_op_batch_2d(b->inst.data(), A.data(), (int)A.size(), b->bd, mode, prec, tangent,
                                            b->stream)
                     : dispatch_op_batch_3d(b->inst.data(), A.data(), (int)A.size(), b->bd, mode, prec, tangent,
                                            b->stream);
}

}  // namespace

extern "C" {

st_status st_batch_setup(const st_params* params, int n, void* cuda_stream, st_batch** out) {
  if (!params || !out || n < 1) return ST_EINVAL;
  *out = nullptr;
  for (int i = 1; i < n; ++i)
    if (params[i].dim != params[0].dim || params[i].k != params[0].k) {
      fprintf(stderr, "st_batch_setup: instance %d has another dim or k than instance 0\n", i);
      return ST_EINVAL;
    }
  st_batch* b = new (std::nothrow) st_batch();
  if (!b) return ST_ENOMEM;
  b->stream = (cudaStream_t)cuda_stream;
  b->dim = params[0].dim;
  b->K1 = params[0].k + 1;
  cudaError_t e = cudaGetDevice(&b->dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->bd.nsm, cudaDevAttrMultiProcessorCount, b->dev);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_main, cudaEventDisableTiming);
  st_status s = ST_OK;
  for (int i = 0; i < n && e == cudaSuccess && s == ST_OK; ++i) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    b->streams.push_back(st);
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) break;
    b->ev.push_back(ev);
    st_problem* h = nullptr;
    s = st_setup_mesh(&params[i], (void*)st, &h);
    if (s == ST_OK) b->inst.push_back(h);
  }
  if (e == cudaSuccess && s == ST_OK) e = cudaMalloc(&b->bd.d_desc, (size_t)n * sizeof(OpArgs));
  if (e == cudaSuccess && s == ST_OK) e = cudaMalloc(&b->bd.d_first, (size_t)(n + 1) * sizeof(long));
  if (e == cudaSuccess && s == ST_OK) e = cudaMalloc(&b->bd.d_queue, sizeof(unsigned));
  // the instances' setup work (constant uploads, zeroed buffers) precedes batched launches
  if (e == cudaSuccess && s == ST_OK) e = join_instances(b);
  if (e != cudaSuccess || s != ST_OK) {
    if (e != cudaSuccess) fprintf(stderr, "st_batch_setup: %s\n", cudaGetErrorString(e));
    st_batch_destroy(b);
    return s != ST_OK ? s : (e == cudaErrorMemoryAllocation ? ST_ENOMEM : ST_ECUDA);
  }
  *out = b;
  return ST_OK;
}

st_status st_batch_destroy(st_batch* b) {
  if (!b) return ST_OK;
  for (size_t i = 0; i < b->streams.size(); ++i) cudaStreamSynchronize(b->streams[i]);
  for (st_problem* h : b->inst) st_destroy(h);
  for (cudaEvent_t ev : b->ev) cudaEventDestroy(ev);
  for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
  if (b->ev_main) cudaEventDestroy(b->ev_main);
  cudaFree(b->bd.d_desc);
  cudaFree(b->bd.d_first);
  cudaFree(b->bd.d_queue);
  delete b;
  return ST_OK;
}

size_t st_batch_num_dofs(const st_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->inst.size()) return 0;
  return st_num_dofs(b->inst[i], (int)b->inst[i]->lev.size() - 1);
}

st_status st_batch_linearize(st_batch* b, st_tangent tangent, const void* const* U) {
  if (!b) return ST_EINVAL;
  if (!U) return batch_error(b, ST_EINVAL, "st_batch_linearize: U is required");
  if (tangent < ST_PIC || tangent > ST_MODN) return batch_error(b, ST_EINVAL, "st_batch_linearize: bad tangent");
  const int n = (int)b->inst.size();
  for (int i = 0; i < n; ++i)
    if (!U[i]) return batch_error(b, ST_EINVAL, "st_batch_linearize: U[" + std::to_string(i) + "] is NULL");
  cudaError_t e = join_instances(b);
  std::vector<OpArgs> A(n);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    st_problem* h = b->inst[i];
    const int L = (int)h->lev.size() - 1;
    e = cudaMemcpyAsync(h->d_Ulin, U[i], h->lev[L].Nst * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
    prepare_op_args(h, L, ST_FP64, tangent, U[i], nullptr, nullptr, nullptr, A[i]);
  }
  if (e == cudaSuccess) e = dispatch(b, A, OP_LIN, ST_FP64, tangent);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    st_problem* h = b->inst[i];
    e = cast_f64_f32(h->d_cache64, h->d_cache32, h->cache_len, b->stream);
    if (e == cudaSuccess && h->lev.back().nfaces > 0)
      e = cast_f64_f32(h->d_fcache64, h->d_fcache32, h->fcache_len, b->stream);
    if (e == cudaSuccess) e = cip_linearize(h, (const double*)U[i], b->stream);
    h->lin_tangent = tangent;
    h->lin_valid = true;
    h->precond_valid = false;
  }
  if (e == cudaSuccess) e = fork_instances(b);
  return batch_cuda(b, e, "st_batch_linearize");
}

st_status st_batch_jacobian_apply(st_batch* b, st_tangent tangent, st_prec prec, const void* const* dU,
                                  void* const* out) {
  if (!b) return ST_EINVAL;
  if (!dU || !out) return batch_error(b, ST_EINVAL, "st_batch_jacobian_apply: dU and out are required");
  if (prec != ST_FP64 && prec != ST_FP32) return batch_error(b, ST_EINVAL, "st_batch_jacobian_apply: bad precision");
  const int n = (int)b->inst.size();
  for (int i = 0; i < n; ++i) {
    if (!dU[i] || !out[i])
      return batch_error(b, ST_EINVAL, "st_batch_jacobian_apply: a NULL vector for instance " + std::to_string(i));
    if (!b->inst[i]->lin_valid || b->inst[i]->lin_tangent != tangent)
      return batch_error(b, ST_EINVAL, "st_batch_jacobian_apply: instance " + std::to_string(i) +
                                           " has no linearisation for this tangent (call st_batch_linearize)");
  }
  cudaError_t e = join_instances(b);
  std::vector<OpArgs> A(n);
  for (int i = 0; i < n; ++i) {
    prepare_op_args(b->inst[i], (int)b->inst[i]->lev.size() - 1, prec, tangent, dU[i], out[i], nullptr, nullptr,
                    A[i]);
    set_cip_args(b->inst[i], OP_JAC, prec, A[i]);
  }
  if (e == cudaSuccess) e = dispatch(b, A, OP_JAC, prec, tangent);
  if (e == cudaSuccess) e = fork_instances(b);
  return batch_cuda(b, e, "st_batch_jacobian_apply");
}

st_status st_batch_residual(st_batch* b, st_prec prec, const void* const* U, const void* const* v_prev,
                            const void* const* f, void* const* R) {
  if (!b) return ST_EINVAL;
  if (!U || !v_prev || !R) return batch_error(b, ST_EINVAL, "st_batch_residual: U, v_prev and R are required");
  if (prec != ST_FP64 && prec != ST_FP32) return batch_error(b, ST_EINVAL, "st_batch_residual: bad precision");
  const int n = (int)b->inst.size();
  for (int i = 0; i < n; ++i)
    if (!U[i] || !v_prev[i] || !R[i])
      return batch_error(b, ST_EINVAL, "st_batch_residual: a NULL vector for instance " + std::to_string(i));
  cudaError_t e = join_instances(b);
  std::vector<OpArgs> A(n);
  for (int i = 0; i < n; ++i) {
    prepare_op_args(b->inst[i], (int)b->inst[i]->lev.size() - 1, prec, 0, U[i], R[i], v_prev[i],
                    f ? f[i] : nullptr, A[i]);
    set_cip_args(b->inst[i], OP_RES, prec, A[i]);
  }
  if (e == cudaSuccess) e = dispatch(b, A, OP_RES, prec, 0);
  if (e == cudaSuccess) e = fork_instances(b);
  return batch_cuda(b, e, "st_batch_residual");
}

st_status st_batch_newton_step(st_batch* b, st_tangent tangent, st_prec vcycle_prec, void* const* U,
                               const void* const* v_prev, const void* const* f, st_newton_info* info) {
  if (!b) return ST_EINVAL;
  if (!U || !v_prev) return batch_error(b, ST_EINVAL, "st_batch_newton_step: U and v_prev are required");
  const int n = (int)b->inst.size();
  for (int i = 0; i < n; ++i)
    if (!U[i] || !v_prev[i])
      return batch_error(b, ST_EINVAL, "st_batch_newton_step: a NULL vector for instance " + std::to_string(i));
  cudaError_t e = fork_instances(b);  // the instances see the caller's earlier work
  if (e != cudaSuccess) return batch_cuda(b, e, "st_batch_newton_step");
  std::vector<st_status> res(n, ST_OK);
  std::vector<st_newton_info> loc(n);
  std::vector<std::thread> th;
  th.reserve(n);
  for (int i = 0; i < n; ++i)
    th.emplace_back([&, i]() {
      cudaSetDevice(b->dev);
      res[i] = st_newton_step(b->inst[i], tangent, vcycle_prec, U[i], v_prev[i], f ? f[i] : nullptr,
                              info ? &info[i] : &loc[i]);
    });
  for (auto& t : th) t.join();
  e = join_instances(b);
  if (e != cudaSuccess) return batch_cuda(b, e, "st_batch_newton_step");
  for (int i = 0; i < n; ++i)
    if (res[i] != ST_OK)
      return batch_error(b, res[i], "st_batch_newton_step: instance " + std::to_string(i) + ": " +
                                        st_last_error(b->inst[i]));
  return ST_OK;
}

st_status st_batch_fgmres_solve(st_batch* b, st_prec vcycle_prec, const void* const* rhs, void* const* x,
                                double rtol, int maxit, st_linsolve_info* info) {
  if (!b) return ST_EINVAL;
  if (!rhs || !x) return batch_error(b, ST_EINVAL, "st_batch_fgmres_solve: rhs and x are required");
  const int n = (int)b->inst.size();
  for (int i = 0; i < n; ++i)
    if (!rhs[i] || !x[i])
      return batch_error(b, ST_EINVAL, "st_batch_fgmres_solve: a NULL vector for instance " + std::to_string(i));
  cudaError_t e = fork_instances(b);  // the instances see the caller's earlier work
  if (e != cudaSuccess) return batch_cuda(b, e, "st_batch_fgmres_solve");
  std::vector<st_status> res(n, ST_OK);
  std::vector<st_linsolve_info> loc(n);
  std::vector<std::thread> th;
  th.reserve(n);
  for (int i = 0; i < n; ++i)
    th.emplace_back([&, i]() {
      cudaSetDevice(b->dev);
      res[i] = st_fgmres_solve(b->inst[i], vcycle_prec, rhs[i], x[i], rtol, maxit, info ? &info[i] : &loc[i]);
    });
  for (auto& t : th) t.join();
  e = join_instances(b);
  if (e != cudaSuccess) return batch_cuda(b, e, "st_batch_fgmres_solve");
  for (int i = 0; i < n; ++i)
    if (res[i] != ST_OK)
      return batch_error(b, res[i], "st_batch_fgmres_solve: instance " + std::to_string(i) + ": " +
                                        st_last_error(b->inst[i]));
  return ST_OK;
}

const char* st_batch_last_error(const st_batch* b) {
  if (!b) return "null batch";
  return b->last_error.c_str();
}

}  // extern "C"
