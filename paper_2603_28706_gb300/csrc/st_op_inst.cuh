// Launch helpers for the operator kernels of one dimension.
#pragma once

#include <vector>

#include "st_cip.cuh"
#include "st_face.cuh"
#include "st_operator.cuh"
#include "st_tune.h"

namespace st {

// occupancy of a kernel (computed once per instantiation, thread-safe)
template <typename K>
int occupancy_once(K kern, int threads, size_t smem) {
  int occ = 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess) return 0;
  return occ < 1 ? 1 : occ;
}

// all boundary faces of one problem, one launch, writing the face scratch
// (or, when linearising, the face caches)
template <int DIM, int K1, typename T, int MODE, int TAN>
cudaError_t launch_faces_t(const st_problem* h, const Level& L, const OpArgs& a, cudaStream_t st, long fcap = 0) {
  using FCfg = FaceCfg<DIM, T>;
  auto fkern = st_face_kernel<DIM, K1, T, MODE, TAN>;
  static const int focc = occupancy_once(fkern, OP_THREADS, FCfg::smem_bytes);
  if (focc == 0) return cudaErrorInvalidConfiguration;
  const long nslots = L.nfaces * K1;
  if (nslots == 0) return cudaSuccess;
  long fgrid = (nslots + FCfg::FS - 1) / FCfg::FS;
  if (fcap <= 0) fcap = 8L * h->nsm;
  if (fgrid > fcap) fgrid = fcap;
  fkern<<<(unsigned)fgrid, OP_THREADS, FCfg::smem_bytes, st>>>(a, L.d_face_cell, L.d_face_side, nslots,
                                                                reinterpret_cast<T*>(h->d_fscr));
  return cudaGetLastError();
}

// out = sum of the class buffers (streaming), then += the face
// contributions of the boundary-cell layer
template <int DIM, int K1, typename T>
cudaError_t launch_node_sum_t(const st_problem* h, const Level& L, const OpArgs& a, cudaStream_t st) {
  long g = (L.Nst / 2 + 255) / 256;
  if (g > 16L * h->nsm) g = 16L * h->nsm;
  if (g < 1) g = 1;
  st_cbuf_sum<DIM, T><<<(unsigned)g, 256, 0, st>>>(reinterpret_cast<const T*>(a.cbuf), a.cbuf_stride, L.Nst,
                                                    reinterpret_cast<T*>(a.out));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || L.n_gather == 0) return e;
  const long items = (long)L.n_gather_vel * K1 * DIM + (long)(L.n_gather - L.n_gather_vel) * K1;
  long gf = (items + 255) / 256;
  if (gf > 16L * h->nsm) gf = 16L * h->nsm;
  st_face_add<DIM, K1, T><<<(unsigned)gf, 256, 0, st>>>(a, L.n_gather_vel, L.n_gather, L.d_gnode, L.d_gptr,
                                                        reinterpret_cast<const GatherEnt*>(L.d_gent),
                                                        reinterpret_cast<const T*>(h->d_fscr),
                                                        reinterpret_cast<T*>(a.out));
  return cudaGetLastError();
}

// CIP face terms added into the class buffers (after the volume kernel, before
// the node sum); the residual first fills its weights from its argument
template <int DIM, int K1, typename T, int MODE>
cudaError_t launch_cip_t(const st_problem* h, const Level& L, const OpArgs& a, cudaStream_t st) {
  if (MODE != OP_JAC && MODE != OP_RES) return cudaSuccess;
  if (!a.cipw || L.ncells == 0) return cudaSuccess;
  T* w = reinterpret_cast<T*>(a.cipw);
  if (MODE == OP_RES) {
    long g = ((long)DIM * L.ncells * K1 + 255) / 256;
    if (g > 16L * h->nsm) g = 16L * h->nsm;
    st_cip_weights<DIM, K1, T><<<(unsigned)g, 256, 0, st>>>(a, reinterpret_cast<const T*>(a.in), w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  long g = ((long)DIM * L.ncells * K1 + 127) / 128;
  if (g > 16L * h->nsm) g = 16L * h->nsm;
  T* fb = reinterpret_cast<T*>(h->d_cipf);
  st_cip_face<DIM, K1, T><<<(unsigned)g, 128, 0, st>>>(a, w, fb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  st_cip_apply<DIM, K1, T><<<(unsigned)g, 128, 0, st>>>(a, fb, MODE == OP_RES ? (T)-1 : (T)1);
  return cudaGetLastError();
}

template <int DIM>
cudaError_t dispatch_cip_weights_dim(const st_problem* h, const OpArgs& a, const double* U, double* w,
                                     cudaStream_t st) {
  const Level& L = h->lev.back();
  long g = ((long)DIM * L.ncells * h->K1 + 255) / 256;
  if (g > 16L * h->nsm) g = 16L * h->nsm;
  if (g < 1) return cudaSuccess;
  switch (h->K1) {
    case 1: st_cip_weights<DIM, 1, double><<<(unsigned)g, 256, 0, st>>>(a, U, w); break;
    case 2: st_cip_weights<DIM, 2, double><<<(unsigned)g, 256, 0, st>>>(a, U, w); break;
    case 3: st_cip_weights<DIM, 3, double><<<(unsigned)g, 256, 0, st>>>(a, U, w); break;
    case 4: st_cip_weights<DIM, 4, double><<<(unsigned)g, 256, 0, st>>>(a, U, w); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// the volume kernel's view of the whole finest level
template <typename T>
void set_volume_args(const st_problem* h, const Level& L, OpArgs& a) {
  a.col_start = 0;
  a.ncol = L.ncells;
  a.cbuf = sizeof(T) == 8 ? h->d_cbuf64 : h->d_cbuf32;
  a.cbuf_stride = L.Nst;
}

template <int DIM, int K1, typename T, int MODE, int TAN>
cudaError_t launch_op_t(const st_problem* h, const Level& L, OpArgs& a) {
  using Cfg = OpCfg<DIM, K1, T>;
  auto kern = st_op_kernel<DIM, K1, T, MODE, TAN>;
  static const int occ = occupancy_once(kern, Cfg::NT, Cfg::smem_bytes);
  if (occ == 0) return cudaErrorInvalidConfiguration;
  // The volume kernel (one launch over all cells in colour order) writes
  // every cell's contributions into the private buffer of its colour class
  // with plain stores.  The face kernel (all boundary faces, one launch) runs
  // on an internal stream that depends only on the work before the volume
  // kernel; its small CTAs fit into the shared memory and registers the
  // volume kernel's CTAs leave free on every SM, so the two can run side by
  // side.  It writes only the face scratch (or, when linearising, the face
  // cache).  The caller's stream then waits for the face kernel;
  // st_cbuf_sum and st_face_add form out = sum of the class buffers + face
  // contributions.
  set_volume_args<T>(h, L, a);
  const std::string tag = std::to_string(DIM) + "," + std::to_string(K1) + "," +
                          (sizeof(T) == 8 ? "double" : "float") + ",OP_JAC," + std::to_string(TAN) +
                          "> cells=" + std::to_string(L.ncells);
  // Default: every resident CTA slot gets an equal share of the cells when
  // there are at least half a batch per slot; smaller meshes use full
  // batches.  The Jacobian action (the hot call) autotunes the number of
  // cells per CTA: the balanced share of one, two or four CTA waves, or one
  // batch of C cells per CTA (each CTA always runs batches of C cells).
  const long cap = (long)occ * h->nsm;
  const long full = (L.ncells + Cfg::C - 1) / Cfg::C;
  long grid = full;
  if (L.ncells >= cap * (Cfg::C / 2)) grid = cap;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  if (MODE == OP_JAC) {
    long cand[4] = {grid, 2 * cap, 4 * cap, full};
    for (long& c : cand) c = c < 1 ? 1 : (c > full ? full : c);
    const int pick = tune_pick(
        "st_op_kernel<" + tag, 4,
        [&](int i) {
          kern<<<(unsigned)cand[i], Cfg::NT, Cfg::smem_bytes, h->stream>>>(a);
          return cudaGetLastError();
        },
        [&](int i) { return "cells/CTA=" + std::to_string((L.ncells + cand[i] - 1) / cand[i]); }, h->stream);
    grid = cand[pick];
  }
  // The whole sequence: the volume kernel, then the face kernel in the space
  // it leaves.  Tuned over the whole apply: the volume grid chosen alone, or
  // the balanced one-wave grid, whose CTAs all start at once and so leave
  // the scheduler free to place face CTAs beside them.
  auto sequence = [&](long vgrid) -> cudaError_t {
    cudaError_t e = cudaEventRecord(h->ev_fork, h->stream);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)vgrid, Cfg::NT, Cfg::smem_bytes, h->stream>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->s_face, h->ev_fork, 0);
    if (e == cudaSuccess) e = launch_faces_t<DIM, K1, T, MODE, TAN>(h, L, a, h->s_face);
    if (e == cudaSuccess) e = launch_cip_t<DIM, K1, T, MODE>(h, L, a, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->s_face);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_join, 0);
    if (e == cudaSuccess && MODE != OP_LIN) e = launch_node_sum_t<DIM, K1, T>(h, L, a, h->stream);
    return e;
  };
  if (MODE == OP_JAC) {
    const long vg[2] = {grid, cap < full ? cap : full};
    const int pick = tune_pick(
        "jacobian apply<" + tag, vg[0] == vg[1] ? 1 : 2, [&](int i) { return sequence(vg[i]); },
        [&](int i) { return "volume cells/CTA=" + std::to_string((L.ncells + vg[i] - 1) / vg[i]) + ", faces beside"; },
        h->stream);
    grid = vg[pick];
  }
  return sequence(grid);
}

// Several problems (same dim and k) in one persistent volume launch over the
// (instance, cell batch) items; faces and node sums per instance on `st`.
// A[i]: argument block of instance i (fill_op_args + data pointers).
template <int DIM, int K1, typename T, int MODE, int TAN>
cudaError_t launch_op_batch_t(st_problem* const* P, OpArgs* A, int n, BatchDev& bd, cudaStream_t st) {
  using Cfg = OpCfg<DIM, K1, T>;
  auto kern = st_op_kernel_batch<DIM, K1, T, MODE, TAN>;
  static const int occ = occupancy_once(kern, Cfg::NT, Cfg::smem_bytes);
  if (occ == 0) return cudaErrorInvalidConfiguration;
  std::vector<long> first(n + 1, 0);
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const Level& L = P[i]->lev.back();
    set_volume_args<T>(P[i], L, A[i]);
    first[i + 1] = first[i] + (L.ncells + Cfg::C - 1) / Cfg::C;
    e = launch_faces_t<DIM, K1, T, MODE, TAN>(P[i], L, A[i], st);
  }
  if (e != cudaSuccess) return e;
  // pageable host sources: the copies are staged before they return
  e = cudaMemcpyAsync(bd.d_desc, A, (size_t)n * sizeof(OpArgs), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bd.d_first, first.data(), (size_t)(n + 1) * sizeof(long), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bd.d_queue, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const long cap = (long)occ * bd.nsm;
  const long grid = first[n] < cap ? (first[n] > 0 ? first[n] : 1) : cap;
  kern<<<(unsigned)grid, Cfg::NT, Cfg::smem_bytes, st>>>(bd.d_desc, bd.d_first, n, bd.d_queue);
  e = cudaGetLastError();
  for (int i = 0; i < n && e == cudaSuccess && MODE != OP_LIN; ++i) {
    e = launch_cip_t<DIM, K1, T, MODE>(P[i], P[i]->lev.back(), A[i], st);
    if (e == cudaSuccess) e = launch_node_sum_t<DIM, K1, T>(P[i], P[i]->lev.back(), A[i], st);
  }
  return e;
}

template <int DIM, int K1>
cudaError_t dispatch_op_batch_k(st_problem* const* P, OpArgs* A, int n, BatchDev& bd, int mode, int prec,
                                int tangent, cudaStream_t st) {
  if (mode == OP_LIN) return launch_op_batch_t<DIM, K1, double, OP_LIN, 0>(P, A, n, bd, st);
  const bool r1 = tangent != ST_PIC;
  if (mode == OP_JAC) {
    if (prec == ST_FP64)
      return r1 ? launch_op_batch_t<DIM, K1, double, OP_JAC, 1>(P, A, n, bd, st)
                : launch_op_batch_t<DIM, K1, double, OP_JAC, 0>(P, A, n, bd, st);
    return r1 ? launch_op_batch_t<DIM, K1, float, OP_JAC, 1>(P, A, n, bd, st)
              : launch_op_batch_t<DIM, K1, float, OP_JAC, 0>(P, A, n, bd, st);
  }
  if (prec == ST_FP64) return launch_op_batch_t<DIM, K1, double, OP_RES, 0>(P, A, n, bd, st);
  return launch_op_batch_t<DIM, K1, float, OP_RES, 0>(P, A, n, bd, st);
}

template <int DIM>
cudaError_t dispatch_op_batch_dim(st_problem* const* P, OpArgs* A, int n, BatchDev& bd, int mode, int prec,
                                  int tangent, cudaStream_t st) {
  switch (P[0]->K1) {
    case 1: return dispatch_op_batch_k<DIM, 1>(P, A, n, bd, mode, prec, tangent, st);
    case 2: return dispatch_op_batch_k<DIM, 2>(P, A, n, bd, mode, prec, tangent, st);
    case 3: return dispatch_op_batch_k<DIM, 3>(P, A, n, bd, mode, prec, tangent, st);
    case 4: return dispatch_op_batch_k<DIM, 4>(P, A, n, bd, mode, prec, tangent, st);
  }
  return cudaErrorInvalidValue;
}

template <int DIM, int K1>
cudaError_t dispatch_op_k(const st_problem* h, const Level& L, OpArgs& a, int mode, int prec, int tangent) {
  if (mode == OP_LIN) return launch_op_t<DIM, K1, double, OP_LIN, 0>(h, L, a);
  const bool r1 = tangent != ST_PIC;
  if (mode == OP_JAC) {
    if (prec == ST_FP64)
      return r1 ? launch_op_t<DIM, K1, double, OP_JAC, 1>(h, L, a) : launch_op_t<DIM, K1, double, OP_JAC, 0>(h, L, a);
    return r1 ? launch_op_t<DIM, K1, float, OP_JAC, 1>(h, L, a) : launch_op_t<DIM, K1, float, OP_JAC, 0>(h, L, a);
  }
  if (prec == ST_FP64) return launch_op_t<DIM, K1, double, OP_RES, 0>(h, L, a);
  return launch_op_t<DIM, K1, float, OP_RES, 0>(h, L, a);
}

template <int DIM>
cudaError_t dispatch_op_dim(const st_problem* h, const Level& L, OpArgs& a, int mode, int prec, int tangent) {
  switch (h->K1) {
    case 1: return dispatch_op_k<DIM, 1>(h, L, a, mode, prec, tangent);
    case 2: return dispatch_op_k<DIM, 2>(h, L, a, mode, prec, tangent);
    case 3: return dispatch_op_k<DIM, 3>(h, L, a, mode, prec, tangent);
    case 4: return dispatch_op_k<DIM, 4>(h, L, a, mode, prec, tangent);
  }
  return cudaErrorInvalidValue;
}


// Spatial element matrices (times tau w_mu) of every cell at node mu from the
// coefficient caches in a.cache / a.fcache: volume part by probing the
// sum-factorised element operator with unit vectors (one column per slot),
// boundary-face part added by st_face_matrix.  E: [ncells][K1][NE][NE].
template <int DIM, int K1, typename T, int TAN>
cudaError_t launch_elm_t(const st_problem* h, const Level& L, OpArgs a, T* E, const int* bcells, int nbc) {
  using Cfg = OpCfg<DIM, K1, T>;
  using FCfg = FaceCfg<DIM, T>;
  auto kern = st_op_kernel<DIM, K1, T, OP_ELM, TAN>;
  auto fkern = st_face_matrix<DIM, K1, T, TAN>;
  constexpr int NE = Dims<DIM>::NE;
  const size_t fsm = (size_t)NE * FCfg::per_slot * sizeof(T) + 64;
  static const int occ = occupancy_once(kern, Cfg::NT, Cfg::smem_bytes);
  static const int focc = occupancy_once(fkern, OP_THREADS, fsm);
  if (occ == 0 || focc == 0) return cudaErrorInvalidConfiguration;
  a.out = E;
  a.ncol = L.ncells * NE;
  a.col_start = 0;
  long grid = (a.ncol + Cfg::S - 1) / Cfg::S;
  if (grid > (long)occ * h->nsm) grid = (long)occ * h->nsm;
  kern<<<(unsigned)grid, Cfg::NT, Cfg::smem_bytes, h->stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || nbc == 0) return e;
  long fg = nbc < 4L * h->nsm ? nbc : 4L * h->nsm;
  fkern<<<(unsigned)fg, OP_THREADS, fsm, h->stream>>>(a, bcells, nbc, E);
  return cudaGetLastError();
}

template <int DIM>
cudaError_t dispatch_elm_dim(const st_problem* h, const Level& L, const OpArgs& a, int prec, int tangent, void* E,
                             const int* bcells, int nbc) {
  const bool r1 = tangent != ST_PIC;
#define ST_ELM_CASE(K)                                                                                            \
  case K:                                                                                                         \
    if (prec == ST_FP64)                                                                                          \
      return r1 ? launch_elm_t<DIM, K, double, 1>(h, L, a, (double*)E, bcells, nbc)                                \
                : launch_elm_t<DIM, K, double, 0>(h, L, a, (double*)E, bcells, nbc);                               \
    return r1 ? launch_elm_t<DIM, K, float, 1>(h, L, a, (float*)E, bcells, nbc)                                    \
              : launch_elm_t<DIM, K, float, 0>(h, L, a, (float*)E, bcells, nbc);
  switch (h->K1) {
    ST_ELM_CASE(1)
    ST_ELM_CASE(2)
    ST_ELM_CASE(3)
    ST_ELM_CASE(4)
  }
#undef ST_ELM_CASE
  return cudaErrorInvalidValue;
}

}  // namespace st
