// Launch helpers for the operator kernels of one dimension.
#pragma once

#include "st_operator.cuh"

namespace st {

template <int DIM, int K1, typename T, int MODE, int TAN>
cudaError_t launch_op_t(const st_problem* h, const Level& L, OpArgs& a) {
  using Cfg = OpCfg<DIM, K1, T>;
  auto kern = st_op_kernel<DIM, K1, T, MODE, TAN>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::smem_bytes);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const int ncolours = 1 << DIM;
  for (int c = 0; c < ncolours; ++c) {
    const long ncol = L.col_start[c + 1] - L.col_start[c];
    if (ncol == 0) continue;
    a.colour = c;
    for (int d = 0; d < 3; ++d) {
      a.cn[d] = L.cn[c][d];
      a.c0[d] = L.c0[c][d];
    }
    a.col_start = L.col_start[c];
    a.ncol = ncol;
    // two resident CTAs per SM; each CTA at least half a batch of cells
    long grid = (ncol + Cfg::C / 2 - 1) / (Cfg::C / 2 > 0 ? Cfg::C / 2 : 1);
    const long cap = 2L * h->nsm;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, OP_THREADS, Cfg::smem_bytes, h->stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
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

}  // namespace st
