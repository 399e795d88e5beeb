// Operator kernels, two space dimensions.
#include "st_op_inst.cuh"

namespace st {
cudaError_t dispatch_op_2d(const st_problem* h, const Level& L, OpArgs& a, int mode, int prec, int tangent) {
  return dispatch_op_dim<2>(h, L, a, mode, prec, tangent);
}
cudaError_t dispatch_elm_2d(const st_problem* h, const Level& L, const OpArgs& a, int prec, int tangent, void* E,
                           const int* bcells, int nbc) {
  return dispatch_elm_dim<2>(h, L, a, prec, tangent, E, bcells, nbc);
}
cudaError_t dispatch_op_batch_2d(st_problem* const* P, OpArgs* A, int n, BatchDev& bd, int mode, int prec,
                                 int tangent, cudaStream_t st) {
  return dispatch_op_batch_dim<2>(P, A, n, bd, mode, prec, tangent, st);
}
cudaError_t dispatch_cip_weights_2d(const st_problem* h, const OpArgs& a, const double* U, double* w, cudaStream_t st) {
  return dispatch_cip_weights_dim<2>(h, a, U, w, st);
}
cudaError_t upload_consts_2d(const ConstTables& t, const ConstTablesF& tf) {
  cudaError_t e = cudaMemcpyToSymbol(cT, &t, sizeof(t));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(cTf, &tf, sizeof(tf));
}
}  // namespace st
