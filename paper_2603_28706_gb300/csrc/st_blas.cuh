// Vector kernels: precision casts, deterministic reductions, the tensor-product
// mass operator (block mass weighting of Sec. 6.1) and Krylov BLAS-1.
#pragma once

#include <cuda_runtime.h>

#include "st_internal.h"

namespace st {

cudaError_t cast_f64_f32(const double* x, float* y, size_t n, cudaStream_t s);
cudaError_t cast_f32_f64(const float* x, double* y, size_t n, cudaStream_t s);

// y = (M_t (x) M) x on a slab vector of level `level` (M = M_x for velocity
// components, M_{x,p} for pressure), by one 1D mass pass per direction.
// work: two slab-sized buffers of type T.
template <typename T>
cudaError_t mass_apply(const st_problem* h, int level, const T* x, T* y, T* work);

// sum_j x_j y_j over n entries, deterministic, result written to dres[0] (device)
cudaError_t dot_f64(const double* x, const double* y, size_t n, double* dres, double* partial, cudaStream_t s);
// dres[j] = <V_j, w>, V_j = V + j*ld, j < nv
cudaError_t multidot_f64(const double* V, size_t ld, int nv, const double* w, size_t n, double* dres, double* partial,
                         cudaStream_t s);
// w -= sum_j c_j V_j  (c on device)
cudaError_t multiaxpy_f64(const double* V, size_t ld, int nv, const double* c, double* w, size_t n, cudaStream_t s);
// y = a*x + b*y (host scalars)
cudaError_t axpby_f64(double a, const double* x, double b, double* y, size_t n, cudaStream_t s);
// y = x * (*scale_dev)^-1
cudaError_t scale_inv_f64(const double* x, const double* sdev, double* y, size_t n, cudaStream_t s);
// y = sum_j c_j Z_j (c on device)
cudaError_t lincomb_f64(const double* Z, size_t ld, int nv, const double* c, double* y, size_t n, cudaStream_t s);

// |r|_M^2 of a FP64 finest-level slab vector (synchronises the stream)
cudaError_t mnorm2_f64(st_problem* h, int level, const double* r, double* out);


}  // namespace st
