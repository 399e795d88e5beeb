// Coarsest-level direct solve of the space-time multigrid hierarchy
// (internal, not part of the ABI).
//
// Sec. 6.3 defers the coarse-grid treatment to its references; this library
// keeps the coarse-grid solve on the FP64 side of the precision split: the
// Galerkin operator A_0 of the coarsest level is assembled densely in FP64,
// inverted once per set-up in FP32 (blocked Gauss-Jordan with partial
// pivoting), and every coarse solve is FP64 iterative refinement
//     x_{s+1} = x_s + A_0^{-1}|_FP32 (b - A_0 x_s),  residual in FP64,
// until |b - A_0 x|_2 <= rtol |b|_2 (rtol = 1e-12) or the residual stops
// decreasing, at most `max_steps` steps.  The refinement loop runs on the
// device with a convergence flag, so the launch sequence is fixed and can be
// captured in the V-cycle's CUDA graph.
#pragma once

#include "st_internal.h"

namespace st {

// largest coarsest level (space-time dofs) the direct solve accepts: the FP64
// matrix (n^2 doubles) and its FP32 inverse (n^2 floats) must stay resident
constexpr long COARSE_DIRECT_MAX = 20000;

struct CoarseState {   // device-side refinement state
  double b2, r2;       // |b|^2, |r|^2 of the accepted iterate
  int done, steps, diverged, accept;
};

struct CoarseDirect {
  long n = 0;
  double* A = nullptr;     // A_0, n x n row-major (FP64)
  float* R = nullptr;      // (P A_0)^{-1}, n x n row-major (FP32), P the pivoting row permutation
  float* T = nullptr;      // CB x n panel rows of the inversion
  int* piv = nullptr;      // pivot rows of the inversion
  int* perm = nullptr;     // composed row permutation: (P v)_j = v[perm[j]]
  double* b = nullptr;     // right-hand side, iterate, residual, trial iterate / residual
  double* x = nullptr;
  double* r = nullptr;
  double* xn = nullptr;
  double* rn = nullptr;
  float* rp = nullptr;     // P r in FP32
  CoarseState* st = nullptr;
};

cudaError_t coarse_direct_alloc(CoarseDirect& cd, long n);
void coarse_direct_free(CoarseDirect& cd);

// Geometry of the coarsest level for the dense assembly.
struct CoarseGeom {
  int dim, K1;
  int pdisc;          // P1disc pressure (element matrices in vertex form, see pdisc_T)
  int n[3];
  long g2[3], g1[3];
  long Nq2, Mv, Mp;
  double Kt[MAX_K1 * MAX_K1];
  double M1h[3][9];   // 1D Q2 mass matrices scaled by the cell size
};

// A_0 = sum over cells of the element matrices E[cell][mu] (spatial part,
// carrying tau w_mu) on the diagonal node blocks plus K_t[mu][nu] M_e on the
// velocity blocks (the temporal coupling of eq. slab-underint-jac), scattered
// colour class by colour class, then inverted.  E: [cell][mu][NE][NE]
// row-major, precision T.  err: device flag set on a zero pivot.
template <typename T>
cudaError_t coarse_direct_setup(const CoarseGeom& g, const T* E, CoarseDirect& cd, int* err, int nsm,
                                cudaStream_t s);

// d = A_0^{-1} r (FP64-accurate); r, d of precision T, length cd.n.
template <typename T>
cudaError_t coarse_direct_solve(CoarseDirect& cd, const T* r, T* d, int max_steps, double rtol, int nsm,
                                cudaStream_t s);

}  // namespace st
