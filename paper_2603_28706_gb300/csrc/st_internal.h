// Internal declarations of the GB300 slab solver library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/st.h"

namespace st {

constexpr int MAX_K1 = 4;      // k <= 3
constexpr int OP_THREADS = 128;

// ---------------------------------------------------------------- tables
// Mesh-independent 1D reference tables on [0,1] (computed on the host).
struct RefTables {
  double B[9];    // Q2 Lagrange basis (nodes 0, 1/2, 1) at the 3 Gauss points, [q][a]
  double Bt[9];   // transpose [a][q]
  double Dc[9];   // collocation derivative through the Gauss points, at the Gauss points [q][q']
  double W[3];    // Gauss weights
  double B1[6];   // Q1 basis at the Gauss points [q][a]
  double E[6];    // Q2 basis at x = 0 and x = 1, [end][a]
  double ED[6];   // d/dx of the Q2 basis at x = 0 and x = 1, [end][a]
  double M1[9];   // 1D Q2 mass matrix on [0,1]
  double P2[15];  // 1D Q2 prolongation: coarse basis at fine nodes 0, 1/4, .., 1, [i][a]
  double P1[6];   // 1D Q1 prolongation at fine nodes 0, 1/2, 1, [i][a]
};

struct TimeTab {
  int k;
  double t[MAX_K1], w[MAX_K1];
  double Kt[MAX_K1 * MAX_K1], mt[MAX_K1];
  double lrep[MAX_K1];  // Lagrange basis at the slab midpoint (t_rep)
};

void make_ref_tables(RefTables& R);
bool make_time_tables(int k, TimeTab& T);

// Diagonalisation of the finest-level surrogate patch in time.  With
// W = diag(w_mu / w_0) the surrogate patch is (W (x) I)(B (x) M_v + I (x) S),
// B = W^{-1} K_t = X diag(lambda) X^{-1}, so its inverse is
// (X (x) I) diag_i((lambda_i M_v + S)^{-1}) (X^{-1} W^{-1} (x) I).  One block
// is kept per real eigenvalue and per complex-conjugate pair (the pair's
// second block is the conjugate for real data):
//   s_b = sum_mu tin[b][mu] r_mu,  z_b = (lambda_b M_v + S)^{-1} s_b,
//   x_mu = sum_b Re(tout[b][mu] z_b)   (tout carries the factor 2 of a pair).
struct TimeEig {
  int nb = 0;                       // kept blocks
  double lam[MAX_K1][2];            // eigenvalue (re, im)
  double tin[MAX_K1][MAX_K1][2];    // rows of X^{-1} W^{-1}
  double tout[MAX_K1][MAX_K1][2];   // columns of X (x2 for a pair), [b][mu]
};
bool make_time_eig(const TimeTab& T, TimeEig& out);

// ----------------------------------------------------------- kernel args
struct OpArgs {
  int n[3];
  double h[3], ih[3];
  long g2[3], g1[3];
  long Nq2, Nq1, Mv, Mp;
  double vol;              // cell volume
  double Dd[3][9];         // collocation derivative along each direction, scaled by 1/h
  double Ddt[3][9];        // its transpose
  double M1d[3][9];        // 1D mass matrix scaled by h (residual mass terms)
  double tw[MAX_K1];       // tau * w_mu
  double KtV[MAX_K1 * MAX_K1];  // K_t * cell volume
  double Kt[MAX_K1 * MAX_K1];
  double mt[MAX_K1];
  // range of colour-ordered cells (or element-matrix items) of the launch
  long col_start, ncol;
  // colour-private output buffers: class c writes cbuf + c * cbuf_stride
  void* cbuf;
  long cbuf_stride;
  // physics
  double p, delta, nu, nu_inf, sigma_max, gamma1, gamma2, q_sign, vbar;
  double L[3];
  unsigned dmask;
  int inflow;
  int pdisc;               // P1disc pressure: (DIM+1) cell coefficients, see pdisc_T
  int tangent;
  // data
  const void* in;          // dU (Jacobian) or U (residual, linearise)
  void* out;               // output slab vector
  const void* vprev;
  const void* f;
  const void* cache;       // volume coefficient cache (T)
  const void* fcache;      // face coefficient cache (T)
  double* wcache;          // FP64 caches written by linearise
  double* wfcache;
  const int* face_off;     // first boundary face of every cell (linear order)
  // CIP (eq. scip-def): gamma_CIP and the face weights (T): the lagged ones
  // (Jacobian), or the scratch the residual fills from its argument; NULL = off
  double gcip;
  void* cipw;
  int* err;                // device error flag
  // colour classes (first colour-ordered index, extents); element-matrix
  // mode: fixed node mu, output matrices
  long col_start_all[9];
  int cn_all[8][3];
  int elm_mu;              // coefficient-cache node of the matrices
  int elm_stride;          // matrices per cell in the output
  int elm_slot;            // which of them is written
};

enum OpMode { OP_LIN = 0, OP_JAC = 1, OP_RES = 2, OP_ELM = 3 };

// P1disc pressure (pressure_space = 1).  On a cell the pressure is
// c_0 + sum_a c_{1+a} (2 r_a - 1), an affine function, so it lies in Q1 and
// its values at the cell's vertices m = (m_0, m_1, m_2) (bit a of m: m_a) are
// sum_j T[m][j] c_j with T[m][0] = 1, T[m][1+a] = 2 m_a - 1.  The kernels keep
// the pressure in this vertex form (element matrices, sum-factorised passes)
// and change basis where they meet slab vectors: values v = T c on input,
// tests T^T t on output.  Global index of coefficient j of cell `cell` in the
// pressure block of one time node: cell * (DIM + 1) + j.
__host__ __device__ __forceinline__ double pdisc_T(int m, int j) {
  return j == 0 ? 1.0 : (((m >> (j - 1)) & 1) ? 1.0 : -1.0);
}

// device scratch of a batched launch (st_batch.cu)
struct BatchDev {
  OpArgs* d_desc = nullptr;   // per-instance argument blocks
  long* d_first = nullptr;    // first work item of every instance (n + 1)
  unsigned* d_queue = nullptr;
  int nsm = 0;
};

template <int DIM> struct Dims {
  static constexpr int NQ = DIM == 3 ? 27 : 9;
  static constexpr int NC = DIM;
  static constexpr int NP = DIM == 3 ? 8 : 4;
  static constexpr int NL = NQ / 3;
  static constexpr int NFQ = DIM == 3 ? 9 : 3;
  static constexpr int NFP = DIM == 3 ? 4 : 2;
  static constexpr int NS = DIM == 3 ? 6 : 3;          // symmetric tensor entries
  static constexpr int NF_VOL = 2 + NS + NC;           // eta_w, c_w, A, -u w
  static constexpr int NF_FACE = 2 + NS + NC + 5 + NS + 1;  // + negw pen1 pen2 etaDw betaDw, Dg, w
  static constexpr int NE = NC * NQ + NP;              // element dofs per time node
};

// ------------------------------------------------------------- levels
struct Level {
  int n[3];
  double h[3];
  long g2[3], g1[3];
  long Nq2, Nq1, Mv, Mp, Nst, ncells;
  int cn[8][3], c0[8][3];
  long col_start[9];
  long nfaces;
  int* d_face_off = nullptr;   // ncells+1: first boundary face of every (linear) cell
  int* d_face_cell = nullptr;  // nfaces: linear cell of each boundary face
  unsigned char* d_face_side = nullptr;  // nfaces: side (2*axis + upper) of each boundary face
  // face gather lists: nodes of the boundary-cell layer (velocity first, then pressure)
  int n_gather = 0, n_gather_vel = 0;
  int* d_gnode = nullptr;
  int* d_gptr = nullptr;
  void* d_gent = nullptr;
  // Vanka / coarse operator storage (set up by the preconditioner)
};

}  // namespace st

struct st_problem {
  st_params P;
  cudaStream_t stream;
  int dim, K1, nsm;
  st::RefTables R;
  st::TimeTab T;
  std::vector<st::Level> lev;  // 0 = coarsest
  // linearisation (finest level)
  int lin_tangent = -1;
  bool lin_valid = false;
  double* d_cache64 = nullptr;
  double* d_fcache64 = nullptr;
  float* d_cache32 = nullptr;
  float* d_fcache32 = nullptr;
  size_t cache_len = 0, fcache_len = 0;
  int* d_err = nullptr;
  double* d_scratch = nullptr;     // small reduction scratch
  size_t scratch_len = 0;
  double* d_work = nullptr;        // 3 finest-level slab vectors (mass operator work)
  double* d_Ulin = nullptr;        // copy of the state of the last linearisation
  double* d_fscr = nullptr;         // compact per-face-slot outputs of the face kernel (FP64 or FP32 view)
  void* d_cbuf64 = nullptr;        // 2^dim colour-private FP64 slab vectors of the volume kernel
  void* d_cbuf32 = nullptr;        // the same in FP32 (entries no cell of a class touches stay zero)
  double* d_cipw64 = nullptr;      // CIP face weights at the linearisation state (gamma_cip > 0 only)
  float* d_cipw32 = nullptr;       // their FP32 copy
  double* d_cipw_res = nullptr;    // CIP face weights of the residual's argument (FP64 or FP32 view)
  double* d_cipf = nullptr;        // CIP tested face jumps of one apply (FP64 or FP32 view)
  size_t cipw_len = 0;
  cudaStream_t s_face = nullptr;   // internal stream: face kernels overlap the volume kernels
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaStream_t s_cap = nullptr;    // internal stream of the V-cycle (captured as a graph)
  cudaEvent_t ev_cap0 = nullptr, ev_cap1 = nullptr;
  std::string last_error;
  bool precond_valid = false;
  int precond_prec = -1;
  void* mg = nullptr;              // multigrid state (st_mg.cu)
  void* kry = nullptr;             // Krylov / Newton workspace (st_solver.cu)
};

namespace st {

// operator launches (st_operator_*.cu)
cudaError_t launch_op(st_problem* h, int level, int mode, int prec, int tangent, const void* in, void* out,
                      const void* vprev, const void* f);
// argument block of one operator launch on `level` (the data pointers included)
void prepare_op_args(const st_problem* h, int level, int prec, int tangent, const void* in, void* out,
                     const void* vprev, const void* f, OpArgs& a);
cudaError_t dispatch_op_batch_2d(st_problem* const* P, OpArgs* A, int n, BatchDev& bd, int mode, int prec,
                                 int tangent, cudaStream_t st);
cudaError_t dispatch_op_batch_3d(st_problem* const* P, OpArgs* A, int n, BatchDev& bd, int mode, int prec,
                                 int tangent, cudaStream_t st);
void fill_op_args(const st_problem* h, int level, OpArgs& a);
// CIP fields of an argument block for the given mode and precision
void set_cip_args(const st_problem* h, int mode, int prec, OpArgs& a);
// CIP face weights of the FP64 state U into the lagged caches (FP64 and FP32)
cudaError_t cip_linearize(st_problem* h, const double* U, cudaStream_t st);
cudaError_t dispatch_cip_weights_2d(const st_problem* h, const OpArgs& a, const double* U, double* w, cudaStream_t st);
cudaError_t dispatch_cip_weights_3d(const st_problem* h, const OpArgs& a, const double* U, double* w, cudaStream_t st);

st_status set_error(st_problem* h, st_status s, const std::string& msg);
st_status mg_setup(st_problem* h, st_prec prec, bool rebuild_finest);
st_status mg_vcycle(st_problem* h, st_prec prec, const void* r, void* d);
st_status cuda_check(st_problem* h, cudaError_t e, const char* where);

}  // namespace st
