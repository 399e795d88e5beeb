// C ABI entry points: setup, residual, linearisation, Jacobian action, M-norm.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "st_blas.cuh"
#include "st_coarse.cuh"
#include "st_internal.h"
#include "st_face.cuh"
#include "st_operator.cuh"

namespace st {

cudaError_t dispatch_op_2d(const st_problem* h, const Level& L, OpArgs& a, int mode, int prec, int tangent);
cudaError_t dispatch_op_3d(const st_problem* h, const Level& L, OpArgs& a, int mode, int prec, int tangent);
cudaError_t upload_consts_2d(const ConstTables& t, const ConstTablesF& tf);
cudaError_t upload_consts_3d(const ConstTables& t, const ConstTablesF& tf);
st_status mg_destroy(st_problem* h);
void krylov_destroy(st_problem* h);

st_status set_error(st_problem* h, st_status s, const std::string& msg) {
  if (h) h->last_error = msg;
  return s;
}

st_status cuda_check(st_problem* h, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return ST_OK;
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  return set_error(h, e == cudaErrorMemoryAllocation ? ST_ENOMEM : ST_ECUDA, buf);
}

namespace {

void build_consts(const RefTables& R, ConstTables& t, ConstTablesF& tf) {
  memset(&t, 0, sizeof(t));
  for (int i = 0; i < 9; ++i) {
    t.B[i] = R.B[i];
    t.Bt[i] = R.Bt[i];
    t.Dc[i] = R.Dc[i];
  }
  const double* mats[2] = {R.B, R.Bt};
  double* outs[2] = {t.BS, t.BtS};
  for (int k = 0; k < 2; ++k) {
    const double* m = mats[k];
    outs[k][0] = 0.5 * (m[0] + m[2]);
    outs[k][1] = 0.5 * (m[0] - m[2]);
    outs[k][2] = m[1];
    outs[k][3] = m[3];
    outs[k][4] = m[4];
  }
  for (int i = 0; i < 3; ++i) t.W[i] = R.W[i];
  for (int i = 0; i < 6; ++i) {
    t.B1[i] = R.B1[i];
    t.E[i] = R.E[i];
    t.ED[i] = R.ED[i];
  }
  for (int qz = 0; qz < 3; ++qz)
    for (int qy = 0; qy < 3; ++qy)
      for (int qx = 0; qx < 3; ++qx) {
        const int q = qx + 3 * qy + 9 * qz;
        t.WQ3[q] = R.W[qx] * R.W[qy] * R.W[qz];
        for (int m = 0; m < 8; ++m)
          t.PSI3[q * 8 + m] = R.B1[qx * 2 + (m & 1)] * R.B1[qy * 2 + ((m >> 1) & 1)] * R.B1[qz * 2 + (m >> 2)];
        if (qz == 0) {
          const int q2 = qx + 3 * qy;
          t.WQ2[q2] = R.W[qx] * R.W[qy];
          for (int m = 0; m < 4; ++m) t.PSI2[q2 * 4 + m] = R.B1[qx * 2 + (m & 1)] * R.B1[qy * 2 + (m >> 1)];
        }
      }
  for (int i2 = 0; i2 < 3; ++i2)
    for (int i1 = 0; i1 < 3; ++i1) {
      const int fq = i1 + 3 * i2;
      t.FW3[fq] = R.W[i1] * R.W[i2];
      for (int m = 0; m < 4; ++m) t.FPSI3[fq * 4 + m] = R.B1[i1 * 2 + (m & 1)] * R.B1[i2 * 2 + (m >> 1)];
    }
  for (int i1 = 0; i1 < 3; ++i1) {
    t.FW2[i1] = R.W[i1];
    for (int m = 0; m < 2; ++m) t.FPSI2[i1 * 2 + m] = R.B1[i1 * 2 + m];
  }
  // float copy
  const double* src = reinterpret_cast<const double*>(&t);
  float* dst = reinterpret_cast<float*>(&tf);
  static_assert(sizeof(ConstTables) == 2 * sizeof(ConstTablesF), "layout");
  for (size_t i = 0; i < sizeof(ConstTables) / sizeof(double); ++i) dst[i] = (float)src[i];
}

bool g_consts_done[2] = {false, false};

void make_level(const st_params& P, int nx, int ny, int nz, Level& L) {
  const int d = P.dim;
  L.n[0] = nx;
  L.n[1] = ny;
  L.n[2] = d == 3 ? nz : 1;
  const double Ls[3] = {P.Lx, P.Ly, d == 3 ? P.Lz : 1.0};
  L.Nq2 = L.Nq1 = L.ncells = 1;
  for (int a = 0; a < 3; ++a) {
    const bool act = a < d;
    L.h[a] = act ? Ls[a] / L.n[a] : 1.0;
    L.g2[a] = act ? 2L * L.n[a] + 1 : 1;
    L.g1[a] = act ? (long)L.n[a] + 1 : 1;
    L.Nq2 *= L.g2[a];
    L.Nq1 *= L.g1[a];
    L.ncells *= L.n[a];
  }
  if (P.pressure_space == 1) L.Nq1 = L.ncells * (d + 1);  // P1disc: 1 + dim coefficients per cell
  L.Mv = d * L.Nq2;
  L.Mp = L.Nq1;
  L.Nst = (long)(P.k + 1) * (L.Mv + L.Mp);
  const int ncol = 1 << d;
  L.col_start[0] = 0;
  for (int c = 0; c < 8; ++c) {
    long cnt = 1;
    for (int a = 0; a < 3; ++a) {
      const int bit = (a < d) ? ((c >> a) & 1) : 0;
      L.c0[c][a] = bit;
      L.cn[c][a] = (a < d) ? (L.n[a] - bit + 1) / 2 : 1;
      if (c >= ncol) L.cn[c][a] = 0;
      cnt *= L.cn[c][a];
    }
    L.col_start[c + 1] = L.col_start[c] + (c < ncol ? cnt : 0);
  }
}

// boundary faces in linear cell order, each cell's boundary sides in
// increasing side order: offsets per cell, cell and side per face
std::vector<int> face_lists(const st_params& P, Level& L, std::vector<int>& fcell, std::vector<unsigned char>& fside) {
  const int d = P.dim;
  std::vector<int> off(L.ncells + 1, 0);
  fcell.clear();
  fside.clear();
  for (long cell = 0; cell < L.ncells; ++cell) {
    const int e3[3] = {(int)(cell % L.n[0]), (int)((cell / L.n[0]) % L.n[1]), (int)(cell / ((long)L.n[0] * L.n[1]))};
    off[cell] = (int)fcell.size();
    for (int sd = 0; sd < 2 * d; ++sd) {
      const int ax = sd >> 1, up = sd & 1;
      const bool on = up ? (e3[ax] == L.n[ax] - 1) : (e3[ax] == 0);
      if (!on) continue;
      fcell.push_back((int)cell);
      fside.push_back((unsigned char)sd);
    }
  }
  off[L.ncells] = (int)fcell.size();
  L.nfaces = (long)fcell.size();
  return off;
}

// Per node of the boundary-cell layer: the (face, face-node) pairs that reach
// it, with the normal-direction weights of the Q2 basis (velocity nodes) or
// the face pressure node (pressure nodes).
cudaError_t build_gather(const st_problem* h, Level& L, const std::vector<int>& off) {
  const int d = h->dim;
  std::vector<std::vector<GatherEnt>> vel(L.Nq2), pres(L.Nq1);
  for (long cell = 0; cell < L.ncells; ++cell) {
    const int e3[3] = {(int)(cell % L.n[0]), (int)((cell / L.n[0]) % L.n[1]), (int)(cell / ((long)L.n[0] * L.n[1]))};
    int rank = 0;
    for (int sd = 0; sd < 2 * d; ++sd) {
      const int ax = sd >> 1, up = sd & 1;
      const bool on = up ? (e3[ax] == L.n[ax] - 1) : (e3[ax] == 0);
      if (!on) continue;
      const int fid = off[cell] + rank++;
      const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
      for (int z = 0; z < (d == 3 ? 3 : 1); ++z)
        for (int y = 0; y < 3; ++y)
          for (int x = 0; x < 3; ++x) {
            const int l3[3] = {x, y, z};
            const long gn = (2L * e3[0] + x) + L.g2[0] * ((2L * e3[1] + y) + L.g2[1] * (2L * e3[2] + z));
            GatherEnt g;
            g.fid = fid;
            g.tn = l3[t1] + 3 * (d == 3 ? l3[t2] : 0);
            g.e = h->R.E[up * 3 + l3[ax]];
            g.ed = h->R.ED[up * 3 + l3[ax]];
            vel[gn].push_back(g);
          }
      for (int z = 0; z < (d == 3 ? 2 : 1); ++z)
        for (int y = 0; y < 2; ++y)
          for (int x = 0; x < 2; ++x) {
            const int m3[3] = {x, y, z};
            if (m3[ax] != up) continue;
            GatherEnt g;
            g.fid = fid;
            g.tn = m3[t1] + 2 * (d == 3 ? m3[t2] : 0);
            g.ed = 0.0;
            if (h->P.pressure_space == 1) {
              // P1disc: the face-vertex test reaches every coefficient j of the cell with weight T[m][j]
              const int mc = x + 2 * y + 4 * z;
              for (int j = 0; j <= d; ++j) {
                g.e = pdisc_T(mc, j);
                pres[cell * (d + 1) + j].push_back(g);
              }
            } else {
              const long gp = (e3[0] + x) + L.g1[0] * ((e3[1] + y) + L.g1[1] * (e3[2] + z));
              g.e = 1.0;
              pres[gp].push_back(g);
            }
          }
    }
  }
  std::vector<int> node, ptr(1, 0);
  std::vector<GatherEnt> ent;
  for (long i = 0; i < L.Nq2; ++i)
    if (!vel[i].empty()) {
      node.push_back((int)i);
      ent.insert(ent.end(), vel[i].begin(), vel[i].end());
      ptr.push_back((int)ent.size());
    }
  L.n_gather_vel = (int)node.size();
  for (long i = 0; i < L.Nq1; ++i)
    if (!pres[i].empty()) {
      node.push_back((int)i);
      ent.insert(ent.end(), pres[i].begin(), pres[i].end());
      ptr.push_back((int)ent.size());
    }
  L.n_gather = (int)node.size();
  if (node.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(&L.d_gnode, node.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(L.d_gnode, node.data(), node.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&L.d_gptr, ptr.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(L.d_gptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&L.d_gent, ent.size() * sizeof(GatherEnt));
  if (e == cudaSuccess) e = cudaMemcpy(L.d_gent, ent.data(), ent.size() * sizeof(GatherEnt), cudaMemcpyHostToDevice);
  return e;
}

st_status check_params(const st_params& P, std::string& why) {
  if (P.dim != 2 && P.dim != 3) return why = "dim must be 2 or 3", ST_EINVAL;
  if (P.nx < 1 || P.ny < 1 || (P.dim == 3 && P.nz < 1)) return why = "cell counts must be >= 1", ST_EINVAL;
  if (!(P.Lx > 0 && P.Ly > 0 && (P.dim == 2 || P.Lz > 0))) return why = "box lengths must be positive", ST_EINVAL;
  if (P.k < 0 || P.k >= MAX_K1) return why = "k must be in [0, 3]", ST_EINVAL;
  if (!(P.dt > 0)) return why = "dt must be positive", ST_EINVAL;
  if (!(P.p > 1.0 && P.p <= 2.0)) return why = "p must be in (1, 2]", ST_EINVAL;
  if (!(P.delta > 0 && P.nu >= 0 && P.nu_inf >= 0)) return why = "need delta > 0, nu >= 0, nu_inf >= 0", ST_EINVAL;
  if (!(P.sigma_max >= 0)) return why = "sigma_max must be >= 0", ST_EINVAL;
  if (!(P.gamma_cip >= 0 && P.gamma_cip < 1e300)) return why = "gamma_cip must be finite and >= 0", ST_EINVAL;
  if (P.finest_patches != 0 && P.finest_patches != 1) return why = "finest_patches must be 0 or 1", ST_EINVAL;
  if (P.finest_patches == 1 && P.gamma_cip > 0)
    return why = "exact finest patches (finest_patches = 1) do not carry the CIP term", ST_EINVAL;
  if (P.levels < 1) return why = "levels must be >= 1", ST_EINVAL;
  const long div = 1L << (P.levels - 1);
  if (P.nx % div || P.ny % div || (P.dim == 3 && P.nz % div))
    return why = "cell counts must be divisible by 2^(levels-1)", ST_EINVAL;
  if (P.inflow_profile != 0 && P.inflow_profile != 1) return why = "inflow_profile must be 0 or 1", ST_EINVAL;
  if (P.coarse_solve != 0 && P.coarse_solve != 1) return why = "coarse_solve must be 0 or 1", ST_EINVAL;
  if (P.pressure_space != 0 && P.pressure_space != 1) return why = "pressure_space must be 0 or 1", ST_EINVAL;
  if (P.smoother < 0 || P.smoother > 2) return why = "smoother must be 0, 1 or 2", ST_EINVAL;
  if (!(P.omega_coarse >= 0.0) || !std::isfinite(P.omega_coarse))
    return why = "omega_coarse must be finite and >= 0", ST_EINVAL;
  if (P.patch_type != 0 && P.patch_type != 1) return why = "patch_type must be 0 or 1", ST_EINVAL;
  if (P.patch_type == 1 && (P.finest_patches != 1 || P.gamma_cip > 0 || P.pressure_space != 0))
    return why = "patch_type = 1 (vertex-star patches) needs finest_patches = 1, gamma_cip = 0 and pressure_space = 0",
           ST_EINVAL;
  if (P.coarse_solve == 1) {
    long n2 = 1, n1 = 1;
    const int nn[3] = {P.nx, P.ny, P.dim == 3 ? P.nz : 0};
    for (int a = 0; a < P.dim; ++a) {
      const long m = nn[a] / div;
      n2 *= 2 * m + 1;
      n1 *= m + 1;
    }
    long ncells0 = 1;
    for (int a = 0; a < P.dim; ++a) ncells0 *= nn[a] / div;
    const long n0 = (long)(P.k + 1) * (P.dim * n2 + (P.pressure_space == 1 ? ncells0 * (P.dim + 1) : n1));
    if (n0 > COARSE_DIRECT_MAX)
      return why = "coarse_solve = 1: the coarsest level has " + std::to_string(n0) + " dofs, the direct solve takes at most " +
                   std::to_string(COARSE_DIRECT_MAX) + " (add levels)", ST_EINVAL;
  }
  const long ncells = (long)P.nx * P.ny * (P.dim == 3 ? P.nz : 1);
  if (ncells > (1L << 30)) return why = "mesh too large", ST_EINVAL;
  return ST_OK;
}

}  // namespace

void fill_op_args(const st_problem* h, int level, OpArgs& a) {
  const Level& L = h->lev[level];
  const st_params& P = h->P;
  memset(&a, 0, sizeof(a));
  for (int d = 0; d < 3; ++d) {
    a.n[d] = L.n[d];
    a.h[d] = L.h[d];
    a.ih[d] = 1.0 / L.h[d];
    a.g2[d] = L.g2[d];
    a.g1[d] = L.g1[d];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        a.Dd[d][i * 3 + j] = h->R.Dc[i * 3 + j] / L.h[d];
        a.Ddt[d][j * 3 + i] = h->R.Dc[i * 3 + j] / L.h[d];
        a.M1d[d][i * 3 + j] = h->R.M1[i * 3 + j] * L.h[d];
      }
  }
  a.Nq2 = L.Nq2;
  a.Nq1 = L.Nq1;
  a.Mv = L.Mv;
  a.Mp = L.Mp;
  a.vol = L.h[0] * L.h[1] * (P.dim == 3 ? L.h[2] : 1.0);
  const int K1 = h->K1;
  for (int i = 0; i < K1; ++i) {
    a.tw[i] = P.dt * h->T.w[i];
    a.mt[i] = h->T.mt[i];
    for (int j = 0; j < K1; ++j) {
      a.Kt[i * K1 + j] = h->T.Kt[i * K1 + j];
      a.KtV[i * K1 + j] = h->T.Kt[i * K1 + j] * a.vol;
    }
  }
  a.p = P.p;
  a.delta = P.delta;
  a.nu = P.nu;
  a.nu_inf = P.nu_inf;
  a.sigma_max = P.sigma_max;
  a.gamma1 = P.gamma1;
  a.gamma2 = P.gamma2;
  a.q_sign = P.q_sign;
  a.vbar = P.vbar;
  a.L[0] = P.Lx;
  a.L[1] = P.Ly;
  a.L[2] = P.dim == 3 ? P.Lz : 1.0;
  a.dmask = P.dirichlet_mask;
  a.inflow = P.inflow_profile;
  a.pdisc = P.pressure_space == 1 ? 1 : 0;
  a.face_off = L.d_face_off;
  a.err = h->d_err;
  a.gcip = P.gamma_cip;
  a.cipw = nullptr;
  for (int c = 0; c < 9; ++c) a.col_start_all[c] = L.col_start[c];
  for (int c = 0; c < 8; ++c)
    for (int d = 0; d < 3; ++d) a.cn_all[c][d] = L.cn[c][d];
}

void prepare_op_args(const st_problem* h, int level, int prec, int tangent, const void* in, void* out,
                     const void* vprev, const void* f, OpArgs& a) {
  fill_op_args(h, level, a);
  a.tangent = tangent;
  a.in = in;
  a.out = out;
  a.vprev = vprev;
  a.f = f;
  a.cache = prec == ST_FP64 ? (const void*)h->d_cache64 : (const void*)h->d_cache32;
  a.fcache = prec == ST_FP64 ? (const void*)h->d_fcache64 : (const void*)h->d_fcache32;
  a.wcache = h->d_cache64;
  a.wfcache = h->d_fcache64;
}

// CIP on the finest level of the Jacobian (lagged weights of the linearisation)
// and of the residual (weights of its argument); off for the linearisation
// and for the element matrices of the preconditioner
void set_cip_args(const st_problem* h, int mode, int prec, OpArgs& a) {
  a.cipw = nullptr;
  if (!(h->P.gamma_cip > 0) || !h->d_cipw64) return;
  if (mode == OP_JAC) a.cipw = prec == ST_FP64 ? (void*)h->d_cipw64 : (void*)h->d_cipw32;
  if (mode == OP_RES) a.cipw = h->d_cipw_res;
}

cudaError_t cip_linearize(st_problem* h, const double* U, cudaStream_t st) {
  if (!(h->P.gamma_cip > 0) || !h->d_cipw64) return cudaSuccess;
  OpArgs a;
  fill_op_args(h, (int)h->lev.size() - 1, a);
  cudaError_t e = h->dim == 2 ? dispatch_cip_weights_2d(h, a, U, h->d_cipw64, st)
                              : dispatch_cip_weights_3d(h, a, U, h->d_cipw64, st);
  if (e == cudaSuccess) e = cast_f64_f32(h->d_cipw64, h->d_cipw32, h->cipw_len, st);
  return e;
}

cudaError_t launch_op(st_problem* h, int level, int mode, int prec, int tangent, const void* in, void* out,
                      const void* vprev, const void* f) {
  OpArgs a;
  fill_op_args(h, level, a);
  a.tangent = tangent;
  a.in = in;
  a.out = out;
  a.vprev = vprev;
  a.f = f;
  a.cache = prec == ST_FP64 ? (const void*)h->d_cache64 : (const void*)h->d_cache32;
  a.fcache = prec == ST_FP64 ? (const void*)h->d_fcache64 : (const void*)h->d_fcache32;
  a.wcache = h->d_cache64;
  a.wfcache = h->d_fcache64;
  if (level == (int)h->lev.size() - 1) set_cip_args(h, mode, prec, a);
  const Level& L = h->lev[level];
  return h->dim == 2 ? dispatch_op_2d(h, L, a, mode, prec, tangent) : dispatch_op_3d(h, L, a, mode, prec, tangent);
}

}  // namespace st

using namespace st;

extern "C" {

st_status st_setup_mesh(const st_params* params, void* cuda_stream, st_problem** out) {
  if (!params || !out) return ST_EINVAL;
  *out = nullptr;
  std::string why;
  st_status s = check_params(*params, why);
  if (s != ST_OK) {
    fprintf(stderr, "st_setup_mesh: %s\n", why.c_str());
    return s;
  }
  st_problem* h = new (std::nothrow) st_problem();
  if (!h) return ST_ENOMEM;
  h->P = *params;
  h->stream = (cudaStream_t)cuda_stream;
  h->dim = params->dim;
  h->K1 = params->k + 1;
  make_ref_tables(h->R);
  if (!make_time_tables(params->k, h->T)) {
    delete h;
    return ST_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    fprintf(stderr, "st_setup_mesh: %s\n", cudaGetErrorString(e));
    delete h;
    return ST_ECUDA;
  }
  const int di = h->dim - 2;
  if (!g_consts_done[di]) {
    ConstTables t;
    ConstTablesF tf;
    build_consts(h->R, t, tf);
    e = di == 0 ? upload_consts_2d(t, tf) : upload_consts_3d(t, tf);
    if (e != cudaSuccess) {
      fprintf(stderr, "st_setup_mesh: constant upload: %s\n", cudaGetErrorString(e));
      delete h;
      return ST_ECUDA;
    }
    g_consts_done[di] = true;
  }
  const int nl = params->levels;
  h->lev.resize(nl);
  for (int l = 0; l < nl; ++l) {
    const int sh = nl - 1 - l;
    make_level(*params, params->nx >> sh, params->ny >> sh, params->dim == 3 ? (params->nz >> sh) : 1, h->lev[l]);
    std::vector<int> fcell;
    std::vector<unsigned char> fside;
    std::vector<int> off = face_lists(*params, h->lev[l], fcell, fside);
    if (fcell.empty()) {
      fcell.push_back(0);
      fside.push_back(0);
    }
    Level& Lv = h->lev[l];
    e = cudaMalloc(&Lv.d_face_off, off.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(Lv.d_face_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&Lv.d_face_cell, fcell.size() * sizeof(int));
    if (e == cudaSuccess)
      e = cudaMemcpy(Lv.d_face_cell, fcell.data(), fcell.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&Lv.d_face_side, fside.size());
    if (e == cudaSuccess) e = cudaMemcpy(Lv.d_face_side, fside.data(), fside.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = build_gather(h, Lv, off);
    if (e != cudaSuccess) {
      st_destroy(h);
      return e == cudaErrorMemoryAllocation ? ST_ENOMEM : ST_ECUDA;
    }
  }
  const Level& F = h->lev.back();
  const int NQ = h->dim == 3 ? 27 : 9, NFQ = h->dim == 3 ? 9 : 3;
  const int NF_VOL = h->dim == 3 ? Dims<3>::NF_VOL : Dims<2>::NF_VOL;
  const int NF_FACE = h->dim == 3 ? Dims<3>::NF_FACE : Dims<2>::NF_FACE;
  h->cache_len = (size_t)F.ncells * h->K1 * NF_VOL * NQ;
  h->fcache_len = (size_t)(F.nfaces > 0 ? F.nfaces : 1) * h->K1 * NF_FACE * NFQ;
  h->scratch_len = 4096;
  e = cudaMalloc(&h->d_cache64, h->cache_len * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_fcache64, h->fcache_len * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_cache32, h->cache_len * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_fcache32, h->fcache_len * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_err, 16 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_scratch, h->scratch_len * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_work, 3 * (size_t)F.Nst * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_Ulin, (size_t)F.Nst * sizeof(double));
  if (h->P.gamma_cip > 0) {
    // CIP face weights: lagged (FP64, FP32 copy) and the residual's scratch
    h->cipw_len = (size_t)h->dim * F.ncells * h->K1 * NFQ;
    if (e == cudaSuccess) e = cudaMalloc(&h->d_cipw64, h->cipw_len * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_cipw32, h->cipw_len * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_cipw_res, h->cipw_len * sizeof(double));
    // tested face jumps: per face, component and node the 3^(dim-1) face-plane values
    if (e == cudaSuccess) e = cudaMalloc(&h->d_cipf, h->cipw_len * h->dim * sizeof(double));
  }
  {
    // colour-private volume outputs; zero once: each class always writes the
    // same entries, the others stay zero
    const size_t nb = (size_t)(1 << h->dim) * F.Nst;
    if (e == cudaSuccess) e = cudaMalloc(&h->d_cbuf64, nb * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_cbuf32, nb * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_cbuf64, 0, nb * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_cbuf32, 0, nb * sizeof(float), h->stream);
  }
  {
    const int nout = h->dim == 3 ? 2 * 3 * 9 + 4 : 2 * 2 * 3 + 2;
    const size_t nf = (size_t)(F.nfaces > 0 ? F.nfaces : 1) * h->K1 * nout;
    if (e == cudaSuccess) e = cudaMalloc(&h->d_fscr, nf * sizeof(double));
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_face, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->s_cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_cap0, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_cap1, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, 16 * sizeof(int), h->stream);
  if (e != cudaSuccess) {
    st_destroy(h);
    return e == cudaErrorMemoryAllocation ? ST_ENOMEM : ST_ECUDA;
  }
  *out = h;
  return ST_OK;
}

st_status st_destroy(st_problem* h) {
  if (!h) return ST_OK;
  mg_destroy(h);
  krylov_destroy(h);
  for (auto& L : h->lev) {
    cudaFree(L.d_face_off);
    cudaFree(L.d_face_cell);
    cudaFree(L.d_face_side);
    cudaFree(L.d_gnode);
    cudaFree(L.d_gptr);
    cudaFree(L.d_gent);
  }
  cudaFree(h->d_cbuf64);
  cudaFree(h->d_cbuf32);
  cudaFree(h->d_cache64);
  cudaFree(h->d_fcache64);
  cudaFree(h->d_cache32);
  cudaFree(h->d_fcache32);
  cudaFree(h->d_err);
  cudaFree(h->d_scratch);
  cudaFree(h->d_work);
  cudaFree(h->d_Ulin);
  cudaFree(h->d_fscr);
  cudaFree(h->d_cipw64);
  cudaFree(h->d_cipw32);
  cudaFree(h->d_cipw_res);
  cudaFree(h->d_cipf);
  if (h->s_face) cudaStreamDestroy(h->s_face);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->s_cap) cudaStreamDestroy(h->s_cap);
  if (h->ev_cap0) cudaEventDestroy(h->ev_cap0);
  if (h->ev_cap1) cudaEventDestroy(h->ev_cap1);
  delete h;
  return ST_OK;
}

size_t st_num_dofs(const st_problem* h, int level) {
  if (!h || level < 0 || level >= (int)h->lev.size()) return 0;
  return (size_t)h->lev[level].Nst;
}

const char* st_last_error(const st_problem* h) {
  if (!h) return "null handle";
  return h->last_error.c_str();
}

st_status st_residual(st_problem* h, st_prec prec, const void* U, const void* v_prev, const void* f, void* R) {
  if (!h) return ST_EINVAL;
  if (!U || !R || !v_prev) return set_error(h, ST_EINVAL, "st_residual: U, v_prev and R are required");
  if (prec != ST_FP64 && prec != ST_FP32) return set_error(h, ST_EINVAL, "st_residual: bad precision");
  const int L = (int)h->lev.size() - 1;
  return cuda_check(h, launch_op(h, L, OP_RES, prec, 0, U, R, v_prev, f), "st_residual");
}

st_status st_linearize(st_problem* h, st_tangent tangent, const void* U) {
  if (!h) return ST_EINVAL;
  if (!U) return set_error(h, ST_EINVAL, "st_linearize: U is required");
  if (tangent < ST_PIC || tangent > ST_MODN) return set_error(h, ST_EINVAL, "st_linearize: bad tangent");
  const int L = (int)h->lev.size() - 1;
  st_status s = cuda_check(h, cudaMemcpyAsync(h->d_Ulin, U, h->lev[L].Nst * sizeof(double), cudaMemcpyDeviceToDevice,
                                              h->stream), "st_linearize copy");
  if (s != ST_OK) return s;
  s = cuda_check(h, launch_op(h, L, OP_LIN, ST_FP64, tangent, U, nullptr, nullptr, nullptr), "st_linearize");
  if (s != ST_OK) return s;
  s = cuda_check(h, cast_f64_f32(h->d_cache64, h->d_cache32, h->cache_len, h->stream), "st_linearize cast");
  if (s != ST_OK) return s;
  if (h->lev[L].nfaces > 0)
    s = cuda_check(h, cast_f64_f32(h->d_fcache64, h->d_fcache32, h->fcache_len, h->stream), "st_linearize cast");
  if (s != ST_OK) return s;
  s = cuda_check(h, cip_linearize(h, (const double*)U, h->stream), "st_linearize CIP weights");
  if (s != ST_OK) return s;
  h->lin_tangent = tangent;
  h->lin_valid = true;
  h->precond_valid = false;
  return ST_OK;
}

st_status st_jacobian_apply(st_problem* h, st_tangent tangent, st_prec prec, const void* U_state, const void* dU,
                            void* out) {
  if (!h) return ST_EINVAL;
  if (!dU || !out) return set_error(h, ST_EINVAL, "st_jacobian_apply: dU and out are required");
  if (prec != ST_FP64 && prec != ST_FP32) return set_error(h, ST_EINVAL, "st_jacobian_apply: bad precision");
  if (U_state) {
    st_status s = st_linearize(h, tangent, U_state);
    if (s != ST_OK) return s;
  } else if (!h->lin_valid || h->lin_tangent != tangent) {
    return set_error(h, ST_EINVAL, "st_jacobian_apply: no linearisation for this tangent (call st_linearize)");
  }
  const int L = (int)h->lev.size() - 1;
  return cuda_check(h, launch_op(h, L, OP_JAC, prec, tangent, dU, out, nullptr, nullptr), "st_jacobian_apply");
}

st_status st_mnorm(st_problem* h, const void* r, double* out) {
  if (!h) return ST_EINVAL;
  if (!r || !out) return set_error(h, ST_EINVAL, "st_mnorm: r and out are required");
  const int L = (int)h->lev.size() - 1;
  double v = 0.0;
  st_status s = cuda_check(h, mnorm2_f64(h, L, (const double*)r, &v), "st_mnorm");
  if (s != ST_OK) return s;
  *out = std::sqrt(v);
  return ST_OK;
}

}  // extern "C"
