// Boundary-face terms of the slab operator (sm_103a).
//
// For the boundary cells of one colour class this kernel adds the face
// integrals of the residual / Jacobian, or (OP_LIN) writes the face
// coefficient cache:
//   on all of Gamma:  ((u.n) u, z)                          (eq. Defc)
//   on Gamma_D:       -((S(Du) - pi I) n, z) + B_gamma(u - g_D, (z, q))  (eq. def-a-gam,
//                     eq. def-b-gam), linearised for the Jacobian with the
//                     selected tangent and the inflow factor (u.n)_- lagged.
// Work decomposition: one launch covers every "face slot" (boundary face,
// Radau node); a CTA takes FS consecutive slots so every stage spreads full
// warps over many faces.  Stages: gather the normal node lines -> face-plane
// values/normal derivatives at the 3x3 face points (tangential passes) ->
// tangential derivatives -> pointwise face terms -> transposed passes ->
// compact per-slot output (values and normal-derivative weights at the face
// nodes, pressure tests) in a scratch array.  st_face_add then adds these
// into the output per global node, after the volume kernel.
#pragma once

#include "st_operator.cuh"

namespace st {

template <int DIM, typename T>
struct FaceCfg {
  using D = Dims<DIM>;
  // face slots per batch: small, so that a face CTA fits in the shared memory
  // the volume kernel's CTAs leave free on an SM and the two kernels overlap
  static constexpr int FS = DIM == 3 ? 8 : 64;
  // per face slot: PV, PN (NC x NFQ), PT (NC x (DIM-1) x NFQ), FQ (NFQ), FPn (NFP)
  static constexpr int oPV = 0;
  static constexpr int oPN = D::NC * D::NFQ;
  static constexpr int oPT = 2 * D::NC * D::NFQ;
  static constexpr int oFQ = oPT + D::NC * (DIM - 1) * D::NFQ;
  static constexpr int oFP = oFQ + D::NFQ;
  static constexpr int per_slot = oFP + D::NFP;
  // + per slot: cell, side, face, node; the cell's first Q2 and Q1 grid index
  static constexpr size_t smem_bytes =
      (size_t)FS * per_slot * sizeof(T) + (size_t)FS * 4 * sizeof(int) + 8 + (size_t)FS * 2 * sizeof(long) + 64;
};

// Pointwise face terms at face point fq of one face slot whose normal is
// +-e_AX (AX a compile-time constant, so every small tensor stays in registers).
template <int DIM, int K1, typename T, int MODE, int TAN, int AX>
__device__ __forceinline__ void face_point(const OpArgs& a, T* w, int fq, int side, int mu, int cellL, int fid) {
  using D = Dims<DIM>;
  using Cfg = FaceCfg<DIM, T>;
  constexpr int NC = D::NC, NFQ = D::NFQ, NS = D::NS, NFP = D::NFP;
  constexpr int ax = AX, t1 = AX == 0 ? 1 : 0, t2 = AX == 2 ? 1 : 2;
  const auto& ct = CT<T>::t();
  const int up = side & 1;
  const bool isD = (a.dmask >> side) & 1u;
      T u[3] = {0, 0, 0}, g[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        u[c] = w[Cfg::oPV + c * NFQ + fq];
        g[c][ax] = w[Cfg::oPN + c * NFQ + fq];
        g[c][t1] = w[Cfg::oPT + (c * (DIM - 1) + 0) * NFQ + fq];
        if (DIM == 3) g[c][t2] = w[Cfg::oPT + (c * (DIM - 1) + 1) * NFQ + fq];
      }
      const T nsg = up ? (T)1 : (T)-1;  // n = nsg e_ax
      T pf = 0;
#pragma unroll
      for (int m = 0; m < NFP; ++m)
        pf += ((DIM == 3) ? ct.FPSI3[fq * 4 + m] : ct.FPSI2[fq * 2 + m]) * w[Cfg::oFP + m];
      const double hD = a.h[ax];
      T V[3] = {0, 0, 0}, Gf[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, Qf = 0;
      if constexpr (MODE == OP_LIN || MODE == OP_RES) {
        // physical point and face weight (Gauss points 1/2 -+ sqrt(15)/10)
        const int cell = cellL;
        const int e3[3] = {cell % a.n[0], (cell / a.n[0]) % a.n[1], (DIM == 3) ? cell / (a.n[0] * a.n[1]) : 0};
        const double gpt[3] = {0.5 - 0.3872983346207417, 0.5, 0.5 + 0.3872983346207417};
        double r3[3] = {0, 0, 0};
        r3[ax] = up ? 1.0 : 0.0;
        r3[t1] = gpt[fq % 3];
        if (DIM == 3) r3[t2] = gpt[fq / 3];
        double x[3];
        for (int d = 0; d < 3; ++d) x[d] = d < DIM ? (e3[d] + r3[d]) * a.h[d] : 0.0;
        double fw = ((DIM == 3) ? cT.FW3[fq] : cT.FW2[fq]) * a.tw[mu];
        for (int d = 0; d < DIM; ++d)
          if (d != ax) fw *= a.h[d];
        double gl[3], ggr[9];
        lifting(a, x, gl, ggr);
        double Dgf[3][3], g2n = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            Dgf[i][j] = 0.5 * (ggr[i * 3 + j] + ggr[j * 3 + i]);
            g2n += Dgf[i][j] * Dgf[i][j];
          }
        const double DgD = a.delta * a.delta + g2n;
        const double etaD = a.nu_inf + a.nu * pow(DgD, 0.5 * (a.p - 2.0));
        const double betaD = a.nu * (a.p - 2.0) * pow(DgD, 0.5 * (a.p - 4.0));
        if constexpr (MODE == OP_LIN) {
          // coefficients of the linearisation at the face point (FP64, Sec. 4.1)
          double Am[NS];
#pragma unroll
          for (int i = 0; i < DIM; ++i) Am[i] = (double)g[i][i];
          Am[DIM] = 0.5 * ((double)g[0][1] + (double)g[1][0]);
          if (DIM == 3) {
            Am[4] = 0.5 * ((double)g[0][2] + (double)g[2][0]);
            Am[5] = 0.5 * ((double)g[1][2] + (double)g[2][1]);
          }
          double a2 = 0.0;
#pragma unroll
          for (int i = 0; i < NS; ++i) a2 += (i < DIM ? 1.0 : 2.0) * Am[i] * Am[i];
          const double D2 = a.delta * a.delta + a2;
          const double mu_m = a.nu * pow(D2, 0.5 * (a.p - 2.0));
          const double eta = a.nu_inf + mu_m;
          double cfac = 0.0;
          if (a.tangent == ST_EXN) {
            cfac = (a.p - 2.0) * mu_m / D2;
          } else if (a.tangent == ST_MODN) {
            const double sig = mu_m * sqrt(a2);
            const double sc = sig > 0.0 ? fmin(1.0, a.sigma_max / sig) : 0.0;
            cfac = sc * (a.p - 2.0) * mu_m / D2;
          }
          const double un = (double)nsg * (double)u[ax];
          const double negp = 0.5 * (fabs(un) - un);
          double Dg[NS];
#pragma unroll
          for (int i = 0; i < DIM; ++i) Dg[i] = Dgf[i][i];
          Dg[DIM] = Dgf[0][1];
          if (DIM == 3) {
            Dg[4] = Dgf[0][2];
            Dg[5] = Dgf[1][2];
          }
          double* cp = a.wfcache + (((long)fid * K1 + mu) * (long)D::NF_FACE) * NFQ + fq;
          int o = 0;
          cp[(o++) * NFQ] = eta * fw;
          cp[(o++) * NFQ] = cfac * fw;
#pragma unroll
          for (int i = 0; i < NS; ++i) cp[(o++) * NFQ] = Am[i];
#pragma unroll
          for (int c = 0; c < NC; ++c) cp[(o++) * NFQ] = (double)u[c] * fw;
          cp[(o++) * NFQ] = negp * fw;
          cp[(o++) * NFQ] = a.gamma1 / hD * etaD * fw;
          cp[(o++) * NFQ] = a.gamma2 / hD * fw;
          cp[(o++) * NFQ] = etaD * fw;
          cp[(o++) * NFQ] = betaD * fw;
#pragma unroll
          for (int i = 0; i < NS; ++i) cp[(o++) * NFQ] = Dg[i];
          cp[(o++) * NFQ] = fw;
          (void)isD;
          (void)pf;
          return;
        } else {
          // residual, F = RHS - LHS
          const T fwt = (T)fw;
          const T un = nsg * u[ax];
#pragma unroll
          for (int c = 0; c < NC; ++c) V[c] = -un * u[c] * fwt;
          if (isD) {
            T A[3][3];
            T a2 = 0;
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
              for (int j = 0; j < DIM; ++j) {
                A[i][j] = (T)0.5 * (g[i][j] + g[j][i]);
                a2 += A[i][j] * A[i][j];
              }
            const T eta = (T)a.nu_inf + (T)a.nu * pow((T)(a.delta * a.delta) + a2, (T)(0.5 * (a.p - 2.0)));
            const T gn = nsg * (T)gl[ax];
            const T negu = (T)0.5 * (fabs(un) - un), negg = (T)0.5 * (fabs(gn) - gn);
            T dlt[3] = {0, 0, 0};
#pragma unroll
            for (int c = 0; c < NC; ++c) dlt[c] = u[c] - (T)gl[c];
            const T dn = nsg * dlt[ax];
            const T p1 = (T)(a.gamma1 / hD * etaD), p2 = (T)(a.gamma2 / hD);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              const T Sn = nsg * eta * A[c][ax];
              V[c] += (Sn - (c == ax ? nsg * pf : (T)0) + negu * u[c] - negg * (T)gl[c] - p1 * dlt[c] -
                       (c == ax ? p2 * dn * nsg : (T)0)) * fwt;
            }
            T Sd[3][3];
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
              for (int j = 0; j < DIM; ++j)
                Sd[i][j] = (T)0.5 * ((j == ax ? nsg * dlt[i] : (T)0) + (i == ax ? nsg * dlt[j] : (T)0));
            T gS = 0;
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
              for (int j = 0; j < DIM; ++j) gS += (T)Dgf[i][j] * Sd[i][j];
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
              for (int j = 0; j < DIM; ++j)
                Gf[i][j] = ((T)etaD * Sd[i][j] + (T)betaD * gS * (T)Dgf[i][j]) * fwt;
            Qf = -(T)a.q_sign * dn * fwt;
          }
        }
      } else {  // OP_JAC
        const T* cp = reinterpret_cast<const T*>(a.fcache) + (((long)fid * K1 + mu) * (long)D::NF_FACE) * NFQ + fq;
        constexpr int oU = 2 + NS, oN = oU + NC;
        T uw[3] = {0, 0, 0};
#pragma unroll
        for (int c = 0; c < NC; ++c) uw[c] = cp[(oU + c) * NFQ];
        const T unw = nsg * uw[ax];
        const T dun = nsg * u[ax];
#pragma unroll
        for (int c = 0; c < NC; ++c) V[c] = unw * u[c] + (TAN == 1 ? dun * uw[c] : (T)0);
        if (isD) {
          const T etaw = cp[0], cw = cp[NFQ];
          T Am[NS];
#pragma unroll
          for (int i = 0; i < NS; ++i) Am[i] = cp[(2 + i) * NFQ];
          const T negw = cp[oN * NFQ], pen1 = cp[(oN + 1) * NFQ], pen2 = cp[(oN + 2) * NFQ];
          const T etaDw = cp[(oN + 3) * NFQ], betaDw = cp[(oN + 4) * NFQ];
          T Dg[NS];
#pragma unroll
          for (int i = 0; i < NS; ++i) Dg[i] = cp[(oN + 5 + i) * NFQ];
          const T fwt = cp[(oN + 5 + NS) * NFQ];
          T Bm[3][3];
#pragma unroll
          for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) Bm[i][j] = (T)0.5 * (g[i][j] + g[j][i]);
          T AB = 0;
          if (TAN == 1) {
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
              for (int j = 0; j < DIM; ++j) AB += Am[sym_idx<DIM>(i, j)] * Bm[i][j];
          }
          const T sfac = cw * AB;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const T Tn = nsg * (etaw * Bm[c][ax] + (TAN == 1 ? sfac * Am[sym_idx<DIM>(c, ax)] : (T)0));
            V[c] += -Tn - negw * u[c] + pen1 * u[c];
          }
          V[ax] += nsg * (pf * fwt) + pen2 * dun * nsg;
          // -(du, DS(Dg)(Dz) n) = -DS(Dg)(sym(du (x) n)) : grad z
          T Sd[3][3];
#pragma unroll
          for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j)
              Sd[i][j] = (T)0.5 * ((j == ax ? nsg * u[i] : (T)0) + (i == ax ? nsg * u[j] : (T)0));
          T gS = 0;
#pragma unroll
          for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) gS += Dg[sym_idx<DIM>(i, j)] * Sd[i][j];
#pragma unroll
          for (int i = 0; i < DIM; ++i)
#pragma unroll
            for (int j = 0; j < DIM; ++j) Gf[i][j] = -(etaDw * Sd[i][j] + betaDw * gS * Dg[sym_idx<DIM>(i, j)]);
          Qf = (T)a.q_sign * dun * fwt;
        }
      }
      if constexpr (MODE != OP_LIN) {
        // fluxes in place: FV <- PV, FGn <- PN, FGt <- PT
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          w[Cfg::oPV + c * NFQ + fq] = V[c];
          w[Cfg::oPN + c * NFQ + fq] = Gf[c][ax];
          w[Cfg::oPT + (c * (DIM - 1) + 0) * NFQ + fq] = Gf[c][t1];
          if (DIM == 3) w[Cfg::oPT + (c * (DIM - 1) + 1) * NFQ + fq] = Gf[c][t2];
        }
        w[Cfg::oFQ + fq] = Qf;
      }
}

template <int DIM, int K1, typename T, int MODE, int TAN>
__global__ void __launch_bounds__(OP_THREADS) st_face_kernel(const OpArgs a, const int* __restrict__ face_cell,
                                                             const unsigned char* __restrict__ face_side,
                                                             long nslots, T* __restrict__ fscr) {
  using D = Dims<DIM>;
  using Cfg = FaceCfg<DIM, T>;
  constexpr int NC = D::NC, NFQ = D::NFQ, NFP = D::NFP;
  constexpr int FS = Cfg::FS, PS = Cfg::per_slot;
  constexpr int FL = (DIM == 3) ? 3 : 1;  // lines per tangential direction of a face plane
  constexpr int NOUT = 2 * NC * NFQ + NFP;  // compact face output per slot
  const auto& ct = CT<T>::t();

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sW = reinterpret_cast<T*>(smem_raw);
  int* sCellL = reinterpret_cast<int*>(sW + FS * PS);  // linear cell id
  int* sSide = sCellL + FS;
  int* sFid = sSide + FS;
  int* sMu = sFid + FS;
  long* sB2 = reinterpret_cast<long*>((reinterpret_cast<uintptr_t>(sMu + FS) + 7) & ~(uintptr_t)7);
  long* sB1 = sB2 + FS;
  __shared__ T sDd[3][9], sDdt[3][9];

  const T* in = reinterpret_cast<const T*>(a.in);
  if (threadIdx.x < 27) {
    const int d = threadIdx.x / 9, e = threadIdx.x % 9;
    sDd[d][e] = (T)a.Dd[d][e];
    sDdt[d][e] = (T)a.Ddt[d][e];
  }
  for (long base = (long)blockIdx.x * FS; base < nslots; base += (long)gridDim.x * FS) {
    const int nfs = (int)min((long)FS, nslots - base);
    // ---- face slot metadata: slot = face * (k+1) + mu
    for (int f = threadIdx.x; f < nfs; f += blockDim.x) {
      const long slot = base + f;
      const int face = (int)(slot / K1);
      sFid[f] = face;
      sMu[f] = (int)(slot % K1);
      const int cell = face_cell[face];
      sCellL[f] = cell;
      sSide[f] = face_side[face];
      const long ex = cell % a.n[0], ey = (cell / a.n[0]) % a.n[1], ez = (DIM == 3) ? cell / (a.n[0] * a.n[1]) : 0;
      sB2[f] = 2 * ex + a.g2[0] * (2 * ey + a.g2[1] * 2 * ez);
      sB1[f] = ex + a.g1[0] * (ey + a.g1[1] * ez);
    }
    __syncthreads();

    // ---- FA: face-plane nodal values and normal derivatives; face pressure nodes
    for (int it = threadIdx.x; it < nfs * (NC * NFQ + NFP); it += blockDim.x) {
      const int f = it / (NC * NFQ + NFP), r = it % (NC * NFQ + NFP);
      const int side = sSide[f], ax = side >> 1, up = side & 1, mu = sMu[f];
      const int cell = sCellL[f];
      const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
      T* w = sW + f * PS;
      if (r < NC * NFQ) {
        const int c = r / NFQ, tn = r % NFQ;
        const int p1 = tn % 3, p2 = (DIM == 3) ? tn / 3 : 0;
        T v[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const int px = ax == 0 ? i : (t1 == 0 ? p1 : 0);
          const int py = ax == 1 ? i : (t1 == 1 ? p1 : (t2 == 1 ? p2 : 0));
          const int pz = ax == 2 ? i : (t2 == 2 ? p2 : 0);
          const long gn = sB2[f] + px + a.g2[0] * (py + a.g2[1] * pz);
          v[i] = in[(long)mu * a.Mv + c * a.Nq2 + gn];
        }
        w[Cfg::oPV + c * NFQ + tn] = up ? v[2] : v[0];
        w[Cfg::oPN + c * NFQ + tn] =
            ((T)ct.ED[up * 3 + 0] * v[0] + (T)ct.ED[up * 3 + 1] * v[1] + (T)ct.ED[up * 3 + 2] * v[2]) * (T)a.ih[ax];
      } else {
        const int m = r - NC * NFQ;
        const int q1 = m & 1, q2 = (DIM == 3) ? (m >> 1) : 0;
        const int mx = ax == 0 ? up : (t1 == 0 ? q1 : 0);
        const int my = ax == 1 ? up : (t1 == 1 ? q1 : (t2 == 1 ? q2 : 0));
        const int mz = ax == 2 ? up : (t2 == 2 ? q2 : 0);
        if (a.pdisc) {
          // P1disc: the cell's affine pressure at this face vertex (pdisc_T)
          const int mc = mx + 2 * my + 4 * mz;
          const T* pc = in + (long)K1 * a.Mv + (long)mu * a.Mp + (long)cell * (DIM + 1);
          T v = pc[0];
#pragma unroll
          for (int j = 1; j <= DIM; ++j) v += ((mc >> (j - 1)) & 1) ? pc[j] : -pc[j];
          w[Cfg::oFP + m] = v;
        } else {
          const long gp = sB1[f] + mx + a.g1[0] * (my + a.g1[1] * mz);
          w[Cfg::oFP + m] = in[(long)K1 * a.Mv + (long)mu * a.Mp + gp];
        }
      }
    }
    __syncthreads();
    // ---- FB: values at the face points (tangential passes on PV and PN)
    for (int td = 0; td < DIM - 1; ++td) {
      for (int it = threadIdx.x; it < nfs * NC * 2 * FL; it += blockDim.x) {
        const int f = it / (NC * 2 * FL), c = (it / (2 * FL)) % NC, wh = (it / FL) % 2, l = it % FL;
        T* x = sW + f * PS + (wh ? Cfg::oPN : Cfg::oPV) + c * NFQ;
        const int b = (td == 0) ? 3 * l : l, st = (td == 0) ? 1 : 3;
        T y0, y1, y2;
        apply3<T, T>(ct.B, x[b], x[b + st], x[b + 2 * st], y0, y1, y2);
        x[b] = y0;
        x[b + st] = y1;
        x[b + 2 * st] = y2;
      }
      __syncthreads();
    }
    // ---- FC: tangential derivatives at the face points (collocation form)
    for (int it = threadIdx.x; it < nfs * NC * (DIM - 1) * FL; it += blockDim.x) {
      const int f = it / (NC * (DIM - 1) * FL), c = (it / ((DIM - 1) * FL)) % NC, td = (it / FL) % (DIM - 1),
                l = it % FL;
      const int ax = sSide[f] >> 1;
      const int tax = (td == 0) ? (ax == 0 ? 1 : 0) : (ax == 2 ? 1 : 2);
      const T* x = sW + f * PS + Cfg::oPV + c * NFQ;
      T* y = sW + f * PS + Cfg::oPT + (c * (DIM - 1) + td) * NFQ;
      const int b = (td == 0) ? 3 * l : l, st = (td == 0) ? 1 : 3;
      T y0, y1, y2;
      apply3<T, T>(sDd[tax], x[b], x[b + st], x[b + 2 * st], y0, y1, y2);
      y[b] = y0;
      y[b + st] = y1;
      y[b + 2 * st] = y2;
    }
    __syncthreads();
    // ---- FD: pointwise face terms (dispatched on the face axis)
    for (int it = threadIdx.x; it < nfs * NFQ; it += blockDim.x) {
      const int f = it / NFQ, fq = it % NFQ;
      const int side = sSide[f], ax = side >> 1;
      T* w = sW + f * PS;
      if (ax == 0) face_point<DIM, K1, T, MODE, TAN, 0>(a, w, fq, side, sMu[f], sCellL[f], sFid[f]);
      else if (ax == 1) face_point<DIM, K1, T, MODE, TAN, 1>(a, w, fq, side, sMu[f], sCellL[f], sFid[f]);
      else if constexpr (DIM == 3) face_point<DIM, K1, T, MODE, TAN, 2>(a, w, fq, side, sMu[f], sCellL[f], sFid[f]);
    }
    __syncthreads();
    if constexpr (MODE != OP_LIN) {
      // ---- FE1: tangential derivative tests, chained into FV
      for (int td = 0; td < DIM - 1; ++td) {
        for (int it = threadIdx.x; it < nfs * NC * FL; it += blockDim.x) {
          const int f = it / (NC * FL), c = (it / FL) % NC, l = it % FL;
          const int ax = sSide[f] >> 1;
          const int tax = (td == 0) ? (ax == 0 ? 1 : 0) : (ax == 2 ? 1 : 2);
          T* w = sW + f * PS;
          const T* x = w + Cfg::oPT + (c * (DIM - 1) + td) * NFQ;
          T* y = w + Cfg::oPV + c * NFQ;
          const int b = (td == 0) ? 3 * l : l, st = (td == 0) ? 1 : 3;
          const T* m = sDdt[tax];
          const T x0 = x[b], x1 = x[b + st], x2 = x[b + 2 * st];
          y[b] += m[0] * x0 + m[1] * x1 + m[2] * x2;
          y[b + st] += m[3] * x0 + m[4] * x1 + m[5] * x2;
          y[b + 2 * st] += m[6] * x0 + m[7] * x1 + m[8] * x2;
        }
        __syncthreads();
      }
      // ---- FE2: transposed tangential value passes on FV and FGn
      for (int td = 0; td < DIM - 1; ++td) {
        for (int it = threadIdx.x; it < nfs * NC * 2 * FL; it += blockDim.x) {
          const int f = it / (NC * 2 * FL), c = (it / (2 * FL)) % NC, wh = (it / FL) % 2, l = it % FL;
          T* x = sW + f * PS + (wh ? Cfg::oPN : Cfg::oPV) + c * NFQ;
          const int b = (td == 0) ? 3 * l : l, st = (td == 0) ? 1 : 3;
          T y0, y1, y2;
          apply3<T, T>(ct.Bt, x[b], x[b + st], x[b + 2 * st], y0, y1, y2);
          x[b] = y0;
          x[b + st] = y1;
          x[b + 2 * st] = y2;
        }
        __syncthreads();
      }
      // ---- compact face output: FV and FGn/h at the face-plane nodes, pressure tests
      for (int it = threadIdx.x; it < nfs * NOUT; it += blockDim.x) {
        const int f = it / NOUT, r = it % NOUT;
        const T* w = sW + f * PS;
        T v;
        if (r < NC * NFQ) {
          v = w[Cfg::oPV + r];
        } else if (r < 2 * NC * NFQ) {
          v = w[Cfg::oPN + (r - NC * NFQ)] * (T)a.ih[sSide[f] >> 1];
        } else {
          const int m = r - 2 * NC * NFQ;
          T acc = 0;
#pragma unroll
          for (int fq = 0; fq < NFQ; ++fq)
            acc += ((DIM == 3) ? ct.FPSI3[fq * 4 + m] : ct.FPSI2[fq * 2 + m]) * w[Cfg::oFQ + fq];
          v = acc;
        }
        fscr[(base + f) * NOUT + r] = v;
      }
    }
    __syncthreads();
  }
}

// Adds the boundary-face contributions into out, one thread per node of the
// boundary-cell layer.  The host lists, per such node, every (face, face-node)
// pair that reaches it with the weights E_i and ED_i of the Q2 basis along the
// face normal (velocity) or the face pressure-test index (pressure).  Each
// node is written by exactly one thread (no atomics, deterministic).
struct GatherEnt {
  int fid;    // boundary face
  int tn;     // face-plane node (velocity) or face pressure node (pressure)
  double e;   // weight of the face value output (pressure: of the face pressure test;
              // 1 for Q1, T[m][j] of pdisc_T for P1disc)
  double ed;  // weight of the face normal-derivative output
};

// out = sum of the 2^DIM class-private volume outputs, fixed class order,
// two entries per thread (16-byte loads when the slab length allows it).
template <int DIM, typename T>
__global__ void st_cbuf_sum(const T* __restrict__ cb, long stride, long n, T* __restrict__ out) {
  constexpr int NCOL = 1 << DIM;
  const long n2 = (stride % 2 == 0) ? n / 2 : 0;  // pairs (aligned when the stride is even)
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n2; t += (long)gridDim.x * blockDim.x) {
    T a0 = cb[2 * t], a1 = cb[2 * t + 1];
#pragma unroll
    for (int c = 1; c < NCOL; ++c) {
      a0 += cb[c * stride + 2 * t];
      a1 += cb[c * stride + 2 * t + 1];
    }
    out[2 * t] = a0;
    out[2 * t + 1] = a1;
  }
  for (long i = 2 * n2 + (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    T a = cb[i];
#pragma unroll
    for (int c = 1; c < NCOL; ++c) a += cb[c * stride + i];
    out[i] = a;
  }
}

// out += the boundary-face contributions of the face scratch: one thread per
// (gather row, Radau node, component) of the boundary-cell layer.
template <int DIM, int K1, typename T>
__global__ void st_face_add(const OpArgs a, int nvel, int ntot, const int* __restrict__ gnode,
                            const int* __restrict__ gptr, const GatherEnt* __restrict__ gent,
                            const T* __restrict__ fscr, T* __restrict__ out) {
  using D = Dims<DIM>;
  constexpr int NC = D::NC, NFQ = D::NFQ;
  constexpr int NOUT = 2 * NC * NFQ + D::NFP;
  const long nv = (long)nvel * K1 * NC, np = (long)(ntot - nvel) * K1;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < nv + np; t += (long)gridDim.x * blockDim.x) {
    if (t < nv) {
      const int row = (int)(t / (K1 * NC)), mc = (int)(t % (K1 * NC)), mu = mc / NC, c = mc % NC;
      const int b = gptr[row], e = gptr[row + 1];
      T acc = 0;
      for (int j = b; j < e; ++j) {
        const GatherEnt ge = gent[j];
        const T* fs = fscr + ((long)ge.fid * K1 + mu) * NOUT + ge.tn + c * NFQ;
        acc += (T)ge.e * fs[0] + (T)ge.ed * fs[NC * NFQ];
      }
      out[(long)mu * a.Mv + (long)c * a.Nq2 + gnode[row]] += acc;
    } else {
      const long u = t - nv;
      const int row = nvel + (int)(u / K1), mu = (int)(u % K1);
      const int b = gptr[row], e = gptr[row + 1];
      T acc = 0;
      for (int j = b; j < e; ++j) {
        const GatherEnt ge = gent[j];
        acc += (T)ge.e * fscr[((long)ge.fid * K1 + mu) * NOUT + 2 * NC * NFQ + ge.tn];
      }
      out[(long)K1 * a.Mv + (long)mu * a.Mp + gnode[row]] += acc;
    }
  }
}


// Boundary-face part of the spatial element matrices (added into E): one CTA
// per boundary cell handles all faces of that cell in turn, so no two CTAs add
// into the same matrix.  For every trial dof j the face-point values of the
// trial function are set up, the same pointwise face terms as the Jacobian
// action (face_point, OP_JAC) are evaluated, and the results are integrated
// against every test function of the cell.
template <int DIM, int K1, typename T, int TAN>
__global__ void __launch_bounds__(OP_THREADS) st_face_matrix(const OpArgs a, const int* __restrict__ bcells, int nbc,
                                                             T* __restrict__ E) {
  using D = Dims<DIM>;
  using Cfg = FaceCfg<DIM, T>;
  constexpr int NC = D::NC, NQ = D::NQ, NFQ = D::NFQ, NE = D::NE, NFP = D::NFP, PS = Cfg::per_slot;
  const auto& ct = CT<T>::t();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sW = reinterpret_cast<T*>(smem_raw);  // NE workspaces of PS entries
  __shared__ double sDn[9];                // Q2 basis derivative at the Gauss points, [q][a]
  __shared__ T stab[D::NQ][D::NFQ][4];     // test functions of the face: value, normal and tangential derivatives
  if (threadIdx.x < 9) {
    const int q = threadIdx.x / 3, aa = threadIdx.x % 3;
    double v = 0.0;
    for (int r = 0; r < 3; ++r) v += cT.Dc[q * 3 + r] * cT.B[r * 3 + aa];
    sDn[threadIdx.x] = v;
  }
  __syncthreads();
  const int mu = a.elm_mu;
  for (int b = blockIdx.x; b < nbc; b += gridDim.x) {
    const int cell = bcells[b];
    const int e3[3] = {cell % a.n[0], (cell / a.n[0]) % a.n[1], (DIM == 3) ? cell / (a.n[0] * a.n[1]) : 0};
    int rank = 0;
    for (int side = 0; side < 2 * DIM; ++side) {
      const int ax = side >> 1, up = side & 1;
      const bool on = up ? (e3[ax] == a.n[ax] - 1) : (e3[ax] == 0);
      if (!on) continue;
      const int fid = a.face_off[cell] + rank++;
      const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
      // (1) trial values at the face points
      for (int it = threadIdx.x; it < NE * NFQ; it += blockDim.x) {
        const int j = it / NFQ, fq = it % NFQ;
        T* w = sW + j * PS;
        const int i1 = fq % 3, i2 = (DIM == 3) ? fq / 3 : 0;
        for (int c = 0; c < NC; ++c) {
          w[Cfg::oPV + c * NFQ + fq] = 0;
          w[Cfg::oPN + c * NFQ + fq] = 0;
          for (int td = 0; td < DIM - 1; ++td) w[Cfg::oPT + (c * (DIM - 1) + td) * NFQ + fq] = 0;
        }
        if (fq == 0)
          for (int m = 0; m < NFP; ++m) w[Cfg::oFP + m] = 0;
        if (j < NC * NQ) {
          const int c = j / NQ, n = j % NQ;
          const int nn[3] = {n % 3, (n / 3) % 3, (DIM == 3) ? n / 9 : 0};
          const double en = cT.E[up * 3 + nn[ax]], edn = cT.ED[up * 3 + nn[ax]] * a.ih[ax];
          const double b1 = cT.B[i1 * 3 + nn[t1]], d1 = sDn[i1 * 3 + nn[t1]] * a.ih[t1];
          const double b2 = (DIM == 3) ? cT.B[i2 * 3 + nn[t2]] : 1.0;
          const double d2 = (DIM == 3) ? sDn[i2 * 3 + nn[t2]] * a.ih[t2] : 0.0;
          w[Cfg::oPV + c * NFQ + fq] = (T)(en * b1 * b2);
          w[Cfg::oPN + c * NFQ + fq] = (T)(edn * b1 * b2);
          w[Cfg::oPT + (c * (DIM - 1) + 0) * NFQ + fq] = (T)(en * d1 * b2);
          if (DIM == 3) w[Cfg::oPT + (c * (DIM - 1) + 1) * NFQ + fq] = (T)(en * b1 * d2);
        } else if (fq == 0) {
          const int m = j - NC * NQ;  // trial pressure node; on the face?
          const int mm[3] = {m & 1, (m >> 1) & 1, (DIM == 3) ? (m >> 2) : 0};
          if (mm[ax] == up) w[Cfg::oFP + (mm[t1] + 2 * ((DIM == 3) ? mm[t2] : 0))] = 1;
        }
      }
      __syncthreads();
      // (2) pointwise face terms, fluxes in place
      for (int it = threadIdx.x; it < NE * NFQ; it += blockDim.x) {
        const int j = it / NFQ, fq = it % NFQ;
        T* w = sW + j * PS;
        if (ax == 0) face_point<DIM, K1, T, OP_JAC, TAN, 0>(a, w, fq, side, mu, cell, fid);
        else if (ax == 1) face_point<DIM, K1, T, OP_JAC, TAN, 1>(a, w, fq, side, mu, cell, fid);
        else if constexpr (DIM == 3) face_point<DIM, K1, T, OP_JAC, TAN, 2>(a, w, fq, side, mu, cell, fid);
      }
      __syncthreads();
      // test-function values and derivatives at the face points (all velocity nodes of the cell)
      for (int it = threadIdx.x; it < NQ * NFQ; it += blockDim.x) {
        const int n = it / NFQ, fq = it % NFQ;
        const int nn[3] = {n % 3, (n / 3) % 3, (DIM == 3) ? n / 9 : 0};
        const int i1 = fq % 3, i2 = (DIM == 3) ? fq / 3 : 0;
        const double en = cT.E[up * 3 + nn[ax]], edn = cT.ED[up * 3 + nn[ax]] * a.ih[ax];
        const double b1 = cT.B[i1 * 3 + nn[t1]], d1 = sDn[i1 * 3 + nn[t1]] * a.ih[t1];
        const double b2 = (DIM == 3) ? cT.B[i2 * 3 + nn[t2]] : 1.0;
        const double d2 = (DIM == 3) ? sDn[i2 * 3 + nn[t2]] * a.ih[t2] : 0.0;
        stab[n][fq][0] = (T)(en * b1 * b2);
        stab[n][fq][1] = (T)(edn * b1 * b2);
        stab[n][fq][2] = (T)(en * d1 * b2);
        stab[n][fq][3] = (T)(en * b1 * d2);
      }
      __syncthreads();
      // (3) integrate against every test function: E[i][j] += ...
      T* Ec = E + ((long)cell * a.elm_stride + a.elm_slot) * NE * NE;
      for (int it = threadIdx.x; it < NE * NE; it += blockDim.x) {
        const int i = it / NE, j = it % NE;
        const T* w = sW + j * PS;
        T acc = 0;
        if (i < NC * NQ) {
          const int c = i / NQ, n = i % NQ;
          const int nn[3] = {n % 3, (n / 3) % 3, (DIM == 3) ? n / 9 : 0};
          const double en = cT.E[up * 3 + nn[ax]], edn = cT.ED[up * 3 + nn[ax]] * a.ih[ax];
          if (en == 0.0 && edn == 0.0) continue;
          for (int fq = 0; fq < NFQ; ++fq) {
            const T* tb = stab[n][fq];
            acc += w[Cfg::oPV + c * NFQ + fq] * tb[0] + w[Cfg::oPN + c * NFQ + fq] * tb[1] +
                   w[Cfg::oPT + (c * (DIM - 1) + 0) * NFQ + fq] * tb[2];
            if (DIM == 3) acc += w[Cfg::oPT + (c * (DIM - 1) + 1) * NFQ + fq] * tb[3];
          }
        } else {
          const int m = i - NC * NQ;
          const int mm[3] = {m & 1, (m >> 1) & 1, (DIM == 3) ? (m >> 2) : 0};
          if (mm[ax] != up) continue;
          const int mf = mm[t1] + 2 * ((DIM == 3) ? mm[t2] : 0);
          for (int fq = 0; fq < NFQ; ++fq)
            acc += ((DIM == 3) ? ct.FPSI3[fq * 4 + mf] : ct.FPSI2[fq * 2 + mf]) * w[Cfg::oFQ + fq];
        }
        Ec[(long)i * NE + j] += acc;
      }
      __syncthreads();
    }
  }
}

}  // namespace st
