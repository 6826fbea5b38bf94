// Hexahedral elements of the general-mesh path: the FR / hybridized-FR residual and the element
// blocks in three dimensions (Pereira & Vermeire, arXiv 2401.16632: the scheme of Secs. 2-4, run
// on hexahedra in Sec. 5.3; compressible Navier-Stokes with u = (rho, rho v, E)).
//
// The 2D operators in tensor product: solution point pt = a + n b + n^2 c; face f has normal axis
// r = f / 2 and side sigma (f odd: +1); face point m = i + n j along the lower then the higher
// tangential axis; the line of solution points through face point m along r is
//     r = 0: s + n i + n^2 j,   r = 1: i + n s + n^2 j,   r = 2: i + n j + n^2 s   (s = 0..n-1).
// With the 1D lift l_s(+-1)/w_s of the DG-recovering corrections folded into
// M = D - dgL lm^T - dgR lp^T (as in two dimensions):
//     Q_r(pt) = sum_s M[a_r][s] U(line) + dgL[a_r] u_bar(face 2r) + dgR[a_r] u_bar(face 2r+1)
//     q_c     = (1/J) sum_r S[r][c] Q_r,            S[r] = x_{xi_s} x x_{xi_t} (cyclic (r, s, t))
//     R       = -(1/J) sum_r [sum_s M[a_r][s] F~_r(line) - dgL[a_r] Fn(2r) + dgR[a_r] Fn(2r+1)]
// where a_r is the point's index along r and Fn = J_f F^.n the common normal flux at the face
// point met by the point's r-line.  Face kinds, common fluxes, trace rows and the viscous readings
// are those of the quadrilateral path (one degree: face points are the element's face nodes).
//
// Element blocks are formed column by column (one warp per seed point, dense tangents through the
// linear chain of the operator) and stored column-major, so that a warp writes its column as one
// contiguous run; the pointwise Jacobians of a CTA's element live in a global slab of that CTA
// (43 200 values for p = 3: too large for shared memory next to the column buffers).
#include <math.h>
#include <string.h>

#include "hfr_general_internal.h"

namespace hfr {
namespace gen {

constexpr int HN = HEX_PMAX + 1;       // points per line (at most)
constexpr int HNS = HN * HN * HN;      // solution points
constexpr int HNF = HN * HN;           // points per face
constexpr int HFP = 6 * HNF;           // face points per element
constexpr int HNV = 5;
constexpr int HT = 128;                // threads of the residual kernel (one CTA per element)
constexpr int HJT = 256, HJW = HJT / 32;  // block kernel

// Navier-Stokes in three dimensions (ideal gas, R = 1, constant mu, Stokes hypothesis,
// kappa = mu gamma / ((gamma - 1) Pr)); F[c][v], q[c][v] = du_v / dx_c
struct NS3 {
  template <typename S, typename R>
  __device__ static void conv(const PhysConst<R>& pc, const S* u, S F[3][HNV]) {
    const S ir = R(1) / u[0];
    const S v0 = u[1] * ir, v1 = u[2] * ir, v2 = u[3] * ir;
    const S p = pc.gm1 * (u[4] - R(0.5) * (u[1] * v0 + u[2] * v1 + u[3] * v2));
    const S v[3] = {v0, v1, v2};
    const S Ep = u[4] + p;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      F[c][0] = u[1 + c];
#pragma unroll
      for (int k = 0; k < 3; ++k) F[c][1 + k] = u[1 + k] * v[c] + (k == c ? p : S(R(0)));
      F[c][4] = Ep * v[c];
    }
  }
  template <typename S, typename R>
  __device__ static void visc(const PhysConst<R>& pc, const S* u, const S q[3][HNV], S F[3][HNV]) {
    const R mu = pc.mu;
    const S ir = R(1) / u[0];
    const S v[3] = {u[1] * ir, u[2] * ir, u[3] * ir};
    const S e = u[4] * ir;
    S dv[3][3], dT[3];  // dv[c][k] = d v_k / d x_c
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int k = 0; k < 3; ++k) dv[c][k] = (q[c][1 + k] - v[k] * q[c][0]) * ir;
      dT[c] = pc.gm1 * ((q[c][4] - e * q[c][0]) * ir - (v[0] * dv[c][0] + v[1] * dv[c][1] + v[2] * dv[c][2]));
    }
    const S div = dv[0][0] + dv[1][1] + dv[2][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      F[c][0] = S(R(0));
#pragma unroll
      for (int k = 0; k < 3; ++k) F[c][1 + k] = mu * (dv[c][k] + dv[k][c] - (k == c ? R(2.0 / 3.0) * div : S(R(0))));
      F[c][4] = v[0] * F[c][1] + v[1] * F[c][2] + v[2] * F[c][3] + pc.kappa * dT[c];
    }
  }
  template <typename S, typename R>
  __device__ static S wave(const PhysConst<R>& pc, const S* u, const R* n) {
    const S ir = R(1) / u[0];
    const S v0 = u[1] * ir, v1 = u[2] * ir, v2 = u[3] * ir;
    const S p = pc.gm1 * (u[4] - R(0.5) * (u[1] * v0 + u[2] * v1 + u[3] * v2));
    return dabs(v0 * n[0] + v1 * n[1] + v2 * n[2]) + dsqrt(pc.gamma * p * ir);
  }
  template <typename S, typename R>
  __device__ static S stab(const PhysConst<R>& pc, const S* u, const R* n) {
    return wave<S, R>(pc, u, n) + pc.mu_lref / u[0];
  }
};

// common normal flux J_f F^.n and the trace row of one face point (as gface_flux in 2D)
template <typename S, typename R>
__device__ __forceinline__ void hface_flux(const PhysConst<R>& pc, bool visc, int kf, bool traced, bool imp,
                                           const S* uf, const S* ub, const S (&qf)[3][HNV], const S* un,
                                           const S (&qn)[3][HNV], R Jf, const R* nr, const R* uinf, S* Fn, S* row) {
  S F[3][HNV];
  if (traced) {
    S Fh[HNV];
    NS3::conv<S, R>(pc, ub, F);
    const S s = NS3::stab<S, R>(pc, ub, nr);
#pragma unroll
    for (int v = 0; v < HNV; ++v) Fh[v] = nr[0] * F[0][v] + nr[1] * F[1][v] + nr[2] * F[2][v] + s * (uf[v] - ub[v]);
    if (visc) {
      NS3::visc<S, R>(pc, ub, qf, F);
#pragma unroll
      for (int v = 0; v < HNV; ++v) Fh[v] = Fh[v] - (nr[0] * F[0][v] + nr[1] * F[1][v] + nr[2] * F[2][v]);
    }
#pragma unroll
    for (int v = 0; v < HNV; ++v) Fn[v] = Jf * Fh[v];
    if (kf == FK_FAR) {
#pragma unroll
      for (int v = 0; v < HNV; ++v) row[v] = Jf * s * ((uf[v] - ub[v]) + (uinf[v] - ub[v]));
    } else if (kf == FK_WALL) {
#pragma unroll
      for (int v = 0; v < HNV; ++v) row[v] = (v == 0 || v == HNV - 1) ? Jf * Fh[v] : Jf * s * ub[v];
    } else {
#pragma unroll
      for (int v = 0; v < HNV; ++v) row[v] = Jf * Fh[v];
    }
    return;
  }
  S G[3][HNV];
  NS3::conv<S, R>(pc, uf, F);
  NS3::conv<S, R>(pc, un, G);
  const S lam = dmax(NS3::wave<S, R>(pc, uf, nr), NS3::wave<S, R>(pc, un, nr));
  S Fh[HNV];
#pragma unroll
  for (int v = 0; v < HNV; ++v)
    Fh[v] = R(0.5) * (nr[0] * (F[0][v] + G[0][v]) + nr[1] * (F[1][v] + G[1][v]) + nr[2] * (F[2][v] + G[2][v])) +
            R(0.5) * lam * (uf[v] - un[v]);
  if (visc) {
    if (kf == FK_FR || kf == FK_FAR) {
      NS3::visc<S, R>(pc, uf, qf, F);
      NS3::visc<S, R>(pc, un, qn, G);
#pragma unroll
      for (int v = 0; v < HNV; ++v)
        Fh[v] = Fh[v] - R(0.5) * (nr[0] * (F[0][v] + G[0][v]) + nr[1] * (F[1][v] + G[1][v]) + nr[2] * (F[2][v] + G[2][v]));
    } else {
      if (imp)
        NS3::visc<S, R>(pc, uf, qf, F);
      else
        NS3::visc<S, R>(pc, un, qn, F);
#pragma unroll
      for (int v = 0; v < HNV; ++v) Fh[v] = Fh[v] - (nr[0] * F[0][v] + nr[1] * F[1][v] + nr[2] * F[2][v]);
    }
  }
#pragma unroll
  for (int v = 0; v < HNV; ++v) {
    Fn[v] = Jf * Fh[v];
    row[v] = S(R(0));
  }
}

// solution point on the r-line through face point m at coordinate s
__device__ __forceinline__ int hline(int r, int m, int s, int n) {
  const int i = m % n, j = m / n;
  return r == 0 ? s + n * i + n * n * j : (r == 1 ? i + n * s + n * n * j : i + n * j + n * n * s);
}
// a point's index along axis r and the face point of its r-line
__device__ __forceinline__ int hcoord(int pt, int r, int n) { return r == 0 ? pt % n : (r == 1 ? (pt / n) % n : pt / (n * n)); }
__device__ __forceinline__ int hfacept(int pt, int r, int n) {
  const int a = pt % n, b = (pt / n) % n, c = pt / (n * n);
  return r == 0 ? b + n * c : (r == 1 ? a + n * c : a + n * b);
}

// ------------------------------------------------------------------------ residual passes
struct HWork {
  double U[HNS][HNV];
  double Uf[HFP][HNV], ub[HFP][HNV];
  double q[HNS][3][HNV];
  double qf[HFP][3][HNV];
  double Ft[HNS][3][HNV];
  double Fn[HFP][HNV];
  double M[HN][HN], lm[HN], lp[HN], dgL[HN], dgR[HN], w[HN];
  int kf[6], tr[6];
};
static_assert(sizeof(HWork) <= 227 * 1024, "hexahedral residual workspace exceeds shared memory");

template <int MODE>
__global__ void __launch_bounds__(HT) k_hex_elem(const __grid_constant__ PhysParams pp, const __grid_constant__ GArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  HWork& w = *reinterpret_cast<HWork*>(smem_raw);
  if ((int)blockIdx.x >= (a.elist ? a.nlist : a.E)) return;
  const int e = a.elist ? a.elist[blockIdx.x] : (int)blockIdx.x;
  const int tid = threadIdx.x;
  const int n = a.deg[e], ns = n * n * n, nf = n * n, FS = a.fs;
  const GenRef& RF = *a.ref;
  const bool visc = phys_viscous(pp);
  const PhysConst<double> pc = phys_const<double>(pp);
  const bool imp = a.implicit[e] != 0;
  for (int i = tid; i < n * n; i += HT) w.M[i / n][i % n] = RF.M[n][i / n][i % n];
  if (tid < n) {
    w.lm[tid] = RF.lm[n][tid];
    w.lp[tid] = RF.lp[n][tid];
    w.dgL[tid] = RF.dgL[n][tid];
    w.dgR[tid] = RF.dgR[n][tid];
    w.w[tid] = RF.w[n][tid];
  }
  if (tid < 6) {
    w.kf[tid] = a.kind[6 * e + tid];
    w.tr[tid] = a.tr_of[6 * e + tid];
  }
  const double* Ue = a.U + a.uoff[e];
  for (int i = tid; i < ns * HNV; i += HT) w.U[i / HNV][i % HNV] = Ue[i];
  __syncthreads();
  // face values
  for (int it = tid; it < 6 * nf * HNV; it += HT) {
    const int f = it / (nf * HNV), m = (it / HNV) % nf, v = it % HNV, r = f >> 1;
    const double* l = (f & 1) ? w.lp : w.lm;
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += l[c] * w.U[hline(r, m, c, n)][v];
    w.Uf[f * nf + m][v] = s;
    if (MODE == GM_UF) a.Uf_out[((size_t)(6 * e + f) * FS + m) * HNV + v] = s;
  }
  if (MODE == GM_UF) return;
  __syncthreads();
  for (int it = tid; it < 6 * nf * HNV; it += HT) {
    const int f = it / (nf * HNV), m = (it / HNV) % nf, v = it % HNV;
    const int kf = w.kf[f], t = w.tr[f];
    const double uf = w.Uf[f * nf + m][v];
    double ub;
    if (t >= 0) {
      ub = a.uhat[(size_t)FR_IDX(a.fnode[(6 * e + f) * FS + m], a.npts, 10) * HNV + v];
    } else if (kf == FK_FAR) {
      ub = 0.5 * (uf + a.uinf[v]);
    } else {
      const int nb = (int)FR_IDX(a.nbr[6 * e + f], a.E, 11), fn = (int)FR_IDX(a.nbr_face[6 * e + f], 6, 12);
      const double un = a.Uf_all[((size_t)(6 * nb + fn) * FS + m) * HNV + v];
      ub = kf == FK_FR ? 0.5 * (uf + un) : (imp ? un : uf);
    }
    w.ub[f * nf + m][v] = ub;
  }
  __syncthreads();
  const double* gs = a.geo_sol + (size_t)a.goff[e] * 10;
  if (visc) {
    for (int it = tid; it < ns * HNV; it += HT) {
      const int i = it / HNV, v = it % HNV;
      double Q[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int ar = hcoord(i, r, n), m = hfacept(i, r, n);
        double s = w.dgL[ar] * w.ub[(2 * r) * nf + m][v] + w.dgR[ar] * w.ub[(2 * r + 1) * nf + m][v];
        for (int c = 0; c < n; ++c) s += w.M[ar][c] * w.U[hline(r, m, c, n)][v];
        Q[r] = s;
      }
      const double* G = gs + i * 10;
#pragma unroll
      for (int c = 0; c < 3; ++c) w.q[i][c][v] = G[0] * (G[1 + c] * Q[0] + G[4 + c] * Q[1] + G[7 + c] * Q[2]);
    }
    __syncthreads();
    for (int it = tid; it < 6 * nf * 3 * HNV; it += HT) {
      const int f = it / (nf * 3 * HNV), m = (it / (3 * HNV)) % nf, c2 = (it / HNV) % 3, v = it % HNV, r = f >> 1;
      const double* l = (f & 1) ? w.lp : w.lm;
      double s = 0.0;
      for (int c = 0; c < n; ++c) s += l[c] * w.q[hline(r, m, c, n)][c2][v];
      w.qf[f * nf + m][c2][v] = s;
      if (MODE == GM_QF) a.qf_out[(((size_t)(6 * e + f) * FS + m) * 3 + c2) * HNV + v] = s;
    }
  } else if (MODE == GM_QF) {
    for (int it = tid; it < 6 * FS * 3 * HNV; it += HT) a.qf_out[(size_t)(6 * e) * FS * 3 * HNV + it] = 0.0;
  }
  if (MODE == GM_QF) return;
  __syncthreads();
  for (int i = tid; i < ns; i += HT) {
    const double* G = gs + i * 10;
    double F[3][HNV];
    NS3::conv<double, double>(pc, w.U[i], F);
    if (visc) {
      double Fv[3][HNV];
      NS3::visc<double, double>(pc, w.U[i], w.q[i], Fv);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int v = 0; v < HNV; ++v) F[c][v] -= Fv[c][v];
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int v = 0; v < HNV; ++v) w.Ft[i][r][v] = G[1 + 3 * r] * F[0][v] + G[2 + 3 * r] * F[1][v] + G[3 + 3 * r] * F[2][v];
  }
  for (int jj = tid; jj < 6 * nf; jj += HT) {
    const int f = jj / nf, m = jj % nf;
    const int kf = w.kf[f];
    const bool traced = w.tr[f] >= 0;
    const double* G = a.geo_face + ((size_t)(6 * e + f) * FS + m) * 4;
    double un[HNV], qn[3][HNV], qf[3][HNV], Fn[HNV], row[HNV];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int v = 0; v < HNV; ++v) qf[c][v] = visc ? w.qf[jj][c][v] : 0.0;
    if (!traced && kf != FK_FAR) {
      const int nb = (int)FR_IDX(a.nbr[6 * e + f], a.E, 11), fn = (int)FR_IDX(a.nbr_face[6 * e + f], 6, 12);
      const size_t nix = (size_t)(6 * nb + fn) * FS + m;
#pragma unroll
      for (int v = 0; v < HNV; ++v) {
        un[v] = a.Uf_all[nix * HNV + v];
#pragma unroll
        for (int c = 0; c < 3; ++c) qn[c][v] = visc ? a.qf_all[(nix * 3 + c) * HNV + v] : 0.0;
      }
    } else {
#pragma unroll
      for (int v = 0; v < HNV; ++v) {
        un[v] = a.uinf[v];
#pragma unroll
        for (int c = 0; c < 3; ++c) qn[c][v] = qf[c][v];
      }
    }
    const double nr[3] = {G[1], G[2], G[3]};
    hface_flux<double, double>(pc, visc, kf, traced, imp, w.Uf[jj], w.ub[jj], qf, un, qn, G[0], nr, a.uinf, Fn, row);
#pragma unroll
    for (int v = 0; v < HNV; ++v) w.Fn[jj][v] = Fn[v];
    if (a.gview) {
      const double wq = traced ? w.w[m % n] * w.w[m / n] : 0.0;
#pragma unroll
      for (int v = 0; v < HNV; ++v) a.gview[((size_t)(6 * e + f) * FS + m) * HNV + v] = wq * row[v];
    }
  }
  __syncthreads();
  for (int it = tid; it < ns * HNV; it += HT) {
    const int i = it / HNV, v = it % HNV;
    double d = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int ar = hcoord(i, r, n), m = hfacept(i, r, n);
      d += -w.dgL[ar] * w.Fn[(2 * r) * nf + m][v] + w.dgR[ar] * w.Fn[(2 * r + 1) * nf + m][v];
      for (int c = 0; c < n; ++c) d += w.M[ar][c] * w.Ft[hline(r, m, c, n)][r][v];
    }
    if (a.R) a.R[a.uoff[e] + it] = -gs[i * 10] * d;
  }
}

cudaError_t hex_elem_pass(GenCtx* g, const GArgs& a, int mode) {
  const size_t smem = sizeof(HWork);
  cudaError_t e;
  auto kern = mode == GM_UF ? k_hex_elem<GM_UF> : (mode == GM_QF ? k_hex_elem<GM_QF> : k_hex_elem<GM_RES>);
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
  const int cnt = a.elist ? a.nlist : a.E;
  if (cnt == 0) return cudaSuccess;
  (count_launch(), kern<<<cnt, HT, smem, g->st>>>(g->pp, a));
  return cudaGetLastError();
}

// ------------------------------------------------------------------------ element blocks
template <typename T>
struct HJWork {
  T U[HNS][HNV];
  T Uf[HFP][HNV], ub[HFP][HNV], un[HFP][HNV];
  T q[HNS][3][HNV];
  T qf[HFP][3][HNV];
  T iJ[HNS], ciJ[HNS], Sm[HNS][3][3];
  T fJ[HFP], fnr[HFP][3], wq[HNF];
  T M[HN][HN], lm[HN], lp[HN], dgL[HN], dgR[HN];
  T uinf[5];
  struct Col {
    T dQ[HNS][3], dq[HNS][3];
    T dqf[HFP][3];
    T dFt[HNS][3][HNV];
    T dFn[HFP][HNV], drow[HFP][HNV];
  } col[HJW];
  int kf[6], tr[6];
};
static_assert(sizeof(HJWork<double>) <= 227 * 1024, "hexahedral block workspace exceeds shared memory");

// pointwise Jacobians of one element (global slab of the CTA), innermost index the input variable
template <typename T>
struct HJac {
  T KU[HNS][3][HNV][HNV];
  T KQ[HNS][3][3][HNV][HNV];
  T GU[HFP][HNV][HNV], GH[HFP][HNV][HNV], GQ[HFP][3][HNV][HNV];
  T RU[HFP][HNV][HNV], RH[HFP][HNV][HNV], RQ[HFP][3][HNV][HNV];
};

// NC: points per line as a compile-time constant (the index arithmetic of the lines folds), or 0
// for the element's own degree at run time
template <typename T, int NC>
__global__ void __launch_bounds__(HJT, sizeof(T) == 4 ? 2 : 1) k_hex_jacobian(const __grid_constant__ PhysParams pp,
                                                        const __grid_constant__ GArgs a,
                                                        const __grid_constant__ JArgs j) {
  using DT = Dual<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  HJWork<T>& w = *reinterpret_cast<HJWork<T>*>(smem_raw);
  HJac<T>& J = reinterpret_cast<HJac<T>*>(j.scratch)[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const bool visc = phys_viscous(pp);
  const PhysConst<T> pc = phys_const<T>(pp);
  const GenRef& RF = *a.ref;
  for (int k = blockIdx.x; k < j.Eim; k += gridDim.x) {
    const int e = j.imp_idx[k];
    const int n = NC > 0 ? NC : a.deg[e], ns = n * n * n, nf = n * n, FS = a.fs;
    const int nA = ns * HNV, nT = 6 * nf * HNV;
    const double* gs = a.geo_sol + (size_t)a.goff[e] * 10;
    __syncthreads();  // the previous element's buffers are free
    for (int i = tid; i < n * n; i += HJT) w.M[i / n][i % n] = T(RF.M[n][i / n][i % n]);
    if (tid < n) {
      w.lm[tid] = T(RF.lm[n][tid]);
      w.lp[tid] = T(RF.lp[n][tid]);
      w.dgL[tid] = T(RF.dgL[n][tid]);
      w.dgR[tid] = T(RF.dgR[n][tid]);
    }
    if (tid < nf) w.wq[tid] = T(RF.w[n][tid % n] * RF.w[n][tid / n]);
    if (tid < 6) {
      w.kf[tid] = a.kind[6 * e + tid];
      w.tr[tid] = a.tr_of[6 * e + tid];
    }
    if (tid < 5) w.uinf[tid] = T(a.uinf[tid]);
    for (int i = tid; i < ns; i += HJT) {
      w.iJ[i] = T(gs[i * 10]);
      w.ciJ[i] = T(j.a_dt * gs[i * 10]);
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) w.Sm[i][r][c] = T(gs[i * 10 + 1 + 3 * r + c]);
    }
    for (int jj = tid; jj < 6 * nf; jj += HJT) {
      const double* G = a.geo_face + ((size_t)(6 * e + jj / nf) * FS + jj % nf) * 4;
      w.fJ[jj] = T(G[0]);
      w.fnr[jj][0] = T(G[1]);
      w.fnr[jj][1] = T(G[2]);
      w.fnr[jj][2] = T(G[3]);
    }
    const double* Ue = a.U + a.uoff[e];
    for (int i = tid; i < nA; i += HJT) w.U[i / HNV][i % HNV] = T(Ue[i]);
    __syncthreads();
    for (int it = tid; it < 6 * nf * HNV; it += HJT) {
      const int f = it / (nf * HNV), m = (it / HNV) % nf, v = it % HNV, r = f >> 1;
      const T* l = (f & 1) ? w.lp : w.lm;
      T s = T(0);
      for (int c = 0; c < n; ++c) s += l[c] * w.U[hline(r, m, c, n)][v];
      w.Uf[f * nf + m][v] = s;
      const int t = w.tr[f];
      if (t >= 0) {
        w.ub[f * nf + m][v] = T(a.uhat[(size_t)FR_IDX(a.fnode[(6 * e + f) * FS + m], a.npts, 10) * HNV + v]);
        w.un[f * nf + m][v] = s;
      } else {  // interface face: the explicit neighbour's state
        const int nb = (int)FR_IDX(a.nbr[6 * e + f], a.E, 11), fn = (int)FR_IDX(a.nbr_face[6 * e + f], 6, 12);
        const T un = T(a.Uf_all[((size_t)(6 * nb + fn) * FS + m) * HNV + v]);
        w.un[f * nf + m][v] = un;
        w.ub[f * nf + m][v] = un;
      }
    }
    __syncthreads();
    if (visc) {
      for (int it = tid; it < ns * HNV; it += HJT) {
        const int i = it / HNV, v = it % HNV;
        T Q[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int ar = hcoord(i, r, n), m = hfacept(i, r, n);
          T s = w.dgL[ar] * w.ub[(2 * r) * nf + m][v] + w.dgR[ar] * w.ub[(2 * r + 1) * nf + m][v];
          for (int c = 0; c < n; ++c) s += w.M[ar][c] * w.U[hline(r, m, c, n)][v];
          Q[r] = s;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) w.q[i][c][v] = w.iJ[i] * (w.Sm[i][0][c] * Q[0] + w.Sm[i][1][c] * Q[1] + w.Sm[i][2][c] * Q[2]);
      }
      __syncthreads();
      for (int it = tid; it < 6 * nf * 3 * HNV; it += HJT) {
        const int f = it / (nf * 3 * HNV), m = (it / (3 * HNV)) % nf, c2 = (it / HNV) % 3, v = it % HNV, r = f >> 1;
        const T* l = (f & 1) ? w.lp : w.lm;
        T s = T(0);
        for (int c = 0; c < n; ++c) s += l[c] * w.q[hline(r, m, c, n)][c2][v];
        w.qf[f * nf + m][c2][v] = s;
      }
    } else {
      for (int i = tid; i < HNS * 3 * HNV; i += HJT) (&w.q[0][0][0])[i] = T(0);
      for (int i = tid; i < HFP * 3 * HNV; i += HJT) (&w.qf[0][0][0])[i] = T(0);
    }
    __syncthreads();
    // pointwise Jacobians (dual numbers) into the CTA's slab
    for (int it = tid; it < 2 * ns * HNV; it += HJT) {
      const bool isq = it >= ns * HNV;
      const int idx = isq ? it - ns * HNV : it;
      const int i = idx / HNV, vp = idx % HNV;
      DT u[HNV], qd[3][HNV], F[3][HNV];
#pragma unroll
      for (int v = 0; v < HNV; ++v) {
        u[v] = DT(w.U[i][v], (!isq && v == vp) ? T(1) : T(0));
#pragma unroll
        for (int c = 0; c < 3; ++c) qd[c][v] = DT(w.q[i][c][v]);
      }
      if (!isq) {
        NS3::conv<DT, T>(pc, u, F);
        if (visc) {
          DT Fv[3][HNV];
          NS3::visc<DT, T>(pc, u, qd, Fv);
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int v = 0; v < HNV; ++v) F[c][v] = F[c][v] - Fv[c][v];
        }
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int v = 0; v < HNV; ++v)
            J.KU[i][r][v][vp] = w.Sm[i][r][0] * F[0][v].d + w.Sm[i][r][1] * F[1][v].d + w.Sm[i][r][2] * F[2][v].d;
      } else {
        T acc[3][3][HNV];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int r2 = 0; r2 < 3; ++r2)
#pragma unroll
            for (int v = 0; v < HNV; ++v) acc[r][r2][v] = T(0);
        if (visc) {
#pragma unroll
          for (int c2 = 0; c2 < 3; ++c2) {
            qd[c2][vp].d = T(1);
            NS3::visc<DT, T>(pc, u, qd, F);
            qd[c2][vp].d = T(0);
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
              for (int v = 0; v < HNV; ++v) {
                const T dFr = -(w.Sm[i][r][0] * F[0][v].d + w.Sm[i][r][1] * F[1][v].d + w.Sm[i][r][2] * F[2][v].d);
#pragma unroll
                for (int r2 = 0; r2 < 3; ++r2) acc[r][r2][v] += dFr * w.iJ[i] * w.Sm[i][r2][c2];
              }
          }
        }
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int r2 = 0; r2 < 3; ++r2)
#pragma unroll
            for (int v = 0; v < HNV; ++v) J.KQ[i][r][r2][v][vp] = acc[r][r2][v];
      }
    }
    for (int it = tid; it < 6 * nf * 5 * HNV; it += HJT) {
      const int jj = it / (5 * HNV), dir = it % (5 * HNV), grp = dir / HNV, vp = dir % HNV;
      const int f = jj / nf;
      const int kf = w.kf[f];
      const bool traced = w.tr[f] >= 0;
      DT uf[HNV], ub[HNV], un[HNV], qf[3][HNV], qn[3][HNV], Fn[HNV], row[HNV];
#pragma unroll
      for (int v = 0; v < HNV; ++v) {
        uf[v] = DT(w.Uf[jj][v], (grp == 0 && v == vp) ? T(1) : T(0));
        ub[v] = DT(w.ub[jj][v], (grp == 1 && v == vp) ? T(1) : T(0));
        un[v] = DT(w.un[jj][v]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          qf[c][v] = DT(w.qf[jj][c][v], (grp == 2 + c && v == vp) ? T(1) : T(0));
          qn[c][v] = DT(T(0));
        }
      }
      const bool zero = (grp >= 2 && !visc) || (grp == 1 && !traced);
      if (!zero) {
        const T nr[3] = {w.fnr[jj][0], w.fnr[jj][1], w.fnr[jj][2]};
        hface_flux<DT, T>(pc, visc, kf, traced, true, uf, ub, qf, un, qn, w.fJ[jj], nr, w.uinf, Fn, row);
      }
#pragma unroll
      for (int v = 0; v < HNV; ++v) {
        const T d = zero ? T(0) : Fn[v].d;
        const T dr = (zero || !traced) ? T(0) : row[v].d;
        if (grp == 0) {
          J.GU[jj][v][vp] = d;
          J.RU[jj][v][vp] = dr;
        } else if (grp == 1) {
          J.GH[jj][v][vp] = d;
          J.RH[jj][v][vp] = dr;
        } else {
          J.GQ[jj][grp - 2][v][vp] = d;
          J.RQ[jj][grp - 2][v][vp] = dr;
        }
      }
    }
    __syncthreads();
    // columns, one seed point per warp (column-major blocks: one contiguous run per column)
    T* AT = reinterpret_cast<T*>(j.A) + j.offA[k];
    T* BT = reinterpret_cast<T*>(j.B) + j.offB[k];
    T* CT = reinterpret_cast<T*>(j.C) + j.offB[k];
    T* DTm = reinterpret_cast<T*>(j.D) + j.offD[k];
    // trace unknowns of faces without a trace: zero columns of B and D
    for (int f = 0; f < 6; ++f) {
      if (w.tr[f] >= 0) continue;
      for (int it = tid; it < nf * HNV * (nA + nT); it += HJT) {
        const int col = f * nf * HNV + it / (nA + nT), rr = it % (nA + nT);
        if (rr < nA)
          BT[(size_t)col * nA + rr] = T(0);
        else
          DTm[(size_t)col * nT + rr - nA] = T(0);
      }
    }
    typename HJWork<T>::Col& cw = w.col[wp];
    int nseed_tr = 0;
    for (int f = 0; f < 6; ++f)
      if (w.tr[f] >= 0) nseed_tr += nf;
    for (int sp = wp; sp < ns + nseed_tr; sp += HJW) {
      const bool vol = sp < ns;
      int f0 = -1, m0 = -1;
      if (!vol) {
        int rem = sp - ns;
        for (int f = 0; f < 6; ++f) {
          if (w.tr[f] < 0) continue;
          if (rem < nf) {
            f0 = f;
            m0 = rem;
            break;
          }
          rem -= nf;
        }
      }
      const int r0 = vol ? -1 : f0 >> 1;
      // the gradient tangents depend on the seed point only: formed once for its HNV columns
      // reference and physical gradient tangents (the seed's lines only)
      if (visc) {
        for (int i = lane; i < ns; i += 32) {
          T Q[3];
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            T s = T(0);
            if (vol) {  // on sp's r-line: M[a_r(i)][a_r(sp)]
              if (hfacept(i, r, n) == hfacept(sp, r, n)) s = w.M[hcoord(i, r, n)][hcoord(sp, r, n)];
            } else if (r == r0 && hfacept(i, r, n) == m0) {
              s = (f0 & 1) ? w.dgR[hcoord(i, r, n)] : w.dgL[hcoord(i, r, n)];
            }
            Q[r] = s;
            cw.dQ[i][r] = s;
          }
#pragma unroll
          for (int c = 0; c < 3; ++c)
            cw.dq[i][c] = w.iJ[i] * (w.Sm[i][0][c] * Q[0] + w.Sm[i][1][c] * Q[1] + w.Sm[i][2][c] * Q[2]);
        }
        __syncwarp();
        for (int it = lane; it < 6 * nf * 3; it += 32) {
          const int jj = it / 3, c2 = it % 3, f = jj / nf, m = jj % nf, r = f >> 1;
          const T* l = (f & 1) ? w.lp : w.lm;
          T s = T(0);
          for (int c = 0; c < n; ++c) s += l[c] * cw.dq[hline(r, m, c, n)][c2];
          cw.dqf[jj][c2] = s;
        }
      }
      __syncwarp();
      for (int v0 = 0; v0 < HNV; ++v0) {
        // flux tangents at the solution points (the gradient tangent vanishes off the seed's lines:
        // the pointwise Jacobians are read only where a tangent is nonzero)
        for (int it = lane; it < ns * 3 * HNV; it += 32) {
          const int i = it / (3 * HNV), r = (it / HNV) % 3, v = it % HNV;
          T s = T(0);
          if (visc) {
            const T q0 = cw.dQ[i][0], q1 = cw.dQ[i][1], q2 = cw.dQ[i][2];
            if (q0 != T(0) || q1 != T(0) || q2 != T(0))
              s = J.KQ[i][r][0][v][v0] * q0 + J.KQ[i][r][1][v][v0] * q1 + J.KQ[i][r][2][v][v0] * q2;
          }
          if (vol && i == sp) s += J.KU[i][r][v][v0];
          cw.dFt[i][r][v] = s;
        }
        // face flux and trace-row tangents
        for (int it = lane; it < 6 * nf * HNV; it += 32) {
          const int jj = it / HNV, v = it % HNV, f = jj / nf, m = jj % nf, r = f >> 1;
          T du = T(0);  // face state tangent: l_sigma[a_r(sp)] on the face point of sp's r-line
          if (vol && hfacept(sp, r, n) == m) du = ((f & 1) ? w.lp : w.lm)[hcoord(sp, r, n)];
          const T dh = (!vol && f == f0 && m == m0) ? T(1) : T(0);
          T s = T(0), sr = T(0);
          if (du != T(0)) {
            s += J.GU[jj][v][v0] * du;
            sr += J.RU[jj][v][v0] * du;
          }
          if (dh != T(0)) {
            s += J.GH[jj][v][v0] * dh;
            sr += J.RH[jj][v][v0] * dh;
          }
          if (visc) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const T dq = cw.dqf[jj][c];
              if (dq != T(0)) {
                s += J.GQ[jj][c][v][v0] * dq;
                sr += J.RQ[jj][c][v][v0] * dq;
              }
            }
          }
          cw.dFn[jj][v] = s;
          cw.drow[jj][v] = sr;
        }
        __syncwarp();
        const int col = vol ? sp * HNV + v0 : (f0 * nf + m0) * HNV + v0;
        T* top = (vol ? AT : BT) + (size_t)col * nA;
        T* bot = (vol ? CT : DTm) + (size_t)col * nT;
        for (int it = lane; it < nA; it += 32) {
          const int i = it / HNV, v = it % HNV;
          T d = T(0);
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            const int ar = hcoord(i, r, n), m = hfacept(i, r, n);
            d += -w.dgL[ar] * cw.dFn[(2 * r) * nf + m][v] + w.dgR[ar] * cw.dFn[(2 * r + 1) * nf + m][v];
            for (int c = 0; c < n; ++c) d += w.M[ar][c] * cw.dFt[hline(r, m, c, n)][r][v];
          }
          T o = w.ciJ[i] * d;
          if (vol && it == col) o += T(1);
          top[it] = o;
        }
        for (int it = lane; it < nT; it += 32) {
          const int jj = it / HNV, v = it % HNV, f = jj / nf, m = jj % nf;
          bot[it] = w.tr[f] >= 0 ? w.wq[m] * cw.drow[jj][v] : T(0);
        }
        __syncwarp();
      }
    }
  }
}

// the kernel for a mesh whose elements all have n points per line (hexahedral meshes carry one
// degree), the run-time form otherwise
template <typename T>
static auto hex_jac_kernel(int n) -> decltype(&k_hex_jacobian<T, 0>) {
  switch (n) {
    case 2: return &k_hex_jacobian<T, 2>;
    case 3: return &k_hex_jacobian<T, 3>;
    case 4: return &k_hex_jacobian<T, 4>;
    default: return &k_hex_jacobian<T, 0>;
  }
}

int hex_jacobian_grid(int prec_bytes) {
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm * (prec_bytes == 8 ? 1 : 2);
}

size_t hex_jacobian_scratch_bytes(int prec_bytes, int grid) {
  return (size_t)grid * (prec_bytes == 8 ? sizeof(HJac<double>) : sizeof(HJac<float>));
}

cudaError_t hex_jacobian(GenCtx* g, const GArgs& a, const JArgs& j) {
  cudaError_t e;
  if (j.Eim == 0) return cudaSuccess;
  if (g->pb == 8) {
    const size_t smem = sizeof(HJWork<double>);
    auto kern = hex_jac_kernel<double>(g->h_deg.empty() ? 0 : g->h_deg[0]);
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    (count_launch(), kern<<<g->jgrid, HJT, smem, g->st>>>(g->pp, a, j));
  } else {
    const size_t smem = sizeof(HJWork<float>);
    auto kern = hex_jac_kernel<float>(g->h_deg.empty() ? 0 : g->h_deg[0]);
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    (count_launch(), kern<<<g->jgrid, HJT, smem, g->st>>>(g->pp, a, j));
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------ geometry (host)
void hex_geometry(const double* verts, int E, const int* deg, const long long* goff, double* gsol, double* gface,
                  double* xyz) {
  for (int e = 0; e < E; ++e) {
    const int n = deg[e];
    double x[HN], wg[HN];
    gauss_legendre_nodes(n, x, wg);
    const double* V = verts + (size_t)e * 24;
    auto map = [&](const double r[3], double X[3], double D[3][3]) {  // D[k] = dx/dxi_k
      for (int c = 0; c < 3; ++c) {
        X[c] = 0.0;
        D[0][c] = D[1][c] = D[2][c] = 0.0;
      }
      for (int k = 0; k < 8; ++k) {
        const double s[3] = {(k & 1) ? 1.0 : -1.0, (k & 2) ? 1.0 : -1.0, (k & 4) ? 1.0 : -1.0};
        const double f0 = 1 + s[0] * r[0], f1 = 1 + s[1] * r[1], f2 = 1 + s[2] * r[2];
        const double N = 0.125 * f0 * f1 * f2;
        const double dN[3] = {0.125 * s[0] * f1 * f2, 0.125 * s[1] * f0 * f2, 0.125 * s[2] * f0 * f1};
        for (int c = 0; c < 3; ++c) {
          X[c] += N * V[3 * k + c];
          for (int d = 0; d < 3; ++d) D[d][c] += dN[d] * V[3 * k + c];
        }
      }
    };
    auto cross = [](const double* u, const double* v, double* o) {
      o[0] = u[1] * v[2] - u[2] * v[1];
      o[1] = u[2] * v[0] - u[0] * v[2];
      o[2] = u[0] * v[1] - u[1] * v[0];
    };
    auto adj = [&](double D[3][3], double S[3][3]) {  // S[r] = x_{xi_s} x x_{xi_t}, (r, s, t) cyclic
      cross(D[1], D[2], S[0]);
      cross(D[2], D[0], S[1]);
      cross(D[0], D[1], S[2]);
      return D[0][0] * S[0][0] + D[0][1] * S[0][1] + D[0][2] * S[0][2];
    };
    for (int c3 = 0; c3 < n; ++c3)
      for (int b = 0; b < n; ++b)
        for (int a2 = 0; a2 < n; ++a2) {
          const size_t pt = (size_t)goff[e] + a2 + n * b + n * n * c3;
          const double r[3] = {x[a2], x[b], x[c3]};
          double X[3], D[3][3], S[3][3];
          map(r, X, D);
          const double J = adj(D, S);
          double* G = gsol + 10 * pt;
          G[0] = 1.0 / J;
          for (int rr = 0; rr < 3; ++rr)
            for (int cc = 0; cc < 3; ++cc) G[1 + 3 * rr + cc] = S[rr][cc];
          for (int cc = 0; cc < 3; ++cc) xyz[3 * pt + cc] = X[cc];
        }
    for (int f = 0; f < 6; ++f) {
      const int rax = f >> 1;
      const double sg = (f & 1) ? 1.0 : -1.0;
      const int t0 = rax == 0 ? 1 : 0, t1 = rax == 2 ? 1 : 2;  // lower and higher tangential axes
      for (int jj = 0; jj < n; ++jj)
        for (int ii = 0; ii < n; ++ii) {
          double r[3];
          r[rax] = sg;
          r[t0] = x[ii];
          r[t1] = x[jj];
          double X[3], D[3][3], S[3][3];
          map(r, X, D);
          adj(D, S);
          const double N[3] = {sg * S[rax][0], sg * S[rax][1], sg * S[rax][2]};
          const double Jf = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
          double* G = gface + 4 * ((size_t)(6 * e + f) * HEX_FS + ii + n * jj);
          G[0] = Jf;
          G[1] = N[0] / Jf;
          G[2] = N[1] / Jf;
          G[3] = N[2] / Jf;
        }
    }
  }
}

}  // namespace gen
}  // namespace hfr

#include "hfr_checked_unit.inc"
