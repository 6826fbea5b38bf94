// The hybridized stage on general quadrilateral meshes: per-element polynomial degree p_e (faces
// between unequal degrees) and wall / far-field boundary faces (Pereira & Vermeire,
// arXiv 2401.16632: element blocks that admit faces with different numbers of trace points,
// Sec. 3.2 eq. elemsystemB; the boundary term of the transmission conditions, Sec. 2.2 eq. hfr2).
//
// Readings (the paper writes no operator for either):
//   * a face carries the Gauss points of the higher degree of its two sides, m = max(n-, n+)
//     (a boundary face its element's own n); both sides evaluate their states, fluxes and
//     gradients there, and the common fluxes, the trace unknowns and the trace residual
//     g_q = w_q J_f (F^.n)_q live there;
//   * an element lifts a face jump h from the m face points onto its own n face nodes by the L2
//     projection with the face rule, (P h)_b = sum_q w_q l_b(s_q) h_q / w_b (the identity when
//     m = n; P T = I for the interpolation T from nodes to points), then spreads it along the
//     normal with its DG-recovering correction derivatives;
//   * boundary faces of implicit elements carry a trace: far field g = w J s(u^)((u_f - u^) +
//     (u_inf - u^)); no-slip adiabatic wall (Navier-Stokes): momentum rows w J s(u^) (rho v)^, mass
//     and energy rows the element's own normal fluxes; explicit elements meet the far field with
//     the FR Rusanov flux against a ghost holding u_inf (BR1 common value the average, viscous flux
//     the average of both sides' with the element's own gradient).
//
// Layouts (packed; element e of degree p_e, n_e = p_e + 1, Ns_e = n_e^2):
//   state u, R       element after element, u[uoff[e] + pt nv + v]
//   trace u^, g      trace after trace (traces in increasing global face id), u^[toff[t] + q nv + v]
//   face data        fixed stride of GN points per element face: [(4 e + f) GN + q][nv]
//   blocks of the    implicit element k: A nA_k^2, B nA_k nT_k, C nT_k nA_k, D and S nT_k^2, packed in
//   implicit ones    increasing k; nT_k = nv sum_f m(e, f) over all four faces in local order (rows
//                    and columns of faces without a trace are zero), trace unknown
//                    l = lto[f] + q nv + v
// Kernels: one warp per element for the residual passes, one CTA of 256 threads per implicit
// element for the blocks (dense tangents of the element operator, one warp per seed point), the
// uneven-shape condensation (shared-memory Gauss-Jordan, or the global-memory LU for blocks too
// large for shared memory), and warp-per-element / warp-per-face trace operators under the
// multi-kernel GMRES driver.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "hfr_general_internal.h"

namespace hfr {
namespace gen {

// n-point Gauss-Lobatto rule: the end points and the roots of P'_{n-1} (Newton from the Chebyshev-
// Gauss-Lobatto points), weights 2 / (n (n - 1) P_{n-1}(x)^2)
static void gauss_lobatto_nodes(int n, double* x, double* w) {
  const int N = n - 1;
  for (int i = 0; i < n; ++i) {
    double z = -cos(M_PI * i / N);
    if (i > 0 && i < N) {
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;  // P_0, P_1 -> P_{N-1}, P_N
        for (int k = 2; k <= N; ++k) {
          const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = pk;
        }
        const double dp = N * (p0 - z * p1) / (1.0 - z * z);            // P'_N
        const double d2 = (2.0 * z * dp - N * (N + 1.0) * p1) / (1.0 - z * z);  // P''_N
        const double dz = dp / d2;
        z -= dz;
        if (fabs(dz) < 1e-16) break;
      }
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= N; ++k) {
      const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    const double PN = N == 0 ? 1.0 : p1;
    x[i] = z;
    w[i] = 2.0 / (N * (N + 1.0) * PN * PN);
  }
}

// barycentric interpolation weights of nodes x (n) at point z into l (exact node hits: unit vector)
static void lagrange_at(int n, const double* x, double z, double* l) {
  int hit = -1;
  for (int b = 0; b < n; ++b)
    if (z == x[b]) hit = b;
  if (hit >= 0) {
    for (int b = 0; b < n; ++b) l[b] = b == hit ? 1.0 : 0.0;
    return;
  }
  double den = 0.0, bw[GN];
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) prod *= (x[j] - x[k]);
    bw[j] = 1.0 / prod;
    den += bw[j] / (z - x[j]);
  }
  for (int b = 0; b < n; ++b) l[b] = (bw[b] / (z - x[b])) / den;
}

static void build_genref(GenRef& R) {
  memset(&R, 0, sizeof(R));
  for (int n = 2; n <= GN; ++n) {
    double xg[GN], wg[GN], xl[GN], wl[GN], l[GN];
    gauss_legendre_nodes(n, xg, wg);
    gauss_lobatto_nodes(n, xl, wl);
    for (int q = 0; q < n; ++q) {
      R.wl[n][q] = wl[q];
      lagrange_at(n, xg, xl[q], l);  // Gauss node basis at GLL point q
      for (int b = 0; b < n; ++b) R.TL[n][q][b] = l[b];
    }
    for (int b = 0; b < n; ++b) {
      lagrange_at(n, xl, xg[b], l);  // GLL point basis at Gauss node b
      for (int q = 0; q < n; ++q) R.PL[n][b][q] = l[q];
    }
  }
  for (int n = 2; n <= GN; ++n) {
    RefOps o;
    build_ref_ops(n - 1, o);
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) R.M[n][i][j] = o.M[i][j];
      R.lm[n][i] = o.lm[i];
      R.lp[n][i] = o.lp[i];
      R.dgL[n][i] = o.dgL[i];
      R.dgR[n][i] = o.dgR[i];
      R.w[n][i] = o.w[i];
    }
  }
  for (int n = 2; n <= GN; ++n) {
    double x[GN], wn[GN], bw[GN];
    gauss_legendre_nodes(n, x, wn);
    for (int j = 0; j < n; ++j) {
      double prod = 1.0;
      for (int k = 0; k < n; ++k)
        if (k != j) prod *= (x[j] - x[k]);
      bw[j] = 1.0 / prod;
    }
    for (int m = n; m <= GN; ++m) {
      double s[GN], ws[GN];
      gauss_legendre_nodes(m, s, ws);
      for (int q = 0; q < m; ++q) {
        // barycentric interpolation at s_q (exact node hits give the unit vector)
        int hit = -1;
        for (int b = 0; b < n; ++b)
          if (s[q] == x[b]) hit = b;
        double den = 0.0;
        if (hit < 0)
          for (int b = 0; b < n; ++b) den += bw[b] / (s[q] - x[b]);
        for (int b = 0; b < n; ++b) {
          const double l = hit >= 0 ? (b == hit ? 1.0 : 0.0) : (bw[b] / (s[q] - x[b])) / den;
          R.T[n][m][q][b] = l;
          R.P[n][m][b][q] = ws[q] * l / wn[b];
        }
      }
    }
  }
}

__device__ __forceinline__ int gline(int r, int m, int c, int n) { return r == 0 ? (c + n * m) : (m + n * c); }

// Common normal flux of one face point, scaled by J_f (Fn: the element's own residual sees it) and
// the element's trace row (row: trace faces only).  ub: the trace (traced faces) or the common
// value; un, qn: the other side's state and gradient (FR / IMEX / explicit far field).
template <int PHYS, typename S, typename R, int NV>
__device__ __forceinline__ void gface_flux(const PhysConst<R>& pc, bool visc, int kf, bool traced, bool imp,
                                           const S* uf, const S* ub, const S (&qf)[2][NV], const S* un,
                                           const S (&qn)[2][NV], R Jf, R n0, R n1, const R* uinf, S* Fn, S* row) {
  S F[2][NV];
  if (traced) {
    S Fh[NV];
    Phys<PHYS>::template conv<S, R>(pc, ub, F);
    const S s = Phys<PHYS>::template stab<S, R>(pc, ub, n0, n1);
#pragma unroll
    for (int v = 0; v < NV; ++v) Fh[v] = n0 * F[0][v] + n1 * F[1][v] + s * (uf[v] - ub[v]);
    if (visc) {
      Phys<PHYS>::template visc<S, R>(pc, ub, qf, F);
#pragma unroll
      for (int v = 0; v < NV; ++v) Fh[v] = Fh[v] - (n0 * F[0][v] + n1 * F[1][v]);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) Fn[v] = Jf * Fh[v];
    if (kf == FK_FAR) {
#pragma unroll
      for (int v = 0; v < NV; ++v) row[v] = Jf * s * ((uf[v] - ub[v]) + (uinf[v] - ub[v]));
    } else if (kf == FK_WALL) {
#pragma unroll
      for (int v = 0; v < NV; ++v) row[v] = (v == 0 || v == NV - 1) ? Jf * Fh[v] : Jf * s * ub[v];
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) row[v] = Jf * Fh[v];
    }
    return;
  }
  S G[2][NV];
  Phys<PHYS>::template conv<S, R>(pc, uf, F);
  Phys<PHYS>::template conv<S, R>(pc, un, G);
  const S lam = dmax(Phys<PHYS>::template wave<S, R>(pc, uf, n0, n1), Phys<PHYS>::template wave<S, R>(pc, un, n0, n1));
  S Fh[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v)
    Fh[v] = R(0.5) * (n0 * (F[0][v] + G[0][v]) + n1 * (F[1][v] + G[1][v])) + R(0.5) * lam * (uf[v] - un[v]);
  if (visc) {
    if (kf == FK_FR || kf == FK_FAR) {  // both sides' viscous fluxes averaged
      Phys<PHYS>::template visc<S, R>(pc, uf, qf, F);
      Phys<PHYS>::template visc<S, R>(pc, un, qn, G);
#pragma unroll
      for (int v = 0; v < NV; ++v) Fh[v] = Fh[v] - R(0.5) * (n0 * (F[0][v] + G[0][v]) + n1 * (F[1][v] + G[1][v]));
    } else {  // IMEX interface: the implicit side's viscous flux
      if (imp)
        Phys<PHYS>::template visc<S, R>(pc, uf, qf, F);
      else
        Phys<PHYS>::template visc<S, R>(pc, un, qn, F);
#pragma unroll
      for (int v = 0; v < NV; ++v) Fh[v] = Fh[v] - (n0 * F[0][v] + n1 * F[1][v]);
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    Fn[v] = Jf * Fh[v];
    row[v] = S(R(0));
  }
}

// ------------------------------------------------------------------------ residual passes

template <int NV>
struct GWork {
  double U[GNS][NV];
  double Ufn[GF][NV], Ufp[GF][NV], ubp[GF][NV], ubn[GF][NV];
  double q[GNS][2][NV];
  double qfn[GF][2][NV], qfp[GF][2][NV];
  double Ft[GNS][2][NV];
  double Fnp[GF][NV], Fnn[GF][NV];
  double M[GN][GN], lm[GN], lp[GN], dgL[GN], dgR[GN];
  double Tf[4][GN][GN], Pf[4][GN][GN], wq[4][GN];
  int nf[4], kf[4], tr[4];
};

template <int PHYS, int MODE>
__global__ void __launch_bounds__(32 * GEPB) k_gen_elem(const __grid_constant__ PhysParams pp,
                                                       const __grid_constant__ GArgs a) {
  constexpr int NV = Phys<PHYS>::NV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GWork<NV>& w = reinterpret_cast<GWork<NV>*>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int idx = blockIdx.x * GEPB + (threadIdx.x >> 5);
  if (idx >= (a.elist ? a.nlist : a.E)) return;  // whole warps leave; only warp-level synchronisation below
  const int e = a.elist ? a.elist[idx] : idx;
  const int n = a.deg[e], ns = n * n;
  const GenRef& RF = *a.ref;
  const bool visc = phys_viscous(pp);
  const PhysConst<double> pc = phys_const<double>(pp);
  const bool imp = a.implicit[e] != 0;
  for (int i = lane; i < n * n; i += 32) w.M[i / n][i % n] = RF.M[n][i / n][i % n];
  if (lane < n) {
    w.lm[lane] = RF.lm[n][lane];
    w.lp[lane] = RF.lp[n][lane];
    w.dgL[lane] = RF.dgL[n][lane];
    w.dgR[lane] = RF.dgR[n][lane];
  }
  if (lane < 4) {
    w.nf[lane] = a.nfp[4 * e + lane];
    w.kf[lane] = a.kind[4 * e + lane];
    w.tr[lane] = a.tr_of[4 * e + lane];
  }
  __syncwarp();
  for (int i = lane; i < 4 * GN * GN; i += 32) {
    const int f = i / (GN * GN), x = (i / GN) % GN, y = i % GN, m = w.nf[f];
    const bool gll = a.fset[4 * e + f] != 0;  // EFR face: its n Gauss-Lobatto points
    w.Tf[f][x][y] = (x < m && y < n) ? (gll ? RF.TL[n][x][y] : RF.T[n][m][x][y]) : 0.0;  // [q][b]
    w.Pf[f][x][y] = (x < n && y < m) ? (gll ? RF.PL[n][x][y] : RF.P[n][m][x][y]) : 0.0;  // [b][q]
  }
  if (lane < GF) {
    const int f = lane / GN, q = lane % GN;
    w.wq[f][q] = q < w.nf[f] ? (a.fset[4 * e + f] ? RF.wl[n][q] : RF.w[w.nf[f]][q]) : 0.0;
  }
  const double* Ue = a.U + a.uoff[e];
  for (int i = lane; i < ns * NV; i += 32) w.U[i / NV][i % NV] = Ue[i];
  __syncwarp();
  // face node values (own degree), then the face points
  for (int it = lane; it < 4 * n * NV; it += 32) {
    const int f = it / (n * NV), b = (it / NV) % n, v = it % NV, r = f >> 1;
    const double* l = (f & 1) ? w.lp : w.lm;
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += l[c] * w.U[gline(r, b, c, n)][v];
    w.Ufn[f * GN + b][v] = s;
  }
  __syncwarp();
  for (int it = lane; it < GF * NV; it += 32) {
    const int f = it / (GN * NV), q = (it / NV) % GN, v = it % NV;
    if (q >= w.nf[f]) continue;
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += w.Tf[f][q][b] * w.Ufn[f * GN + b][v];
    w.Ufp[f * GN + q][v] = s;
    if (MODE == GM_UF) a.Uf_out[((size_t)(4 * e + f) * GN + q) * NV + v] = s;
  }
  if (MODE == GM_UF) return;
  __syncwarp();
  // trace or common value at the face points
  for (int it = lane; it < GF * NV; it += 32) {
    const int f = it / (GN * NV), q = (it / NV) % GN, v = it % NV;
    if (q >= w.nf[f]) continue;
    const int kf = w.kf[f], t = w.tr[f];
    const double uf = w.Ufp[f * GN + q][v];
    double ub;
    if (t >= 0) {
      ub = a.uhat[(size_t)FR_IDX(a.fnode[(4 * e + f) * GN + q], a.npts, 1) * NV + v];
    } else if (kf == FK_FAR) {
      ub = 0.5 * (uf + a.uinf[v]);
    } else {
      const int nb = (int)FR_IDX(a.nbr[4 * e + f], a.E, 2), fn = (int)FR_IDX(a.nbr_face[4 * e + f], 4, 3);
      const double un = a.Uf_all[((size_t)(4 * nb + fn) * GN + q) * NV + v];
      ub = kf == FK_FR ? 0.5 * (uf + un) : (imp ? un : uf);
    }
    w.ubp[f * GN + q][v] = ub;
  }
  __syncwarp();
  // common value at the own face nodes: u_f + P (u_bar - u_f(points))
  for (int it = lane; it < 4 * n * NV; it += 32) {
    const int f = it / (n * NV), b = (it / NV) % n, v = it % NV;
    double s = w.Ufn[f * GN + b][v];
    for (int q = 0; q < w.nf[f]; ++q) s += w.Pf[f][b][q] * (w.ubp[f * GN + q][v] - w.Ufp[f * GN + q][v]);
    w.ubn[f * GN + b][v] = s;
  }
  __syncwarp();
  const double* gs = a.geo_sol + (size_t)a.goff[e] * 5;
  if (visc) {
    for (int it = lane; it < ns * NV; it += 32) {
      const int i = it / NV, v = it % NV, ai = i % n, bi = i / n;
      const double* G = gs + i * 5;
      double q0 = w.dgL[ai] * w.ubn[0 * GN + bi][v] + w.dgR[ai] * w.ubn[1 * GN + bi][v];
      double q1 = w.dgL[bi] * w.ubn[2 * GN + ai][v] + w.dgR[bi] * w.ubn[3 * GN + ai][v];
      for (int c = 0; c < n; ++c) {
        q0 += w.M[ai][c] * w.U[c + n * bi][v];
        q1 += w.M[bi][c] * w.U[ai + n * c][v];
      }
      w.q[i][0][v] = G[0] * (G[1] * q0 + G[3] * q1);
      w.q[i][1][v] = G[0] * (G[2] * q0 + G[4] * q1);
    }
    __syncwarp();
    for (int it = lane; it < 4 * n * 2 * NV; it += 32) {
      const int f = it / (n * 2 * NV), b = (it / (2 * NV)) % n, c2 = (it / NV) % 2, v = it % NV, r = f >> 1;
      const double* l = (f & 1) ? w.lp : w.lm;
      double s = 0.0;
      for (int c = 0; c < n; ++c) s += l[c] * w.q[gline(r, b, c, n)][c2][v];
      w.qfn[f * GN + b][c2][v] = s;
    }
    __syncwarp();
    for (int it = lane; it < GF * 2 * NV; it += 32) {
      const int f = it / (GN * 2 * NV), q = (it / (2 * NV)) % GN, c2 = (it / NV) % 2, v = it % NV;
      if (q >= w.nf[f]) continue;
      double s = 0.0;
      for (int b = 0; b < n; ++b) s += w.Tf[f][q][b] * w.qfn[f * GN + b][c2][v];
      w.qfp[f * GN + q][c2][v] = s;
      if (MODE == GM_QF) a.qf_out[(((size_t)(4 * e + f) * GN + q) * 2 + c2) * NV + v] = s;
    }
  } else if (MODE == GM_QF) {
    for (int it = lane; it < GF * 2 * NV; it += 32) a.qf_out[(size_t)(4 * e) * GN * 2 * NV + it] = 0.0;
  }
  if (MODE == GM_QF) return;
  __syncwarp();
  // transformed flux at the solution points
  for (int i = lane; i < ns; i += 32) {
    const double* G = gs + i * 5;
    double F[2][NV];
    Phys<PHYS>::template conv<double, double>(pc, w.U[i], F);
    if (visc) {
      double Fv[2][NV];
      Phys<PHYS>::template visc<double, double>(pc, w.U[i], w.q[i], Fv);
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int v = 0; v < NV; ++v) F[c][v] -= Fv[c][v];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      w.Ft[i][0][v] = G[1] * F[0][v] + G[2] * F[1][v];
      w.Ft[i][1][v] = G[3] * F[0][v] + G[4] * F[1][v];
    }
  }
  // common normal flux at the face points
  for (int j = lane; j < GF; j += 32) {
    const int f = j / GN, q = j % GN;
    if (q >= w.nf[f]) continue;
    const int kf = w.kf[f];
    const bool traced = w.tr[f] >= 0;
    const double* G = a.geo_face + ((size_t)(4 * e + f) * GN + q) * 3;
    double un[NV], qn[2][NV], Fn[NV], row[NV];
    if (!traced) {
      if (kf == FK_FAR) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          un[v] = a.uinf[v];
          qn[0][v] = w.qfp[j][0][v];
          qn[1][v] = w.qfp[j][1][v];
        }
      } else {
        const int nb = (int)FR_IDX(a.nbr[4 * e + f], a.E, 2), fn = (int)FR_IDX(a.nbr_face[4 * e + f], 4, 3);
        const size_t nix = (size_t)(4 * nb + fn) * GN + q;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          un[v] = a.Uf_all[nix * NV + v];
          qn[0][v] = a.qf_all[(nix * 2 + 0) * NV + v];
          qn[1][v] = a.qf_all[(nix * 2 + 1) * NV + v];
        }
      }
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) un[v] = qn[0][v] = qn[1][v] = 0.0;
    }
    if (!visc) {
#pragma unroll
      for (int v = 0; v < NV; ++v) w.qfp[j][0][v] = w.qfp[j][1][v] = 0.0;
    }
    gface_flux<PHYS, double, double, NV>(pc, visc, kf, traced, imp, w.Ufp[j], w.ubp[j], w.qfp[j], un, qn, G[0], G[1],
                                         G[2], a.uinf, Fn, row);
#pragma unroll
    for (int v = 0; v < NV; ++v) w.Fnp[j][v] = Fn[v];
    if (a.gview) {
      const double wq = traced ? w.wq[f][q] : 0.0;
#pragma unroll
      for (int v = 0; v < NV; ++v) a.gview[((size_t)(4 * e + f) * GN + q) * NV + v] = wq * row[v];
    }
  }
  __syncwarp();
  for (int it = lane; it < 4 * n * NV; it += 32) {
    const int f = it / (n * NV), b = (it / NV) % n, v = it % NV;
    double s = 0.0;
    for (int q = 0; q < w.nf[f]; ++q) s += w.Pf[f][b][q] * w.Fnp[f * GN + q][v];
    w.Fnn[f * GN + b][v] = s;
  }
  __syncwarp();
  for (int it = lane; it < ns * NV; it += 32) {
    const int i = it / NV, v = it % NV, ai = i % n, bi = i / n;
    double d = -w.dgL[ai] * w.Fnn[0 * GN + bi][v] + w.dgR[ai] * w.Fnn[1 * GN + bi][v] -
               w.dgL[bi] * w.Fnn[2 * GN + ai][v] + w.dgR[bi] * w.Fnn[3 * GN + ai][v];
    for (int c = 0; c < n; ++c) d += w.M[ai][c] * w.Ft[c + n * bi][0][v] + w.M[bi][c] * w.Ft[ai + n * c][1][v];
    if (a.R) a.R[a.uoff[e] + it] = -gs[i * 5] * d;
  }
}

// trace residual: every trace point's value is the sum of the element rows at the element face
// points that carry it (two sides on HFR faces, every face meeting at an EFR node)
__global__ void k_gen_trace_sum(size_t npts, int nv, const long long* __restrict__ gptr,
                                const long long* __restrict__ gidx, const double* __restrict__ gview,
                                double* __restrict__ g, long long nview) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts * nv) return;
  const size_t pt = i / nv;
  const int v = (int)(i % nv);
  double s = 0.0;
  for (long long c = gptr[pt]; c < gptr[pt + 1]; ++c) s += gview[(size_t)FR_IDX(gidx[c], nview, 5) * nv + v];
  g[i] = s;
}

// initial trace: the average of the states at the element face points that carry the trace point;
// a boundary trace point (one side): far field, the average with u_inf; wall, the element's state
// with zero momentum
__global__ void k_gen_initial_trace(size_t npts, int nv, const long long* __restrict__ gptr,
                                    const long long* __restrict__ gidx, const int* __restrict__ kind,
                                    const double* __restrict__ Uf, GArgs a, double* __restrict__ uhat) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npts * nv) return;
  const size_t pt = i / nv;
  const int v = (int)(i % nv);
  const long long c0 = gptr[pt], c1 = gptr[pt + 1];
  const long long nview = (long long)a.nface * a.E * a.fs;  // the bound of the checked build
  (void)nview;
  const long long i0 = FR_IDX(gidx[c0], nview, 6);
  const int kf = kind[i0 / a.fs];
  double x;
  if (kf == FK_FAR) {
    x = 0.5 * (Uf[(size_t)i0 * nv + v] + a.uinf[v]);
  } else if (kf == FK_WALL) {
    x = (v == 0 || v == nv - 1) ? Uf[(size_t)i0 * nv + v] : 0.0;  // zero momentum
  } else {
    double s = 0.0;
    for (long long c = c0; c < c1; ++c) s += Uf[(size_t)FR_IDX(gidx[c], nview, 6) * nv + v];
    x = s / (double)(c1 - c0);
  }
  uhat[i] = x;
}

// ------------------------------------------------------------------------ element blocks
// One CTA per implicit element.  Primal state, pointwise Jacobians of the volume flux (state and
// reference gradient) and of the face flux and trace row (face state, trace, face gradient) by
// dual numbers, then one warp per seed point (a solution point: NV columns of A and C; a trace
// face point: NV columns of B and D) propagating the unit tangent through the linear chain of the
// element operator: face nodes -> face points -> common values at the nodes -> corrected gradient
// -> flux tangents at the solution points and the face points -> projection to the face nodes ->
// divergence.  Columns are staged per seed point and written as rows of NV consecutive values.

template <int NV, typename T>
struct JWork {
  T U[GNS][NV];
  T Ufn[GF][NV], Ufp[GF][NV], ubp[GF][NV], ubn[GF][NV], un[GF][NV];
  T q[GNS][2][NV];
  T qfn[GF][2][NV], qfp[GF][2][NV];
  T iJ[GNS], ciJ[GNS], Sm[GNS][2][2];
  T fJ[GF], fnr[GF][2];
  T M[GN][GN], lm[GN], lp[GN], dgL[GN], dgR[GN];
  T Tf[4][GN][GN], Pf[4][GN][GN], wq[4][GN];
  // pointwise Jacobians, innermost index the input variable
  T KU[GNS][2][NV][NV];
  T KQ[GNS][2][2][NV][NV];
  T GU[GF][NV][NV], GH[GF][NV][NV], GQ[GF][2][NV][NV];
  T RU[GF][NV][NV], RH[GF][NV][NV], RQ[GF][2][NV][NV];
  struct Col {
    T dUfn[GF], dUfp[GF], dubp[GF], dubn[GF];
    T dQ[GNS][2], dq[GNS][2];
    T dqfn[GF][2], dqfp[GF][2];
    T dFt[GNS][2][NV];
    T dFnp[GF][NV], drow[GF][NV], dFnn[GF][NV];
  } col[JW];
  T uinf[5];
  int nf[4], kf[4], tr[4], lto[4];
};

static_assert(sizeof(JWork<4, double>) <= 227 * 1024, "block kernel workspace exceeds shared memory");
static_assert(sizeof(GWork<4>) * GEPB <= 227 * 1024, "residual workspace exceeds shared memory");

template <int PHYS, typename T>
__global__ void __launch_bounds__(JT, sizeof(T) == 4 ? 3 : 1) k_gen_jacobian(const __grid_constant__ PhysParams pp,
                                                    const __grid_constant__ GArgs a,
                                                    const __grid_constant__ JArgs j) {
  constexpr int NV = Phys<PHYS>::NV;
  using DT = Dual<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  JWork<NV, T>& w = *reinterpret_cast<JWork<NV, T>*>(smem_raw);
  const int k = blockIdx.x;
  if (k >= j.Eim) return;
  const int e = j.imp_idx[k];
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int n = a.deg[e], ns = n * n;
  const int nA = ns * NV;
  const GenRef& RF = *a.ref;
  const bool visc = phys_viscous(pp);
  const PhysConst<T> pc = phys_const<T>(pp);
  const double* gs = a.geo_sol + (size_t)a.goff[e] * 5;
  for (int i = tid; i < n * n; i += JT) w.M[i / n][i % n] = T(RF.M[n][i / n][i % n]);
  if (tid < n) {
    w.lm[tid] = T(RF.lm[n][tid]);
    w.lp[tid] = T(RF.lp[n][tid]);
    w.dgL[tid] = T(RF.dgL[n][tid]);
    w.dgR[tid] = T(RF.dgR[n][tid]);
  }
  if (tid < 4) {
    w.nf[tid] = a.nfp[4 * e + tid];
    w.kf[tid] = a.kind[4 * e + tid];
    w.tr[tid] = a.tr_of[4 * e + tid];
    w.lto[tid] = j.lto[4 * k + tid];
  }
  if (tid < 5) w.uinf[tid] = T(a.uinf[tid]);
  for (int i = tid; i < ns; i += JT) {
    w.iJ[i] = T(gs[i * 5]);
    w.ciJ[i] = T(j.a_dt * gs[i * 5]);
    w.Sm[i][0][0] = T(gs[i * 5 + 1]);
    w.Sm[i][0][1] = T(gs[i * 5 + 2]);
    w.Sm[i][1][0] = T(gs[i * 5 + 3]);
    w.Sm[i][1][1] = T(gs[i * 5 + 4]);
  }
  const double* Ue = a.U + a.uoff[e];
  for (int i = tid; i < nA; i += JT) w.U[i / NV][i % NV] = T(Ue[i]);
  __syncthreads();
  for (int i = tid; i < 4 * GN * GN; i += JT) {
    const int f = i / (GN * GN), x = (i / GN) % GN, y = i % GN, m = w.nf[f];
    const bool gll = a.fset[4 * e + f] != 0;
    w.Tf[f][x][y] = (x < m && y < n) ? T(gll ? RF.TL[n][x][y] : RF.T[n][m][x][y]) : T(0);
    w.Pf[f][x][y] = (x < n && y < m) ? T(gll ? RF.PL[n][x][y] : RF.P[n][m][x][y]) : T(0);
  }
  for (int jj = tid; jj < GF; jj += JT) {
    const int f = jj / GN, q = jj % GN;
    w.wq[f][q] = q < w.nf[f] ? T(a.fset[4 * e + f] ? RF.wl[n][q] : RF.w[w.nf[f]][q]) : T(0);
    const double* G = a.geo_face + ((size_t)(4 * e + f) * GN + q) * 3;
    w.fJ[jj] = q < w.nf[f] ? T(G[0]) : T(0);
    w.fnr[jj][0] = q < w.nf[f] ? T(G[1]) : T(0);
    w.fnr[jj][1] = q < w.nf[f] ? T(G[2]) : T(0);
  }
  for (int it = tid; it < 4 * n * NV; it += JT) {
    const int f = it / (n * NV), b = (it / NV) % n, v = it % NV, r = f >> 1;
    const T* l = (f & 1) ? w.lp : w.lm;
    T s = T(0);
    for (int c = 0; c < n; ++c) s += l[c] * w.U[gline(r, b, c, n)][v];
    w.Ufn[f * GN + b][v] = s;
  }
  __syncthreads();
  for (int it = tid; it < GF * NV; it += JT) {
    const int f = it / (GN * NV), q = (it / NV) % GN, v = it % NV;
    T s = T(0), ub = T(0), un = T(0);
    if (q < w.nf[f]) {
      for (int b = 0; b < n; ++b) s += w.Tf[f][q][b] * w.Ufn[f * GN + b][v];
      const int t = w.tr[f];
      if (t >= 0) {
        ub = T(a.uhat[(size_t)FR_IDX(a.fnode[(4 * e + f) * GN + q], a.npts, 4) * NV + v]);
        un = s;
      } else {  // interface face of an implicit element: the explicit neighbour's state
        const int nb = (int)FR_IDX(a.nbr[4 * e + f], a.E, 2), fn = (int)FR_IDX(a.nbr_face[4 * e + f], 4, 3);
        un = T(a.Uf_all[((size_t)(4 * nb + fn) * GN + q) * NV + v]);
        ub = un;
      }
    }
    w.Ufp[f * GN + q][v] = s;
    w.ubp[f * GN + q][v] = ub;
    w.un[f * GN + q][v] = un;
  }
  __syncthreads();
  for (int it = tid; it < 4 * GN * NV; it += JT) {
    const int f = it / (GN * NV), b = (it / NV) % GN, v = it % NV;
    T s = T(0);
    if (b < n) {
      s = w.Ufn[f * GN + b][v];
      for (int q = 0; q < w.nf[f]; ++q) s += w.Pf[f][b][q] * (w.ubp[f * GN + q][v] - w.Ufp[f * GN + q][v]);
    }
    w.ubn[f * GN + b][v] = s;
  }
  __syncthreads();
  if (visc) {
    for (int it = tid; it < ns * NV; it += JT) {
      const int i = it / NV, v = it % NV, ai = i % n, bi = i / n;
      T q0 = w.dgL[ai] * w.ubn[0 * GN + bi][v] + w.dgR[ai] * w.ubn[1 * GN + bi][v];
      T q1 = w.dgL[bi] * w.ubn[2 * GN + ai][v] + w.dgR[bi] * w.ubn[3 * GN + ai][v];
      for (int c = 0; c < n; ++c) {
        q0 += w.M[ai][c] * w.U[c + n * bi][v];
        q1 += w.M[bi][c] * w.U[ai + n * c][v];
      }
      w.q[i][0][v] = w.iJ[i] * (w.Sm[i][0][0] * q0 + w.Sm[i][1][0] * q1);
      w.q[i][1][v] = w.iJ[i] * (w.Sm[i][0][1] * q0 + w.Sm[i][1][1] * q1);
    }
    __syncthreads();
    for (int it = tid; it < 4 * n * 2 * NV; it += JT) {
      const int f = it / (n * 2 * NV), b = (it / (2 * NV)) % n, c2 = (it / NV) % 2, v = it % NV, r = f >> 1;
      const T* l = (f & 1) ? w.lp : w.lm;
      T s = T(0);
      for (int c = 0; c < n; ++c) s += l[c] * w.q[gline(r, b, c, n)][c2][v];
      w.qfn[f * GN + b][c2][v] = s;
    }
    __syncthreads();
    for (int it = tid; it < GF * 2 * NV; it += JT) {
      const int f = it / (GN * 2 * NV), q = (it / (2 * NV)) % GN, c2 = (it / NV) % 2, v = it % NV;
      T s = T(0);
      if (q < w.nf[f])
        for (int b = 0; b < n; ++b) s += w.Tf[f][q][b] * w.qfn[f * GN + b][c2][v];
      w.qfp[f * GN + q][c2][v] = s;
    }
  } else {
    for (int i = tid; i < GNS * 2 * NV; i += JT) (&w.q[0][0][0])[i] = T(0);
    for (int i = tid; i < GF * 2 * NV; i += JT) (&w.qfp[0][0][0])[i] = T(0);
  }
  __syncthreads();

  // -------------------------------------------------- pointwise Jacobians
  for (int it = tid; it < 2 * ns * NV; it += JT) {
    const bool isq = it >= ns * NV;
    const int idx = isq ? it - ns * NV : it;
    const int i = idx / NV, vp = idx % NV;
    DT u[NV], qd[2][NV], F[2][NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      u[v] = DT(w.U[i][v], (!isq && v == vp) ? T(1) : T(0));
      qd[0][v] = DT(w.q[i][0][v]);
      qd[1][v] = DT(w.q[i][1][v]);
    }
    if (!isq) {
      Phys<PHYS>::template conv<DT, T>(pc, u, F);
      if (visc) {
        DT Fv[2][NV];
        Phys<PHYS>::template visc<DT, T>(pc, u, qd, Fv);
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int v = 0; v < NV; ++v) F[c][v] = F[c][v] - Fv[c][v];
      }
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int v = 0; v < NV; ++v) w.KU[i][r][v][vp] = w.Sm[i][r][0] * F[0][v].d + w.Sm[i][r][1] * F[1][v].d;
    } else {
      T acc[2][2][NV];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int r2 = 0; r2 < 2; ++r2)
#pragma unroll
          for (int v = 0; v < NV; ++v) acc[r][r2][v] = T(0);
      if (visc) {
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2) {
          qd[c2][vp].d = T(1);
          Phys<PHYS>::template visc<DT, T>(pc, u, qd, F);
          qd[c2][vp].d = T(0);
#pragma unroll
          for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              const T dFr = -(w.Sm[i][r][0] * F[0][v].d + w.Sm[i][r][1] * F[1][v].d);
#pragma unroll
              for (int r2 = 0; r2 < 2; ++r2) acc[r][r2][v] += dFr * w.iJ[i] * w.Sm[i][r2][c2];
            }
        }
      }
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int r2 = 0; r2 < 2; ++r2)
#pragma unroll
          for (int v = 0; v < NV; ++v) w.KQ[i][r][r2][v][vp] = acc[r][r2][v];
    }
  }
  for (int it = tid; it < GF * 4 * NV; it += JT) {
    const int jj = it / (4 * NV), dir = it % (4 * NV), grp = dir / NV, vp = dir % NV;
    const int f = jj / GN, q = jj % GN;
    const bool live = q < w.nf[f];
    const int kf = w.kf[f];
    const bool traced = w.tr[f] >= 0;
    DT uf[NV], ub[NV], un[NV], qf[2][NV], qn[2][NV], Fn[NV], row[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      uf[v] = DT(w.Ufp[jj][v], (grp == 0 && v == vp) ? T(1) : T(0));
      ub[v] = DT(w.ubp[jj][v], (grp == 1 && v == vp) ? T(1) : T(0));
      un[v] = DT(w.un[jj][v]);
      qf[0][v] = DT(w.qfp[jj][0][v], (grp == 2 && v == vp) ? T(1) : T(0));
      qf[1][v] = DT(w.qfp[jj][1][v], (grp == 3 && v == vp) ? T(1) : T(0));
      qn[0][v] = qn[1][v] = DT(T(0));
    }
    const bool zero = !live || (grp >= 2 && !visc) || (grp == 1 && !traced);
    if (!zero)
      gface_flux<PHYS, DT, T, NV>(pc, visc, kf, traced, true, uf, ub, qf, un, qn, w.fJ[jj], w.fnr[jj][0],
                                  w.fnr[jj][1], w.uinf, Fn, row);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T d = zero ? T(0) : Fn[v].d;
      const T dr = (zero || !traced) ? T(0) : row[v].d;
      if (grp == 0) {
        w.GU[jj][v][vp] = d;
        w.RU[jj][v][vp] = dr;
      } else if (grp == 1) {
        w.GH[jj][v][vp] = d;
        w.RH[jj][v][vp] = dr;
      } else {
        w.GQ[jj][grp - 2][v][vp] = d;
        w.RQ[jj][grp - 2][v][vp] = dr;
      }
    }
  }
  __syncthreads();

  // -------------------------------------------------- columns, one seed point per warp
  int nseed_tr = 0;
  for (int f = 0; f < 4; ++f)
    if (w.tr[f] >= 0) nseed_tr += w.nf[f];
  int nT = 0;
  for (int f = 0; f < 4; ++f) nT += w.nf[f] * NV;
  T* Ab = reinterpret_cast<T*>(j.A) + j.offA[k];
  T* Bb = reinterpret_cast<T*>(j.B) + j.offB[k];
  T* Cb = reinterpret_cast<T*>(j.C) + j.offB[k];
  T* Db = reinterpret_cast<T*>(j.D) + j.offD[k];
  // columns of faces without a trace are zero in B and D
  for (int f = 0; f < 4; ++f) {
    if (w.tr[f] >= 0) continue;
    const int c0 = w.lto[f], cn = w.nf[f] * NV;
    for (int it = tid; it < (nA + nT) * cn; it += JT) {
      const int rrow = it / cn, c = c0 + it % cn;
      if (rrow < nA)
        Bb[(size_t)rrow * nT + c] = T(0);
      else
        Db[(size_t)(rrow - nA) * nT + c] = T(0);
    }
  }
  typename JWork<NV, T>::Col& cw = w.col[wp];
  for (int sp = wp; sp < ns + nseed_tr; sp += JW) {
    const bool vol = sp < ns;
    int a0 = 0, b0 = 0, f0 = -1, q0 = -1;
    if (vol) {
      a0 = sp % n;
      b0 = sp / n;
    } else {
      int rem = sp - ns;
      for (int f = 0; f < 4; ++f) {
        if (w.tr[f] < 0) continue;
        if (rem < w.nf[f]) {
          f0 = f;
          q0 = rem;
          break;
        }
        rem -= w.nf[f];
      }
    }
    // the tangents of the linear chain (face values, common values, gradients) depend on the seed
    // point only: formed once for its NV columns
    // face node and face point tangents of the state, trace tangent
    for (int jj = lane; jj < GF; jj += 32) {
      const int f = jj / GN, b = jj % GN, r = f >> 1;
      T d = T(0);
      if (vol && b < n) {
        const T* l = (f & 1) ? w.lp : w.lm;
        if (r == 0 && b == b0) d = l[a0];
        if (r == 1 && b == a0) d = l[b0];
      }
      cw.dUfn[jj] = d;
      cw.dubp[jj] = (!vol && f == f0 && b == q0) ? T(1) : T(0);
    }
    __syncwarp();
    for (int jj = lane; jj < GF; jj += 32) {
      const int f = jj / GN, q = jj % GN;
      T s = T(0);
      if (q < w.nf[f])
        for (int b = 0; b < n; ++b) s += w.Tf[f][q][b] * cw.dUfn[f * GN + b];
      cw.dUfp[jj] = s;
    }
    __syncwarp();
    if (visc) {
      for (int jj = lane; jj < GF; jj += 32) {
        const int f = jj / GN, b = jj % GN;
        T s = T(0);
        if (b < n) {
          s = cw.dUfn[jj];
          for (int q = 0; q < w.nf[f]; ++q) s += w.Pf[f][b][q] * (cw.dubp[f * GN + q] - cw.dUfp[f * GN + q]);
        }
        cw.dubn[jj] = s;
      }
      __syncwarp();
      for (int i = lane; i < ns; i += 32) {
        const int ai = i % n, bi = i / n;
        T q0v = w.dgL[ai] * cw.dubn[0 * GN + bi] + w.dgR[ai] * cw.dubn[1 * GN + bi];
        T q1v = w.dgL[bi] * cw.dubn[2 * GN + ai] + w.dgR[bi] * cw.dubn[3 * GN + ai];
        if (vol && bi == b0) q0v += w.M[ai][a0];
        if (vol && ai == a0) q1v += w.M[bi][b0];
        cw.dQ[i][0] = q0v;
        cw.dQ[i][1] = q1v;
        cw.dq[i][0] = w.iJ[i] * (w.Sm[i][0][0] * q0v + w.Sm[i][1][0] * q1v);
        cw.dq[i][1] = w.iJ[i] * (w.Sm[i][0][1] * q0v + w.Sm[i][1][1] * q1v);
      }
      __syncwarp();
      for (int it = lane; it < GF * 2; it += 32) {
        const int jj = it >> 1, c2 = it & 1, f = jj / GN, b = jj % GN, r = f >> 1;
        T s = T(0);
        if (b < n) {
          const T* l = (f & 1) ? w.lp : w.lm;
          for (int c = 0; c < n; ++c) s += l[c] * cw.dq[gline(r, b, c, n)][c2];
        }
        cw.dqfn[jj][c2] = s;
      }
      __syncwarp();
      for (int it = lane; it < GF * 2; it += 32) {
        const int jj = it >> 1, c2 = it & 1, f = jj / GN, q = jj % GN;
        T s = T(0);
        if (q < w.nf[f])
          for (int b = 0; b < n; ++b) s += w.Tf[f][q][b] * cw.dqfn[f * GN + b][c2];
        cw.dqfp[jj][c2] = s;
      }
    }
    __syncwarp();
    // the seed point's NV columns, written column by column (the writes of one seed point's
    // columns meet in the same sectors in L2)
    const int col0 = vol ? sp * NV : w.lto[f0] + q0 * NV;
    const int ncol = vol ? nA : nT;
    T* top = vol ? Ab : Bb;
    T* bot = vol ? Cb : Db;
    for (int v0 = 0; v0 < NV; ++v0) {
      // flux tangents at the solution points
      for (int it = lane; it < ns * 2 * NV; it += 32) {
        const int i = it / (2 * NV), r = (it / NV) % 2, v = it % NV;
        T s = T(0);
        if (visc) s = w.KQ[i][r][0][v][v0] * cw.dQ[i][0] + w.KQ[i][r][1][v][v0] * cw.dQ[i][1];
        if (vol && i == sp) s += w.KU[i][r][v][v0];
        cw.dFt[i][r][v] = s;
      }
      // face-point flux and trace-row tangents
      for (int it = lane; it < GF * NV; it += 32) {
        const int jj = it / NV, v = it % NV, f = jj / GN, q = jj % GN;
        T s = T(0), sr = T(0);
        if (q < w.nf[f]) {
          const T du = cw.dUfp[jj], dh = cw.dubp[jj];
          s = w.GU[jj][v][v0] * du + w.GH[jj][v][v0] * dh;
          sr = w.RU[jj][v][v0] * du + w.RH[jj][v][v0] * dh;
          if (visc) {
            s += w.GQ[jj][0][v][v0] * cw.dqfp[jj][0] + w.GQ[jj][1][v][v0] * cw.dqfp[jj][1];
            sr += w.RQ[jj][0][v][v0] * cw.dqfp[jj][0] + w.RQ[jj][1][v][v0] * cw.dqfp[jj][1];
          }
        }
        cw.dFnp[jj][v] = s;
        cw.drow[jj][v] = sr;
      }
      __syncwarp();
      for (int it = lane; it < GF * NV; it += 32) {
        const int jj = it / NV, v = it % NV, f = jj / GN, b = jj % GN;
        T s = T(0);
        if (b < n)
          for (int q = 0; q < w.nf[f]; ++q) s += w.Pf[f][b][q] * cw.dFnp[f * GN + q][v];
        cw.dFnn[jj][v] = s;
      }
      __syncwarp();
      // A / B column: a dt / J times the divergence tangent (plus the identity of A)
      for (int it = lane; it < nA; it += 32) {
        const int i = it / NV, v = it % NV, ai = i % n, bi = i / n;
        T d = -w.dgL[ai] * cw.dFnn[0 * GN + bi][v] + w.dgR[ai] * cw.dFnn[1 * GN + bi][v] -
              w.dgL[bi] * cw.dFnn[2 * GN + ai][v] + w.dgR[bi] * cw.dFnn[3 * GN + ai][v];
        for (int c = 0; c < n; ++c) d += w.M[ai][c] * cw.dFt[c + n * bi][0][v] + w.M[bi][c] * cw.dFt[ai + n * c][1][v];
        T o = w.ciJ[i] * d;
        if (vol && i == sp && v == v0) o += T(1);
        top[(size_t)it * ncol + col0 + v0] = o;
      }
      // C / D column: the element's trace rows w_q (row tangent), zero off traces
      for (int it = lane; it < nT; it += 32) {
        int f = 0, rem = it;
        while (rem >= w.nf[f] * NV) {
          rem -= w.nf[f] * NV;
          ++f;
        }
        const int q = rem / NV, v = rem % NV;
        bot[(size_t)it * ncol + col0 + v0] = w.tr[f] >= 0 ? w.wq[f][q] * cw.drow[f * GN + q][v] : T(0);
      }
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------------------ Newton pieces
// r_k = -(u - u* - a dt R), s_k = -(element trace rows), one warp per implicit element
__global__ void k_gen_form_rhs(int Eim, int nv, int nface, int fs, int dim, const int* __restrict__ imp_idx,
                               const int* __restrict__ deg,
                               const long long* __restrict__ uoff, const long long* __restrict__ offr,
                               const long long* __restrict__ offs, const int* __restrict__ nfp,
                               const int* __restrict__ lto, const double* __restrict__ U,
                               const double* __restrict__ Ustar, const double* __restrict__ R,
                               const double* __restrict__ gview, double adt, double* __restrict__ r,
                               double* __restrict__ s) {
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= Eim) return;
  const int e = imp_idx[k];
  const long long u0 = uoff[e];
  const int nA = (int)(uoff[e + 1] - u0);
  (void)deg;
  (void)dim;
  for (int i = lane; i < nA; i += 32) {
    const double us = Ustar ? Ustar[u0 + i] : U[u0 + i];
    r[offr[k] + i] = -(U[u0 + i] - us - adt * R[u0 + i]);
  }
  for (int f = 0; f < nface; ++f) {
    const int cnt = nfp[nface * e + f] * nv;
    for (int i = lane; i < cnt; i += 32)
      s[offs[k] + lto[nface * k + f] + i] = -gview[(size_t)(nface * e + f) * fs * nv + i];
  }
}

// element view of the trace operator: yv_k = S_k x[gmap_k]
template <typename T>
__global__ void __launch_bounds__(256) k_gen_matvec_elem(int Eim, const int* __restrict__ nTk,
                                                         const long long* __restrict__ offD,
                                                         const long long* __restrict__ offs,
                                                         const int* __restrict__ gmap, const T* __restrict__ S,
                                                         const double* __restrict__ x, double* __restrict__ yv,
                                                         const int* gate, int gj, long long nh) {
  // y_k = S_k x_k, one warp per implicit element: the element's gathered trace values staged in the
  // warp's shared memory, then 8 rows at a time with 4 lanes per row, each lane taking every 4th
  // 16-byte run of the row (FP32 rows of a multiple of 4 values on 16-byte boundaries; scalar
  // otherwise), a 4-lane sum per row
  __shared__ __align__(16) T xs[8][512];
  if (gate && *gate >= 0 && gj >= *gate) return;
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + wp;
  if (k >= Eim) return;
  const int nT = nTk[k];
  const T* Sk = S + offD[k];
  const int* gm = gmap + offs[k];
  T* xk = xs[wp];
  for (int l = lane; l < nT; l += 32) {
    const int g = gm[l];
    xk[l] = g >= 0 ? T(x[FR_IDX(g, nh, 8)]) : T(0);
  }
  __syncwarp();
  const int r8 = lane >> 2, c4 = lane & 3;
  const bool vec = sizeof(T) == 4 && (nT & 3) == 0 && (offD[k] & 3) == 0;
  for (int r0 = 0; r0 < nT; r0 += 8) {
    const int row = r0 + r8;
    T acc = T(0);
    if (row < nT) {
      const T* Sr = Sk + (size_t)row * nT;
      if (vec) {
        const float4* S4 = reinterpret_cast<const float4*>(Sr);
        const float4* x4 = reinterpret_cast<const float4*>(xk);
        for (int c = c4; c < (nT >> 2); c += 4) {
          const float4 sv = __ldg(S4 + c), xv = x4[c];
          acc += sv.x * xv.x + sv.y * xv.y + sv.z * xv.z + sv.w * xv.w;
        }
      } else {
        for (int l = c4; l < nT; l += 4) acc += Sr[l] * xk[l];
      }
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (c4 == 0 && row < nT) yv[offs[k] + row] = double(acc);
  }
}

// y[d] = the sum of the element-view values of trace value d (CSR over its entries)
__global__ void k_gen_gather_sum(size_t nh, const long long* __restrict__ vptr, const long long* __restrict__ vidx,
                                 const double* __restrict__ yv, double* __restrict__ y, const int* gate, int gj,
                                 long long nview) {
  if (gate && *gate >= 0 && gj >= *gate) return;
  const size_t d = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= nh) return;
  double s = 0.0;
  for (long long c = vptr[d]; c < vptr[d + 1]; ++c) s += yv[FR_IDX(vidx[c], nview, 7)];
  y[d] = s;
}

// EFR node-block Jacobi: P_i = sum over the element entries of node i of the nv x nv diagonal
// block of S_k at that entry, inverted by Gauss-Jordan with partial pivoting (one thread per node,
// FP64), stored in the block precision
template <typename T>
__global__ void k_gen_precond_build_node(size_t nnode, int nv, const long long* __restrict__ nptr,
                                         const int* __restrict__ nent_k, const int* __restrict__ nent_l,
                                         const int* __restrict__ nTk, const long long* __restrict__ offD,
                                         const T* __restrict__ S, T* __restrict__ Pinv, int* status) {
  const size_t node = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nnode) return;
  double W[5][10];
  for (int r = 0; r < nv; ++r)
    for (int c = 0; c < 2 * nv; ++c) W[r][c] = (c >= nv && c - nv == r) ? 1.0 : 0.0;
  for (long long e = nptr[node]; e < nptr[node + 1]; ++e) {
    const int k = nent_k[e], l = nent_l[e], nT = nTk[k];
    const T* Sk = S + offD[k];
    for (int r = 0; r < nv; ++r)
      for (int c = 0; c < nv; ++c) W[r][c] += double(Sk[(size_t)(l + r) * nT + l + c]);
  }
  for (int c = 0; c < nv; ++c) {
    int pr = c;
    double bv = fabs(W[c][c]);
    for (int r = c + 1; r < nv; ++r)
      if (fabs(W[r][c]) > bv) {
        bv = fabs(W[r][c]);
        pr = r;
      }
    if (!(bv > 0.0)) {
      atomicOr(status, DEV_ERR_SINGULAR);
      atomicMin(status + 1, -1);
      return;
    }
    if (pr != c)
      for (int x = 0; x < 2 * nv; ++x) {
        const double u = W[c][x];
        W[c][x] = W[pr][x];
        W[pr][x] = u;
      }
    const double inv = 1.0 / W[c][c];
    for (int x = 0; x < 2 * nv; ++x) W[c][x] *= inv;
    for (int r = 0; r < nv; ++r) {
      if (r == c) continue;
      const double l = W[r][c];
      for (int x = 0; x < 2 * nv; ++x) W[r][x] -= l * W[c][x];
    }
  }
  T* P = Pinv + node * nv * nv;
  for (int r = 0; r < nv; ++r)
    for (int c = 0; c < nv; ++c) P[r * nv + c] = T(W[r][nv + c]);
}

// face-block Jacobi: P_t = sum over the sides of the face's diagonal block of S_k, inverted in
// place in shared memory by Gauss-Jordan elimination with partial pivoting (row interchanges,
// undone at the end as column interchanges in reverse order), in the block precision T; one CTA
// of GP_THREADS per trace face, bs x bs values plus bs multipliers and bs pivot rows of shared memory
constexpr int GP_THREADS = 128;
template <typename T>
size_t precond_smem_bytes(int bsmax) {
  return ((size_t)bsmax * bsmax + bsmax) * sizeof(T) + (size_t)bsmax * sizeof(int);
}
template <typename T>
__global__ void __launch_bounds__(GP_THREADS) k_gen_precond_build(int ntrace, int nv, const int* __restrict__ tpts,
                                                                const long long* __restrict__ poff,
                                                                const int* __restrict__ pside,
                                                                const int* __restrict__ nTk,
                                                                const long long* __restrict__ offD,
                                                                const T* __restrict__ S, T* __restrict__ Pinv,
                                                                int* status) {
  extern __shared__ __align__(16) unsigned char gp_smem[];
  __shared__ int s_piv, s_bad;
  const int t = blockIdx.x, tid = threadIdx.x;
  if (t >= ntrace) return;
  const int bs = tpts[t] * nv;
  T* W = reinterpret_cast<T*>(gp_smem);  // bs x bs, row-major
  T* L = W + (size_t)bs * bs;             // multipliers of the current column
  int* perm = reinterpret_cast<int*>(L + bs);
  for (int i = tid; i < bs * bs; i += GP_THREADS) {
    const int r = i / bs, c = i % bs;
    T v = T(0);
    for (int sd = 0; sd < 2; ++sd) {
      const int kk = pside[4 * t + 2 * sd], lo = pside[4 * t + 2 * sd + 1];
      if (kk < 0) continue;
      const int nT = nTk[kk];
      v += S[offD[kk] + (size_t)(lo + r) * nT + lo + c];
    }
    W[i] = v;
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int c = 0; c < bs; ++c) {
    if (tid < 32) {
      T bv = T(-1);
      int bi = bs;
      for (int r = c + tid; r < bs; r += 32) {
        const T v = fabs(W[r * bs + c]);
        if (v > bv || (v == bv && r < bi)) {
          bv = v;
          bi = r;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (tid == 0) {
        s_piv = bi;
        perm[c] = bi;
        if (!(bv > T(0))) s_bad = 1;
      }
    }
    __syncthreads();
    if (s_bad) break;
    const int pv = s_piv;
    if (pv != c)
      for (int x = tid; x < bs; x += GP_THREADS) {
        const T u = W[c * bs + x];
        W[c * bs + x] = W[pv * bs + x];
        W[pv * bs + x] = u;
      }
    __syncthreads();
    const T inv = T(1) / W[c * bs + c];
    for (int r = tid; r < bs; r += GP_THREADS) L[r] = r == c ? T(0) : W[r * bs + c];
    __syncthreads();
    for (int x = tid; x < bs; x += GP_THREADS) W[c * bs + x] = (x == c ? T(1) : W[c * bs + x]) * inv;
    __syncthreads();
    for (int r = tid >> 5; r < bs; r += GP_THREADS / 32) {  // one warp per row, lanes along it
      if (r == c) continue;
      const T l = L[r];
      for (int x = tid & 31; x < bs; x += 32) W[r * bs + x] = (x == c ? T(0) : W[r * bs + x]) - l * W[c * bs + x];
    }
    __syncthreads();
  }
  if (s_bad) {
    if (tid == 0) {
      atomicOr(status, DEV_ERR_SINGULAR);
      atomicMin(status + 1, -1 - t);
    }
    return;
  }
  for (int c = bs - 1; c >= 0; --c) {
    const int pv = perm[c];
    if (pv != c)
      for (int r = tid; r < bs; r += GP_THREADS) {
        const T u = W[r * bs + c];
        W[r * bs + c] = W[r * bs + pv];
        W[r * bs + pv] = u;
      }
    __syncthreads();
  }
  T* P = Pinv + poff[t];
  for (int i = tid; i < bs * bs; i += GP_THREADS) P[i] = W[i];
}

// z_t = Pinv_t v_t (v first normalised in place by *inv_h when given); one warp per trace face
template <typename T>
__global__ void k_gen_precond_apply(int ntrace, int nv, const int* __restrict__ tpts, const long long* __restrict__ toff,
                                    const long long* __restrict__ poff, const T* __restrict__ Pinv,
                                    double* __restrict__ x, double* __restrict__ y, const int* gate, int gj,
                                    const double* inv_h, float* __restrict__ y32) {
  if (gate && *gate >= 0 && gj >= *gate) return;
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (t >= ntrace) return;
  const int bs = tpts[t] * nv;
  const long long o = toff[t];
  const T* P = Pinv + poff[t];
  // the product runs in the block precision (FP32 blocks: the FP32 pipe; the FP64 pipe of this
  // part is a small fraction of the FP32 one)
  T xl[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int i = lane + 32 * c;
    double v = i < bs ? x[o + i] : 0.0;
    if (inv_h && i < bs) {
      v *= *inv_h;
      x[o + i] = v;
    }
    xl[c] = T(v);
  }
  for (int row = 0; row < bs; ++row) {
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = lane + 32 * c;
      if (i < bs) acc += P[(size_t)row * bs + i] * xl[c];
    }
#pragma unroll
    for (int of = 16; of > 0; of >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, of);
    if (lane == 0) {
      y[o + row] = double(acc);
      if (y32) y32[o + row] = float(acc);
    }
  }
}

// the same for blocks of at most 8 values (EFR node blocks, bs = nv): one thread per trace unit
template <typename T>
__global__ void k_gen_precond_apply_small(int ntrace, int nv, const int* __restrict__ tpts,
                                          const long long* __restrict__ toff, const long long* __restrict__ poff,
                                          const T* __restrict__ Pinv, double* __restrict__ x, double* __restrict__ y,
                                          const int* gate, int gj, const double* inv_h, float* __restrict__ y32) {
  if (gate && *gate >= 0 && gj >= *gate) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntrace) return;
  const int bs = tpts[t] * nv;
  const long long o = toff[t];
  const T* P = Pinv + poff[t];
  const double sc = inv_h ? *inv_h : 1.0;
  T xl[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    double v = c < bs ? x[o + c] : 0.0;
    if (inv_h && c < bs) {
      v *= sc;
      x[o + c] = v;
    }
    xl[c] = T(v);
  }
  for (int r = 0; r < bs; ++r) {
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (c < bs) acc += P[(size_t)r * bs + c] * xl[c];
    y[o + r] = double(acc);
    if (y32) y32[o + r] = float(acc);
  }
}

// du_k = x_r - X_B du^_k, one warp per implicit element
template <typename T>
__global__ void k_gen_backsolve(int Eim, const int* __restrict__ nAk, const int* __restrict__ nTk,
                                const long long* __restrict__ offB, const long long* __restrict__ offr,
                                const long long* __restrict__ offs, const int* __restrict__ gmap,
                                const T* __restrict__ XB, const double* __restrict__ xr,
                                const double* __restrict__ duhat, double* __restrict__ du, long long nh) {
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= Eim) return;
  const int nA = nAk[k], nT = nTk[k];
  const T* X = XB + offB[k];
  const int* gm = gmap + offs[k];
  // the product in the block precision; x_r and the difference in FP64
  T dl[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const int l = lane + 32 * c;
    const int g = l < nT ? gm[l] : -1;
    dl[c] = g >= 0 ? T(duhat[FR_IDX(g, nh, 9)]) : T(0);
  }
  for (int i = 0; i < nA; ++i) {
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int l = lane + 32 * c;
      if (l < nT) acc += X[(size_t)i * nT + l] * dl[c];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) du[offr[k] + i] = xr[offr[k] + i] - double(acc);
  }
}

// u[uoff[e_k] + i] += du_k[i]
__global__ void k_gen_apply_du(int Eim, int nv, const int* __restrict__ imp_idx, const int* __restrict__ deg,
                               const long long* __restrict__ uoff, const long long* __restrict__ offr,
                               const double* __restrict__ du, double* __restrict__ U) {
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= Eim) return;
  const int e = imp_idx[k];
  const int nA = (int)(uoff[e + 1] - uoff[e]);
  (void)deg;
  (void)nv;
  for (int i = lane; i < nA; i += 32) U[uoff[e] + i] += du[offr[k] + i];
}

__global__ void k_gen_axpy(size_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

struct StageCoefG {
  int nterm;
  double ci[8], ce[8];
  int hi[8];
};
// out = base + sum_j c_j R_hist[h_j], per value with its element's implicit flag
__global__ void k_gen_stage_combine(size_t tot, const unsigned char* __restrict__ dof_imp,
                                    const double* __restrict__ base, const double* __restrict__ Rh, StageCoefG sc,
                                    double* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const bool im = dof_imp[i] != 0;
  double v = base[i];
  for (int jj = 0; jj < sc.nterm; ++jj) {
    const double c = im ? sc.ci[jj] : sc.ce[jj];
    if (c != 0.0) v += c * Rh[(size_t)sc.hi[jj] * tot + i];
  }
  out[i] = v;
}

__global__ void k_gen_sumsq_part(const double* __restrict__ a, size_t na, const double* __restrict__ b, size_t nb,
                                 double* __restrict__ partial) {
  __shared__ double red[8];
  double s = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < na + nb; x += stride) {
    const double v = x < na ? a[x] : b[x - na];
    s += v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    partial[blockIdx.x] = t;
  }
}
__global__ void k_gen_sumsq_final(const double* __restrict__ partial, int nblk, double* out) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  double t = 0.0;
  for (int i = lane; i < nblk; i += 32) t += partial[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) *out = t;
}

__global__ void k_gen_status_reset(int* status) {
  status[0] = 0;
  status[1] = 0x7fffffff;
}

// ------------------------------------------------------------------------ context

static int err(GenCtx* g, int code, const char* msg, int elem = -1, int it = -1, double val = 0.0) {
  if (g && g->hk.set_err) return g->hk.set_err(g->hk.owner, code, msg, elem, it, val);
  return code;
}
#define GCK(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) return err(g, FR_ERR_CUDA, cudaGetErrorString(e_));     \
  } while (0)
static int pbeg(GenCtx* g, int ph) {
  return (g->hk.prof_begin && !g->capturing) ? g->hk.prof_begin(g->hk.owner, ph) : -1;
}
static void pend(GenCtx* g, int h) {
  if (g->hk.prof_end) g->hk.prof_end(g->hk.owner, h);
}
static inline unsigned nb256(size_t n) { return (unsigned)((n + 255) / 256); }
static inline unsigned nbw(size_t nwarps, int wpb = 8) { return (unsigned)((nwarps + wpb - 1) / wpb); }

template <typename T>
static T* galloc(GenCtx* g, size_t count, int* rc) {
  if (count == 0) count = 1;
  void* p = nullptr;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    *rc = FR_ERR_OOM;
    return nullptr;
  }
  g->allocs.push_back(p);
  g->bytes += count * sizeof(T);
  return (T*)p;
}

bool mesh_is_general(const fr_mesh_desc* mesh) {
  if (!mesh) return false;
  if (mesh->elem_type == FR_ELEM_HEX) return true;
  if (mesh->p_elem)
    for (int e = 1; e < mesh->nelem; ++e)
      if (mesh->p_elem[e] != mesh->p_elem[0]) return true;
  if (mesh->nbr)
    for (long long i = 0; i < 4LL * mesh->nelem; ++i)
      if (mesh->nbr[i] < 0) return true;
  return false;
}

static void bilinear_g(const double* V, double xi, double eta, double* J, double S[2][2], double* xy) {
  const double sa[4] = {-1, 1, -1, 1}, sb[4] = {-1, -1, 1, 1};
  double xx = 0, xe = 0, yx = 0, ye = 0, px = 0, py = 0;
  for (int c = 0; c < 4; ++c) {
    const double dNx = 0.25 * sa[c] * (1 + sb[c] * eta), dNe = 0.25 * sb[c] * (1 + sa[c] * xi);
    const double Nc = 0.25 * (1 + sa[c] * xi) * (1 + sb[c] * eta);
    xx += dNx * V[2 * c];
    yx += dNx * V[2 * c + 1];
    xe += dNe * V[2 * c];
    ye += dNe * V[2 * c + 1];
    px += Nc * V[2 * c];
    py += Nc * V[2 * c + 1];
  }
  *J = xx * ye - xe * yx;
  S[0][0] = ye;
  S[0][1] = -xe;
  S[1][0] = -yx;
  S[1][1] = xx;
  if (xy) {
    xy[0] = px;
    xy[1] = py;
  }
}

void destroy(GenCtx* g) {
  if (!g) return;
  if (g->gexec) cudaGraphExecDestroy(g->gexec);
  if (g->graph) cudaGraphDestroy(g->graph);
  for (auto& c : g->cap)
    if (c) cudaStreamDestroy(c);
  for (void* p : g->allocs) cudaFree(p);
  delete g;
}

int create(const fr_mesh_desc* mesh, const fr_config* cfg, cudaStream_t st, const Hooks& hooks, GenCtx** out) {
  *out = nullptr;
  const int E = mesh->nelem;
  if (cfg->physics != FR_PHYS_ADVDIFF && cfg->physics != FR_PHYS_NAVIER_STOKES) return FR_ERR_UNSUPPORTED;
  if (cfg->precision != FR_PREC_FP64 && cfg->precision != FR_PREC_FP32) return FR_ERR_UNSUPPORTED;
  const bool hex = mesh->elem_type == FR_ELEM_HEX;
  const bool efr = cfg->trace_kind == FR_TRACE_EFR;
  if (cfg->trace_kind != FR_TRACE_HFR && cfg->trace_kind != FR_TRACE_EFR) return FR_ERR_INVALID_ARG;
  if (efr && hex) return FR_ERR_UNSUPPORTED;  // EFR: quadrilaterals
  if (hex && cfg->physics != FR_PHYS_NAVIER_STOKES) return FR_ERR_UNSUPPORTED;  // hexahedra: Navier-Stokes
  const int DIM = hex ? 3 : 2, NF = hex ? 6 : 4, FS = hex ? HEX_FS : GN, NC = hex ? 8 : 4;
  const int nv = cfg->physics == FR_PHYS_ADVDIFF ? 1 : (hex ? 5 : 4);
  std::vector<int> deg(E);
  for (int e = 0; e < E; ++e) {
    const int p = mesh->p_elem ? mesh->p_elem[e] : mesh->p;
    if (p < 1 || p > (hex ? HEX_PMAX : 5)) return FR_ERR_UNSUPPORTED;
    if ((hex || efr) && p != (mesh->p_elem ? mesh->p_elem[0] : mesh->p)) return FR_ERR_UNSUPPORTED;  // one degree
    deg[e] = p + 1;
  }
  // connectivity, face kinds, face point counts
  std::vector<int> kind(NF * (size_t)E), nfp(NF * (size_t)E), nbr(NF * (size_t)E), nbf(NF * (size_t)E);
  bool need_nbr = false;
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < NF; ++f) {
      const size_t i = NF * (size_t)e + f;
      const int nb = mesh->nbr[i], nf = mesh->nbr_face[i], id = mesh->face_of[i];
      const bool ie = mesh->implicit[e] != 0;
      if (id < 0 || (long long)id >= (long long)NF * E) return FR_ERR_INVALID_ARG;
      if (nb < 0) {
        const int bc = mesh->bc ? mesh->bc[i] : 0;
        if (bc == BC_WALL) {
          if (!ie || cfg->physics != FR_PHYS_NAVIER_STOKES) return FR_ERR_UNSUPPORTED;  // explicit walls: not built
          kind[i] = FK_WALL;
        } else if (bc == BC_FAR) {
          kind[i] = FK_FAR;
          if (!ie) need_nbr = true;
        } else {
          return FR_ERR_INVALID_ARG;
        }
        nbr[i] = -1;
        nbf[i] = -1;
        nfp[i] = hex ? deg[e] * deg[e] : deg[e];
        continue;
      }
      if (nb >= E || nf < 0 || nf >= NF || mesh->nbr[NF * (size_t)nb + nf] != e || mesh->nbr_face[NF * (size_t)nb + nf] != f ||
          mesh->face_of[NF * (size_t)nb + nf] != id)
        return FR_ERR_INVALID_ARG;
      const bool in = mesh->implicit[nb] != 0;
      kind[i] = (ie && in) ? FK_TRACE : (ie != in ? FK_IMEX : FK_FR);
      if (kind[i] != FK_TRACE) need_nbr = true;
      nbr[i] = nb;
      nbf[i] = nf;
      nfp[i] = hex ? deg[e] * deg[e] : std::max(deg[e], deg[nb]);
    }
  GenCtx* g = new GenCtx();
  g->hk = hooks;
  g->st = st;
  g->E = E;
  g->nv = nv;
  g->pb = cfg->precision == FR_PREC_FP64 ? 8 : 4;
  g->tableau = cfg->tableau;
  g->restart = cfg->gmres_restart > 0 ? std::min(cfg->gmres_restart, GM_MAXM) : 30;
  g->need_nbr = need_nbr;
  g->has_explicit = need_nbr;
  memset(&g->pp, 0, sizeof(g->pp));
  g->pp.kind = hex ? 3 : cfg->physics;
  g->dim = DIM;
  g->nface = NF;
  g->fs = FS;
  g->efr = efr ? 1 : 0;
  // EFR: interior trace faces carry the Gauss-Lobatto points (n of them: one degree)
  std::vector<unsigned char> fset(NF * (size_t)E, 0);
  if (efr)
    for (size_t i = 0; i < fset.size(); ++i) fset[i] = kind[i] == FK_TRACE ? 1 : 0;
  g->pp.beta[0] = cfg->beta[0];
  g->pp.beta[1] = cfg->beta[1];
  g->pp.nu = cfg->nu;
  g->pp.gamma = cfg->gamma;
  g->pp.mu = cfg->mu;
  g->pp.Pr = cfg->Pr;
  g->pp.lref = cfg->lref > 0 ? cfg->lref : 1.0;
  for (int v = 0; v < 5; ++v) g->uinf[v] = cfg->u_inf[v];
  g->h_deg = deg;
  // trace units.  HFR: the trace faces (both sides implicit, or a boundary face of an implicit
  // element) in increasing global face id, each with its face points.  EFR: the trace nodes
  // (vertices of the implicit skeleton, interior Gauss-Lobatto points of the trace faces, the
  // Gauss points of boundary trace faces; efr_trace_nodes), one point each.  fnode: the trace
  // point of every element face point.
  std::vector<int> tr_of(NF * (size_t)E, -1), tpts, sides, fnode(NF * (size_t)E * FS, -1);
  int nt = 0;
  if (efr) {
    const int n0 = deg[0];
    std::vector<int> node_of((size_t)E * 4 * n0);
    int nvert = 0, nnode = 0;
    const int lrc = efr_trace_nodes(E, mesh->nbr, mesh->nbr_face, mesh->face_of, mesh->bc, mesh->implicit, n0 - 1,
                                    node_of.data(), &nvert, &nnode);
    if (lrc != FR_OK) {
      destroy(g);
      return lrc;
    }
    nt = nnode;
    tpts.assign(nt, 1);
    for (int e = 0; e < E; ++e)
      for (int f = 0; f < NF; ++f) {
        const size_t i = NF * (size_t)e + f;
        if (node_of[i * n0] < 0) continue;
        tr_of[i] = node_of[i * n0];  // a face with a trace (its first node)
        for (int q = 0; q < n0; ++q) fnode[i * FS + q] = node_of[i * n0 + q];
      }
  } else {
    std::vector<int> tr_of_fid(NF * (size_t)E, -1), pts_of_fid(NF * (size_t)E, 0);
    for (int e = 0; e < E; ++e)
      for (int f = 0; f < NF; ++f) {
        const size_t i = NF * (size_t)e + f;
        if (kind[i] == FK_TRACE || (nbr[i] < 0 && mesh->implicit[e])) {
          tr_of_fid[mesh->face_of[i]] = 0;
          pts_of_fid[mesh->face_of[i]] = nfp[i];
        }
      }
    for (size_t id = 0; id < tr_of_fid.size(); ++id)
      if (tr_of_fid[id] == 0) {
        tr_of_fid[id] = nt++;
        tpts.push_back(pts_of_fid[id]);
      }
    sides.assign(4 * (size_t)std::max(nt, 1), -1);
    std::vector<long long> tpt0(nt + 1, 0);
    for (int t = 0; t < nt; ++t) tpt0[t + 1] = tpt0[t] + tpts[t];
    for (int e = 0; e < E; ++e)
      for (int f = 0; f < NF; ++f) {
        const size_t i = NF * (size_t)e + f;
        if (kind[i] == FK_TRACE || (nbr[i] < 0 && mesh->implicit[e])) {
          const int t = tr_of_fid[mesh->face_of[i]];
          tr_of[i] = t;
          const int slot = sides[4 * (size_t)t] < 0 ? 0 : 1;
          sides[4 * (size_t)t + 2 * slot] = e;
          sides[4 * (size_t)t + 2 * slot + 1] = f;
          for (int q = 0; q < nfp[i]; ++q) fnode[i * FS + q] = (int)(tpt0[t] + q);
        }
      }
  }
  g->ntrace = nt;
  std::vector<long long> toff(nt + 1, 0);
  for (int t = 0; t < nt; ++t) toff[t + 1] = toff[t] + (long long)tpts[t] * nv;
  g->nh = (size_t)toff[nt];
  g->npts = g->nh / nv;
  // trace point <- element face points (CSR, element order)
  std::vector<long long> gptr(g->npts + 1, 0), gidx;
  for (size_t i = 0; i < fnode.size(); ++i)
    if (fnode[i] >= 0) ++gptr[fnode[i] + 1];
  for (size_t q = 0; q < g->npts; ++q) gptr[q + 1] += gptr[q];
  gidx.assign(std::max((size_t)gptr[g->npts], (size_t)1), 0);
  {
    std::vector<long long> fill(gptr.begin(), gptr.end() - 1);
    for (size_t i = 0; i < fnode.size(); ++i)
      if (fnode[i] >= 0) gidx[fill[fnode[i]]++] = (long long)i;
  }
  // state offsets, implicit blocks
  std::vector<long long> uoff(E + 1, 0), goff(E + 1, 0);
  for (int e = 0; e < E; ++e) {
    const long long ns = hex ? (long long)deg[e] * deg[e] * deg[e] : (long long)deg[e] * deg[e];
    uoff[e + 1] = uoff[e] + ns * nv;
    goff[e + 1] = goff[e] + ns;
    g->pmax = std::max(g->pmax, deg[e] - 1);
  }
  g->nstate = (size_t)uoff[E];
  std::vector<int> imp_idx, exp_idx, comp(E, -1);
  for (int e = 0; e < E; ++e)
    if (mesh->implicit[e]) {
      comp[e] = (int)imp_idx.size();
      imp_idx.push_back(e);
    } else {
      exp_idx.push_back(e);
    }
  g->Eex = (int)exp_idx.size();
  const int Eim = (int)imp_idx.size();
  g->Eim = Eim;
  std::vector<int> nAk(std::max(Eim, 1)), nTk(std::max(Eim, 1)), lto(NF * (size_t)std::max(Eim, 1));
  std::vector<long long> offA(Eim + 1, 0), offB(Eim + 1, 0), offD(Eim + 1, 0), offr(Eim + 1, 0), offs(Eim + 1, 0);
  for (int k = 0; k < Eim; ++k) {
    const int e = imp_idx[k];
    nAk[k] = (int)(uoff[e + 1] - uoff[e]);
    int o = 0;
    for (int f = 0; f < NF; ++f) {
      lto[NF * (size_t)k + f] = o;
      o += nfp[NF * (size_t)e + f] * nv;
    }
    nTk[k] = o;
    if (o > 512 || nAk[k] > 32 * 5 * (hex ? 2 : 1)) {
      destroy(g);
      return FR_ERR_UNSUPPORTED;
    }
    offA[k + 1] = offA[k] + (long long)nAk[k] * nAk[k];
    offB[k + 1] = offB[k] + (long long)nAk[k] * nTk[k];
    offD[k + 1] = offD[k] + (long long)nTk[k] * nTk[k];
    offr[k + 1] = offr[k] + nAk[k];
    offs[k + 1] = offs[k] + nTk[k];
    g->maxA = std::max(g->maxA, nAk[k]);
    g->maxT = std::max(g->maxT, nTk[k]);
  }
  g->sumA = (size_t)offr[Eim];
  g->sumT = (size_t)offs[Eim];
  g->sumAA = (size_t)offA[Eim];
  g->sumAT = (size_t)offB[Eim];
  g->sumTT = (size_t)offD[Eim];
  g->h_nA.assign(nAk.begin(), nAk.begin() + Eim);
  g->h_nT.assign(nTk.begin(), nTk.begin() + Eim);
  // gather map (element-local trace unknown -> trace value) and its inverse (CSR, element order);
  // HFR face blocks: the two sides' local offsets; EFR node blocks: every entry of each node
  std::vector<int> gmap(std::max(g->sumT, (size_t)1), -1);
  std::vector<int> pside(4 * (size_t)std::max(nt, 1), -1);
  std::vector<long long> vptr(g->nh + 1, 0), nptr(efr ? g->npts + 1 : 1, 0);
  for (int k = 0; k < Eim; ++k) {
    const int e = imp_idx[k];
    for (int f = 0; f < NF; ++f) {
      const size_t i = NF * (size_t)e + f;
      const int t = tr_of[i];
      if (t < 0) continue;
      if (!efr) {
        const int sd = sides[4 * (size_t)t] == e && sides[4 * (size_t)t + 1] == f ? 0 : 1;
        pside[4 * (size_t)t + 2 * sd] = k;
        pside[4 * (size_t)t + 2 * sd + 1] = lto[NF * (size_t)k + f];
      }
      for (int q = 0; q < nfp[i]; ++q) {
        const int pt = fnode[i * FS + q];
        if (efr) ++nptr[pt + 1];
        for (int v = 0; v < nv; ++v) {
          const long long l = offs[k] + lto[NF * (size_t)k + f] + q * nv + v;
          gmap[l] = pt * nv + v;
          ++vptr[(size_t)pt * nv + v + 1];
        }
      }
    }
  }
  for (size_t d = 0; d < g->nh; ++d) vptr[d + 1] += vptr[d];
  std::vector<long long> vidx(std::max((size_t)vptr[g->nh], (size_t)1), 0);
  {
    std::vector<long long> fill(vptr.begin(), vptr.end() - 1);
    for (size_t l = 0; l < g->sumT; ++l)
      if (gmap[l] >= 0) vidx[fill[gmap[l]]++] = (long long)l;
  }
  for (size_t q = 0; efr && q < g->npts; ++q) nptr[q + 1] += nptr[q];
  std::vector<int> nent_k(efr ? std::max((size_t)nptr[g->npts], (size_t)1) : 1, 0), nent_l(nent_k.size(), 0);
  if (efr) {
    std::vector<long long> fill(nptr.begin(), nptr.end() - 1);
    for (int k = 0; k < Eim; ++k) {
      const int e = imp_idx[k];
      for (int f = 0; f < NF; ++f) {
        const size_t i = NF * (size_t)e + f;
        if (tr_of[i] < 0) continue;
        for (int q = 0; q < nfp[i]; ++q) {
          const int pt = fnode[i * FS + q];
          nent_k[fill[pt]] = k;
          nent_l[fill[pt]++] = lto[NF * (size_t)k + f] + q * nv;
        }
      }
    }
  }
  std::vector<long long> poff(nt + 1, 0);
  for (int t = 0; t < nt; ++t) poff[t + 1] = poff[t] + (long long)(tpts[t] * nv) * (tpts[t] * nv);
  g->sumP = (size_t)poff[nt];
  g->bsmax = 0;
  for (int t = 0; t < nt; ++t) g->bsmax = std::max(g->bsmax, tpts[t] * nv);
  if (!efr && nt > 0) {
    const size_t sm = g->pb == 8 ? precond_smem_bytes<double>(g->bsmax) : precond_smem_bytes<float>(g->bsmax);
    const cudaError_t ea = g->pb == 8 ? cudaFuncSetAttribute(k_gen_precond_build<double>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                                   : cudaFuncSetAttribute(k_gen_precond_build<float>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (ea != cudaSuccess) {
      destroy(g);
      return FR_ERR_UNSUPPORTED;
    }
  }
  // geometry at the own solution points and at every face's points
  const int GS = hex ? 10 : 5, GFC = hex ? 4 : 3;  // values per solution point / face point
  std::vector<double> gsol(GS * (size_t)goff[E]), gface(GFC * NF * (size_t)E * FS, 0.0);
  g->xy.assign(DIM * (size_t)goff[E], 0.0);
  if (hex)
    hex_geometry(mesh->verts, E, deg.data(), goff.data(), gsol.data(), gface.data(), g->xy.data());
  else
    for (int e = 0; e < E; ++e) {
    const int n = deg[e];
    double xg[GN], wg[GN];
    gauss_legendre_nodes(n, xg, wg);
    const double* V = mesh->verts + (size_t)e * 2 * NC;
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        const size_t pt = (size_t)goff[e] + a + n * b;
        double J, S[2][2];
        bilinear_g(V, xg[a], xg[b], &J, S, &g->xy[2 * pt]);
        double* G = &gsol[5 * pt];
        G[0] = 1.0 / J;
        G[1] = S[0][0];
        G[2] = S[0][1];
        G[3] = S[1][0];
        G[4] = S[1][1];
      }
    for (int f = 0; f < NF; ++f) {
      const int m = nfp[NF * (size_t)e + f], r = f >> 1;
      const double sg = (f & 1) ? 1.0 : -1.0;
      double sq[GN], wq[GN];
      if (fset[NF * (size_t)e + f])
        gauss_lobatto_nodes(m, sq, wq);
      else
        gauss_legendre_nodes(m, sq, wq);
      for (int q = 0; q < m; ++q) {
        const double xi = r == 0 ? sg : sq[q], eta = r == 0 ? sq[q] : sg;
        double J, S[2][2];
        bilinear_g(V, xi, eta, &J, S, nullptr);
        const double N0 = sg * S[r][0], N1 = sg * S[r][1];
        const double Jf = sqrt(N0 * N0 + N1 * N1);
        double* G = &gface[3 * ((size_t)(NF * e + f) * FS + q)];
        G[0] = Jf;
        G[1] = N0 / Jf;
        G[2] = N1 / Jf;
      }
    }
  }
  std::vector<unsigned char> dof_imp(std::max(g->nstate, (size_t)1), 0), impv(mesh->implicit, mesh->implicit + E);
  (void)NC;
  for (int e = 0; e < E; ++e)
    if (mesh->implicit[e])
      for (long long i = uoff[e]; i < uoff[e + 1]; ++i) dof_imp[i] = 1;
  GenRef href;
  build_genref(href);
  // condensation tables: FP32 quadrilateral shapes with a tensor-core form go by class (skipped
  // by the uneven launch)
  std::vector<unsigned char> tc_skip(std::max(Eim, 1), 0);
  std::vector<std::pair<std::pair<int, int>, std::vector<int>>> tc_cls;
  if (g->pb == 4 && !hex)
    for (int k = 0; k < Eim; ++k) {
      if (condense_tc_available(4, nAk[k], nTk[k]) < 2) continue;
      size_t c = 0;
      while (c < tc_cls.size() && tc_cls[c].first != std::make_pair(nAk[k], nTk[k])) ++c;
      if (c == tc_cls.size()) tc_cls.push_back({{nAk[k], nTk[k]}, {}});
      tc_cls[c].second.push_back(k);
      tc_skip[k] = 1;
    }
  UnevenTables tb;
  if (Eim > 0 && uneven_tables(g->pb, Eim, nAk.data(), nTk.data(), &tb, tc_skip.data()) != 0) {
    destroy(g);
    return FR_ERR_INVALID_ARG;
  }
  // device memory
  int rc = FR_OK;
  const size_t pb = g->pb;
  g->ref = galloc<GenRef>(g, 1, &rc);
  g->deg = galloc<int>(g, E, &rc);
  g->nbr = galloc<int>(g, NF * (size_t)E, &rc);
  g->nbr_face = galloc<int>(g, NF * (size_t)E, &rc);
  g->kind = galloc<int>(g, NF * (size_t)E, &rc);
  g->tr_of = galloc<int>(g, NF * (size_t)E, &rc);
  g->nfp = galloc<int>(g, NF * (size_t)E, &rc);
  g->uoff = galloc<long long>(g, E + 1, &rc);
  g->goff = galloc<long long>(g, E + 1, &rc);
  g->toff = galloc<long long>(g, nt + 1, &rc);
  g->geo_sol = galloc<double>(g, gsol.size(), &rc);
  g->geo_face = galloc<double>(g, gface.size(), &rc);
  g->implicit = galloc<unsigned char>(g, E, &rc);
  g->dof_imp = galloc<unsigned char>(g, dof_imp.size(), &rc);
  g->tpts = galloc<int>(g, std::max(nt, 1), &rc);
  g->sides = galloc<int>(g, std::max(sides.size(), (size_t)1), &rc);
  g->pside = galloc<int>(g, pside.size(), &rc);
  g->poff = galloc<long long>(g, nt + 1, &rc);
  g->imp_idx = galloc<int>(g, std::max(Eim, 1), &rc);
  g->exp_list = galloc<int>(g, std::max(g->Eex, 1), &rc);
  g->lto = galloc<int>(g, lto.size(), &rc);
  g->nAk = galloc<int>(g, nAk.size(), &rc);
  g->nTk = galloc<int>(g, nTk.size(), &rc);
  g->gmap = galloc<int>(g, gmap.size(), &rc);
  g->fnode = galloc<int>(g, fnode.size(), &rc);
  g->fset = galloc<unsigned char>(g, fset.size(), &rc);
  g->gptr = galloc<long long>(g, gptr.size(), &rc);
  g->gidx = galloc<long long>(g, gidx.size(), &rc);
  g->vptr = galloc<long long>(g, vptr.size(), &rc);
  g->vidx = galloc<long long>(g, vidx.size(), &rc);
  g->nptr = galloc<long long>(g, nptr.size(), &rc);
  g->nent_k = galloc<int>(g, nent_k.size(), &rc);
  g->nent_l = galloc<int>(g, nent_l.size(), &rc);
  g->offA = galloc<long long>(g, Eim + 1, &rc);
  g->offB = galloc<long long>(g, Eim + 1, &rc);
  g->offD = galloc<long long>(g, Eim + 1, &rc);
  g->offr = galloc<long long>(g, Eim + 1, &rc);
  g->offs = galloc<long long>(g, Eim + 1, &rc);
  if (need_nbr) {
    g->Uf_all = galloc<double>(g, NF * (size_t)E * FS * nv, &rc);
    g->qf_all = galloc<double>(g, NF * (size_t)E * FS * DIM * nv, &rc);
  }
  g->Rw = galloc<double>(g, g->nstate, &rc);
  g->gview = galloc<double>(g, NF * (size_t)E * FS * nv, &rc);
  g->gw = galloc<double>(g, g->nh, &rc);
  g->Ustar = galloc<double>(g, g->nstate, &rc);
  g->r = galloc<double>(g, g->sumA, &rc);
  g->s = galloc<double>(g, g->sumT, &rc);
  g->xr = galloc<double>(g, g->sumA, &rc);
  g->te = galloc<double>(g, g->sumT, &rc);
  g->tg = galloc<double>(g, g->nh, &rc);
  g->yv = galloc<double>(g, g->sumT, &rc);
  g->duhat = galloc<double>(g, g->nh, &rc);
  g->du = galloc<double>(g, g->sumA, &rc);
  g->red = galloc<double>(g, 1024 + 8, &rc);
  g->A = galloc<unsigned char>(g, g->sumAA * pb, &rc);
  g->B = galloc<unsigned char>(g, g->sumAT * pb, &rc);
  g->C = galloc<unsigned char>(g, g->sumAT * pb, &rc);
  g->D = galloc<unsigned char>(g, g->sumTT * pb, &rc);
  g->LU = galloc<unsigned char>(g, g->sumAA * pb, &rc);
  g->XB = galloc<unsigned char>(g, g->sumAT * pb, &rc);
  g->S = galloc<unsigned char>(g, g->sumTT * pb, &rc);
  g->Pinv = galloc<unsigned char>(g, g->sumP * pb, &rc);
  g->piv = galloc<int>(g, g->sumA, &rc);
  g->status = galloc<int>(g, 2, &rc);
  void* ubuf = Eim > 0 ? galloc<unsigned char>(g, uneven_dev_bytes(tb), &rc) : nullptr;
  g->gm.n = g->nh;
  g->gm.V = galloc<double>(g, (size_t)(GM_MAXM + 1) * std::max(g->nh, (size_t)1), &rc);
  g->gm.Z = galloc<double>(g, (size_t)GM_MAXM * std::max(g->nh, (size_t)1), &rc);
  g->gm.z32 = nullptr;
  g->gm.partial = galloc<double>(g, (size_t)GM_NBLK * (GM_MAXM + 1), &rc);
  g->gm.ticket = galloc<unsigned int>(g, 1, &rc);
  g->gm.state = galloc<GmresState>(g, 1, &rc);
  if (hex && Eim > 0) {
    g->jgrid = std::min(hex_jacobian_grid((int)pb), Eim);
    g->jscratch = galloc<unsigned char>(g, hex_jacobian_scratch_bytes((int)pb, g->jgrid), &rc);
  }
  if (rc != FR_OK) {
    destroy(g);
    return rc;
  }
#define GUP(dst, src, cnt)                                                                              \
  if ((cnt) > 0 && cudaMemcpyAsync(dst, src, (cnt) * sizeof(*(src)), cudaMemcpyHostToDevice, st) != cudaSuccess) { \
    destroy(g);                                                                                         \
    return FR_ERR_CUDA;                                                                                 \
  }
  GUP(g->ref, &href, 1);
  GUP(g->deg, deg.data(), (size_t)E);
  GUP(g->nbr, nbr.data(), nbr.size());
  GUP(g->nbr_face, nbf.data(), nbf.size());
  GUP(g->kind, kind.data(), kind.size());
  GUP(g->tr_of, tr_of.data(), tr_of.size());
  GUP(g->nfp, nfp.data(), nfp.size());
  GUP(g->uoff, uoff.data(), uoff.size());
  GUP(g->goff, goff.data(), goff.size());
  GUP(g->toff, toff.data(), toff.size());
  GUP(g->geo_sol, gsol.data(), gsol.size());
  GUP(g->geo_face, gface.data(), gface.size());
  GUP(g->implicit, impv.data(), impv.size());
  GUP(g->dof_imp, dof_imp.data(), dof_imp.size());
  GUP(g->tpts, tpts.data(), tpts.size());
  if (!sides.empty()) GUP(g->sides, sides.data(), sides.size());
  GUP(g->pside, pside.data(), pside.size());
  GUP(g->poff, poff.data(), poff.size());
  GUP(g->imp_idx, imp_idx.data(), imp_idx.size());
  if (!exp_idx.empty()) GUP(g->exp_list, exp_idx.data(), exp_idx.size());
  GUP(g->lto, lto.data(), lto.size());
  GUP(g->nAk, nAk.data(), nAk.size());
  GUP(g->nTk, nTk.data(), nTk.size());
  GUP(g->gmap, gmap.data(), gmap.size());
  GUP(g->fnode, fnode.data(), fnode.size());
  GUP(g->fset, fset.data(), fset.size());
  GUP(g->gptr, gptr.data(), gptr.size());
  GUP(g->gidx, gidx.data(), gidx.size());
  GUP(g->vptr, vptr.data(), vptr.size());
  GUP(g->vidx, vidx.data(), vidx.size());
  GUP(g->nptr, nptr.data(), nptr.size());
  GUP(g->nent_k, nent_k.data(), nent_k.size());
  GUP(g->nent_l, nent_l.data(), nent_l.size());
  GUP(g->offA, offA.data(), offA.size());
  GUP(g->offB, offB.data(), offB.size());
  GUP(g->offD, offD.data(), offD.size());
  GUP(g->offr, offr.data(), offr.size());
  GUP(g->offs, offs.data(), offs.size());
#undef GUP
  if (Eim > 0 && uneven_upload(tb, ubuf, &g->udev, st) != cudaSuccess) {
    destroy(g);
    return FR_ERR_CUDA;
  }
  g->udev.colmajor = hex ? 1 : 0;
  // class lists and one scratch batch for the largest class chunk
  {
    constexpr int CLASS_CAP = 16384;
    size_t sbytes = 0;
    for (auto& c : tc_cls) {
      GenCtx::TcClass tc;
      tc.nA = c.first.first;
      tc.nT = c.first.second;
      tc.count = (int)c.second.size();
      const int kf = c.second.front(), kl = c.second.back();
      if (kl - kf + 1 == tc.count) {  // increasing ids: consecutive exactly when the span matches
        tc.k0 = kf;
        tc.off0[0] = offA[kf];
        tc.off0[1] = offB[kf];
        tc.off0[2] = offD[kf];
        tc.off0[3] = offr[kf];
        tc.off0[4] = offs[kf];
      }
      tc.list = galloc<int>(g, c.second.size(), &rc);
      if (rc != FR_OK || cudaMemcpyAsync(tc.list, c.second.data(), c.second.size() * sizeof(int),
                                         cudaMemcpyHostToDevice, st) != cudaSuccess) {
        destroy(g);
        return rc != FR_OK ? rc : FR_ERR_CUDA;
      }
      g->tc_classes.push_back(tc);
      if (tc.k0 < 0) g->ccap = std::max(g->ccap, std::min(tc.count, CLASS_CAP));
    }
    for (auto& tc : g->tc_classes)
      sbytes = std::max(sbytes, tc.k0 < 0 ? class_scratch_bytes(tc.nA, tc.nT, g->ccap) : (size_t)64);
    if (sbytes) {
      g->cscratch = galloc<unsigned char>(g, sbytes, &rc);
      if (rc != FR_OK || class_scratch_init_status(g->cscratch, st) != cudaSuccess) {
        destroy(g);
        return rc != FR_OK ? rc : FR_ERR_CUDA;
      }
    }
  }
  if (cudaMemsetAsync(g->status, 0, 2 * sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(g->gm.ticket, 0, sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(g->gview, 0, NF * (size_t)E * FS * nv * sizeof(double), st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    destroy(g);
    return FR_ERR_CUDA;
  }
  g->h_uoff = uoff;
  g->h_toff = toff;
  *out = g;
  return FR_OK;
}

void query(const GenCtx* g, fr_ctx_info* info) {
  info->nelem = g->E;
  info->nimplicit = g->Eim;
  info->p = g->pmax;
  info->n = g->pmax + 1;
  info->ns = g->dim == 3 ? info->n * info->n * info->n : info->n * info->n;
  info->nv = g->nv;
  info->nA = g->maxA;
  info->nT = g->maxT;
  info->ntrace = g->ntrace;
  info->nstages = g->tableau == FR_TAB_SDIRK2 ? 2 : 1;
  info->has_explicit = g->has_explicit ? 1 : 0;
  info->workspace_bytes = g->bytes;
  info->general = 1;
  info->state_values = g->nstate;
  info->trace_values = g->nh;
  info->face_points = g->nface * g->E * g->fs;
}

int nstages(const GenCtx* g) { return g->tableau == FR_TAB_SDIRK2 ? 2 : 1; }
size_t state_values(const GenCtx* g) { return g->nstate; }

int layout(const GenCtx* g, long long* elem_off, long long* trace_off, int* blk_nA, int* blk_nT) {
  if (elem_off) memcpy(elem_off, g->h_uoff.data(), sizeof(long long) * (g->E + 1));
  if (trace_off) memcpy(trace_off, g->h_toff.data(), sizeof(long long) * (g->ntrace + 1));
  if (blk_nA && g->Eim) memcpy(blk_nA, g->h_nA.data(), sizeof(int) * g->Eim);
  if (blk_nT && g->Eim) memcpy(blk_nT, g->h_nT.data(), sizeof(int) * g->Eim);
  return FR_OK;
}

int solution_points(GenCtx* g, double* xy) {
  GCK(cudaMemcpyAsync(xy, g->xy.data(), g->xy.size() * sizeof(double), cudaMemcpyHostToDevice, g->st));
  GCK(cudaStreamSynchronize(g->st));
  return FR_OK;
}

static GArgs gargs(GenCtx* g, const double* u, const double* uhat) {
  GArgs a;
  memset(&a, 0, sizeof(a));
  a.E = g->E;
  a.deg = g->deg;
  a.uoff = g->uoff;
  a.goff = g->goff;
  a.geo_sol = g->geo_sol;
  a.geo_face = g->geo_face;
  a.nbr = g->nbr;
  a.nbr_face = g->nbr_face;
  a.kind = g->kind;
  a.tr_of = g->tr_of;
  a.nfp = g->nfp;
  a.toff = g->toff;
  a.implicit = g->implicit;
  a.ref = g->ref;
  a.U = u;
  a.uhat = uhat;
  a.Uf_all = g->Uf_all;
  a.qf_all = g->qf_all;
  a.Uf_out = g->Uf_all;
  a.qf_out = g->qf_all;
  for (int v = 0; v < 5; ++v) a.uinf[v] = g->uinf[v];
  a.nface = g->nface;
  a.fs = g->fs;
  a.fnode = g->fnode;
  a.fset = g->fset;
  a.npts = (long long)g->npts;
  return a;
}

template <int PHYS, int MODE>
static cudaError_t launch_gen_elem(GenCtx* g, const GArgs& a) {
  constexpr int NV = Phys<PHYS>::NV;
  const size_t smem = sizeof(GWork<NV>) * GEPB;
  auto kern = k_gen_elem<PHYS, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = ((a.elist ? a.nlist : a.E) + GEPB - 1) / GEPB;
  if (grid == 0) return cudaSuccess;
  (count_launch(), kern<<<grid, 32 * GEPB, smem, g->st>>>(g->pp, a));
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t gen_elem(GenCtx* g, const GArgs& a) {
  if (g->dim == 3) return hex_elem_pass(g, a, MODE);
  return g->pp.kind == 0 ? launch_gen_elem<0, MODE>(g, a) : launch_gen_elem<1, MODE>(g, a);
}

// R, the element trace rows (gview) and, if g_out, the assembled trace residual
static int residual_into(GenCtx* g, const double* u, const double* uhat, double* R, double* g_out) {
  const int ph = pbeg(g, 0);
  GArgs a = gargs(g, u, uhat);
  if (g->need_nbr) {
    GCK(gen_elem<GM_UF>(g, a));
    GCK(gen_elem<GM_QF>(g, a));
  }
  a.R = R;
  a.gview = g->gview;
  GCK(gen_elem<GM_RES>(g, a));
  if (g_out && g->ntrace) {
    (count_launch(), k_gen_trace_sum<<<nb256(g->nh), 256, 0, g->st>>>(g->npts, g->nv, g->gptr, g->gidx, g->gview,
                                                                       g_out, (long long)g->nface * g->E * g->fs));
    GCK(cudaGetLastError());
  }
  pend(g, ph);
  return FR_OK;
}

// The residual inside the Newton loop of a stage.  The explicit elements' states are fixed during
// the loop, and so are their face states and gradients: an implicit element reads them at its
// interface faces, while an explicit element takes its own state there.  So the explicit
// elements' face passes run once before the loop (stage_res_prepare), each Newton iterate
// evaluates the implicit elements alone (stage_res_newton: R and the trace rows), and once the loop
// ends the implicit elements' face passes and the explicit elements' residual at the final state
// complete R (stage_res_finish), as a full residual_into would.
static GArgs gargs_list(GenCtx* g, const double* u, const double* uhat, const int* list, int n) {
  GArgs a = gargs(g, u, uhat);
  a.elist = list;
  a.nlist = n;
  return a;
}
static int stage_res_prepare(GenCtx* g, const double* u) {
  if (!g->need_nbr || g->Eex == 0) return FR_OK;
  const int ph = pbeg(g, 0);
  GArgs a = gargs_list(g, u, nullptr, g->exp_list, g->Eex);
  GCK(gen_elem<GM_UF>(g, a));
  GCK(gen_elem<GM_QF>(g, a));
  pend(g, ph);
  return FR_OK;
}
static int stage_res_newton(GenCtx* g, const double* u, const double* uhat) {
  const int ph = pbeg(g, 0);
  GArgs a = gargs_list(g, u, uhat, g->imp_idx, g->Eim);
  a.R = g->Rw;
  a.gview = g->gview;
  if (g->Eim) GCK(gen_elem<GM_RES>(g, a));
  if (g->ntrace) {
    (count_launch(), k_gen_trace_sum<<<nb256(g->nh), 256, 0, g->st>>>(g->npts, g->nv, g->gptr, g->gidx, g->gview,
                                                                       g->gw, (long long)g->nface * g->E * g->fs));
    GCK(cudaGetLastError());
  }
  pend(g, ph);
  return FR_OK;
}
static int stage_res_finish(GenCtx* g, const double* u, const double* uhat) {
  if (g->Eex == 0) return FR_OK;
  const int ph = pbeg(g, 0);
  if (g->need_nbr && g->Eim) {
    GArgs ai = gargs_list(g, u, uhat, g->imp_idx, g->Eim);
    GCK(gen_elem<GM_UF>(g, ai));
    GCK(gen_elem<GM_QF>(g, ai));
  }
  GArgs a = gargs_list(g, u, uhat, g->exp_list, g->Eex);
  a.R = g->Rw;
  a.gview = g->gview;
  GCK(gen_elem<GM_RES>(g, a));
  pend(g, ph);
  return FR_OK;
}

int residual(GenCtx* g, const double* u, const double* uhat, double* R, double* gtrace) {
  int rc = residual_into(g, u, uhat, R, gtrace);
  if (rc) return rc;
  GCK(cudaStreamSynchronize(g->st));
  return FR_OK;
}

int initial_trace(GenCtx* g, const double* u, double* uhat) {
  GArgs a = gargs(g, u, nullptr);
  double* buf = g->gview;  // face-point states of every element, scratch
  a.Uf_out = buf;
  GCK(gen_elem<GM_UF>(g, a));
  if (g->ntrace) {
    (count_launch(), k_gen_initial_trace<<<nb256(g->nh), 256, 0, g->st>>>(g->npts, g->nv, g->gptr, g->gidx, g->kind,
                                                                           buf, a, uhat));
    GCK(cudaGetLastError());
  }
  GCK(cudaMemsetAsync(g->gview, 0, (size_t)g->nface * g->E * g->fs * g->nv * sizeof(double), g->st));
  GCK(cudaStreamSynchronize(g->st));
  return FR_OK;
}

template <int PHYS, typename T>
static cudaError_t launch_gen_jac(GenCtx* g, const GArgs& a, const JArgs& j) {
  constexpr int NV = Phys<PHYS>::NV;
  const size_t smem = sizeof(JWork<NV, T>);
  auto kern = k_gen_jacobian<PHYS, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (j.Eim == 0) return cudaSuccess;
  (count_launch(), kern<<<j.Eim, JT, smem, g->st>>>(g->pp, a, j));
  return cudaGetLastError();
}

static int jacobian_blocks(GenCtx* g, const double* u, const double* uhat, double a_dt) {
  if (g->Eim == 0) return FR_OK;
  const int ph = pbeg(g, 1);
  GArgs a = gargs(g, u, uhat);
  JArgs j;
  j.Eim = g->Eim;
  j.imp_idx = g->imp_idx;
  j.offA = g->offA;
  j.offB = g->offB;
  j.offD = g->offD;
  j.lto = g->lto;
  j.a_dt = a_dt;
  j.A = g->A;
  j.B = g->B;
  j.C = g->C;
  j.D = g->D;
  j.scratch = g->jscratch;
  cudaError_t e;
  if (g->dim == 3)
    e = hex_jacobian(g, a, j);
  else if (g->pb == 8)
    e = g->pp.kind == 0 ? launch_gen_jac<0, double>(g, a, j) : launch_gen_jac<1, double>(g, a, j);
  else
    e = g->pp.kind == 0 ? launch_gen_jac<0, float>(g, a, j) : launch_gen_jac<1, float>(g, a, j);
  GCK(e);
  pend(g, ph);
  g->lin_valid = true;
  return FR_OK;
}

static int form_rhs(GenCtx* g, const double* u, const double* ustar, double a_dt) {
  if (g->Eim == 0) return FR_OK;
  (count_launch(), k_gen_form_rhs<<<nbw(g->Eim), 256, 0, g->st>>>(g->Eim, g->nv, g->nface, g->fs, g->dim, g->imp_idx,
                                                                   g->deg, g->uoff, g->offr,
                                                                   g->offs, g->nfp, g->lto, u, ustar, g->Rw, g->gview,
                                                                   a_dt, g->r, g->s));
  GCK(cudaGetLastError());
  return FR_OK;
}

int local_jacobian(GenCtx* g, const double* u, const double* uhat, const double* ustar, double a_dt) {
  int rc = residual_into(g, u, uhat, g->Rw, nullptr);
  if (!rc) rc = form_rhs(g, u, ustar, a_dt);
  if (!rc) rc = jacobian_blocks(g, u, uhat, a_dt);
  if (rc) return rc;
  GCK(cudaStreamSynchronize(g->st));
  return FR_OK;
}

static int condense_impl(GenCtx* g) {
  (count_launch(), k_gen_status_reset<<<1, 1, 0, g->st>>>(g->status));
  GCK(cudaGetLastError());
  if (g->Eim == 0) return FR_OK;
  int ph = pbeg(g, 2);
  for (const auto& tc : g->tc_classes)
    GCK(launch_condense_class(tc.list, tc.count, tc.nA, tc.nT, g->udev.off, g->A, g->B, g->C, g->D, g->r, g->s, g->LU,
                              g->piv, g->XB, g->xr, g->S, g->te, g->status, g->cscratch, g->ccap, 2, g->st, tc.k0,
                              tc.off0));
  GCK(launch_condense_uneven_dev(g->pb, g->udev, g->A, g->B, g->C, g->D, g->r, g->s, g->LU, g->piv, g->XB, g->xr,
                                 g->S, g->te, g->status, g->st));
  pend(g, ph);
  ph = pbeg(g, 3);
  if (g->ntrace) {
    (count_launch(), k_gen_gather_sum<<<nb256(g->nh), 256, 0, g->st>>>(g->nh, g->vptr, g->vidx, g->te, g->tg, nullptr, 0,
                                                                        (long long)g->sumT));
    GCK(cudaGetLastError());
    if (g->efr && g->pb == 8)
      (count_launch(), k_gen_precond_build_node<double><<<nb256(g->npts), 256, 0, g->st>>>(
           g->npts, g->nv, g->nptr, g->nent_k, g->nent_l, g->nTk, g->offD, (const double*)g->S, (double*)g->Pinv,
           g->status));
    else if (g->efr)
      (count_launch(), k_gen_precond_build_node<float><<<nb256(g->npts), 256, 0, g->st>>>(
           g->npts, g->nv, g->nptr, g->nent_k, g->nent_l, g->nTk, g->offD, (const float*)g->S, (float*)g->Pinv,
           g->status));
    else if (g->pb == 8)
      (count_launch(), k_gen_precond_build<double><<<g->ntrace, GP_THREADS, precond_smem_bytes<double>(g->bsmax),
                                                      g->st>>>(g->ntrace, g->nv, g->tpts, g->poff, g->pside, g->nTk,
                                                               g->offD, (const double*)g->S, (double*)g->Pinv,
                                                               g->status));
    else
      (count_launch(), k_gen_precond_build<float><<<g->ntrace, GP_THREADS, precond_smem_bytes<float>(g->bsmax),
                                                     g->st>>>(g->ntrace, g->nv, g->tpts, g->poff, g->pside, g->nTk,
                                                              g->offD, (const float*)g->S, (float*)g->Pinv,
                                                              g->status));
    GCK(cudaGetLastError());
  }
  pend(g, ph);
  return FR_OK;
}

static int check_status(GenCtx* g, const char* where) {
  int hs[2];
  GCK(cudaMemcpyAsync(hs, g->status, sizeof(hs), cudaMemcpyDeviceToHost, g->st));
  GCK(cudaStreamSynchronize(g->st));
  if (hs[0] & DEV_ERR_SINGULAR) {
    GCK(cudaMemsetAsync(g->status, 0, sizeof(int), g->st));
    // element blocks report their compact index, face preconditioner blocks -1 - trace
    return err(g, FR_ERR_SINGULAR, where, hs[1] >= 0 ? hs[1] : -1);
  }
  return FR_OK;
}

int condense(GenCtx* g, int refine) {
  if (refine != 0) return err(g, FR_ERR_UNSUPPORTED, "hfr_condense: refinement sweeps are not built for general meshes");
  int rc = condense_impl(g);
  if (rc) return rc;
  return check_status(g, "hfr_condense: zero pivot");
}

// GMRES callbacks
static void cb_matvec_g(void* c, const double* x, double* y, cudaStream_t s) {
  GenCtx* g = (GenCtx*)c;
  const int ph = pbeg(g, 8);
  if (g->pb == 8)
    (count_launch(), k_gen_matvec_elem<double><<<nbw(g->Eim), 256, 0, s>>>(g->Eim, g->nTk, g->offD, g->offs, g->gmap,
                                                                           (const double*)g->S, x, g->yv, nullptr, 0,
                                                                           (long long)g->nh));
  else
    (count_launch(), k_gen_matvec_elem<float><<<nbw(g->Eim), 256, 0, s>>>(g->Eim, g->nTk, g->offD, g->offs, g->gmap,
                                                                          (const float*)g->S, x, g->yv, nullptr, 0,
                                                                          (long long)g->nh));
  (count_launch(), k_gen_gather_sum<<<nb256(g->nh), 256, 0, s>>>(g->nh, g->vptr, g->vidx, g->yv, y, nullptr, 0,
                                                                    (long long)g->sumT));
  pend(g, ph);
}
static void cb_gmatvec_g(void* c, const GmresState* st, int j, const double* x, const float*, double* y, cudaStream_t s) {
  GenCtx* g = (GenCtx*)c;
  if (g->pb == 8)
    (count_launch(), k_gen_matvec_elem<double><<<nbw(g->Eim), 256, 0, s>>>(g->Eim, g->nTk, g->offD, g->offs, g->gmap,
                                                                           (const double*)g->S, x, g->yv, &st->kdone, j,
                                                                           (long long)g->nh));
  else
    (count_launch(), k_gen_matvec_elem<float><<<nbw(g->Eim), 256, 0, s>>>(g->Eim, g->nTk, g->offD, g->offs, g->gmap,
                                                                          (const float*)g->S, x, g->yv, &st->kdone, j,
                                                                          (long long)g->nh));
  (count_launch(), k_gen_gather_sum<<<nb256(g->nh), 256, 0, s>>>(g->nh, g->vptr, g->vidx, g->yv, y, &st->kdone, j,
                                                                    (long long)g->sumT));
}
static void cb_precond_g(void* c, const GmresState* st, int j, double* x, double* y, float* y32, cudaStream_t s) {
  GenCtx* g = (GenCtx*)c;
  if (g->bsmax <= 8) {  // small blocks (EFR nodes): one thread per block
    if (g->pb == 8)
      (count_launch(), k_gen_precond_apply_small<double><<<nb256(g->ntrace), 256, 0, s>>>(
           g->ntrace, g->nv, g->tpts, g->toff, g->poff, (const double*)g->Pinv, x, y, &st->kdone, j,
           j > 0 ? &st->inv_hn : nullptr, y32));
    else
      (count_launch(), k_gen_precond_apply_small<float><<<nb256(g->ntrace), 256, 0, s>>>(
           g->ntrace, g->nv, g->tpts, g->toff, g->poff, (const float*)g->Pinv, x, y, &st->kdone, j,
           j > 0 ? &st->inv_hn : nullptr, y32));
    return;
  }
  if (g->pb == 8)
    (count_launch(), k_gen_precond_apply<double><<<nbw(g->ntrace), 256, 0, s>>>(
         g->ntrace, g->nv, g->tpts, g->toff, g->poff, (const double*)g->Pinv, x, y, &st->kdone, j,
         j > 0 ? &st->inv_hn : nullptr, y32));
  else
    (count_launch(), k_gen_precond_apply<float><<<nbw(g->ntrace), 256, 0, s>>>(
         g->ntrace, g->nv, g->tpts, g->toff, g->poff, (const float*)g->Pinv, x, y, &st->kdone, j,
         j > 0 ? &st->inv_hn : nullptr, y32));
}

static int gmres_impl(GenCtx* g, double* duhat, double rtol, int maxit, int* iters, double* final_rel) {
  if (g->ntrace == 0) {
    if (iters) *iters = 0;
    if (final_rel) *final_rel = 0.0;
    return FR_OK;
  }
  GmresOps ops;
  ops.ctx = g;
  ops.matvec = cb_matvec_g;
  ops.gated_matvec = cb_gmatvec_g;
  ops.precond = cb_precond_g;
  GmresResult res;
  memset(&res, 0, sizeof(res));
  const int ph = pbeg(g, 4);
  const int grc = run_gmres(ops, g->gm, g->tg, duhat, rtol, g->restart, maxit, 4, &res, g->st);
  pend(g, ph);
  if (grc != 0) return err(g, FR_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  GCK(cudaGetLastError());
  if (iters) *iters = res.iterations;
  if (final_rel) *final_rel = res.rel;
  if (res.nan) return err(g, FR_ERR_DIVERGED, "hfr_trace_gmres: non-finite residual", -1, res.iterations);
  if (!res.converged && res.rel > rtol)
    return err(g, FR_ERR_NOT_CONVERGED, "hfr_trace_gmres: iteration limit", -1, res.iterations, res.rel);
  return FR_OK;
}

int trace_gmres(GenCtx* g, double* duhat, double rtol, int maxit, int* iters, double* final_rel) {
  return gmres_impl(g, duhat, rtol, maxit, iters, final_rel);
}

static int backsolve_impl(GenCtx* g, const double* duhat, double* du) {
  if (g->Eim == 0) return FR_OK;
  const int ph = pbeg(g, 5);
  if (g->pb == 8)
    (count_launch(), k_gen_backsolve<double><<<nbw(g->Eim), 256, 0, g->st>>>(
         g->Eim, g->nAk, g->nTk, g->offB, g->offr, g->offs, g->gmap, (const double*)g->XB, g->xr, duhat, du,
         (long long)g->nh));
  else
    (count_launch(), k_gen_backsolve<float><<<nbw(g->Eim), 256, 0, g->st>>>(
         g->Eim, g->nAk, g->nTk, g->offB, g->offr, g->offs, g->gmap, (const float*)g->XB, g->xr, duhat, du,
         (long long)g->nh));
  GCK(cudaGetLastError());
  pend(g, ph);
  return FR_OK;
}

int backsolve(GenCtx* g, const double* duhat, double* du, int refine) {
  if (refine != 0) return err(g, FR_ERR_UNSUPPORTED, "hfr_backsolve: refinement sweeps are not built for general meshes");
  int rc = backsolve_impl(g, duhat, du);
  if (rc) return rc;
  GCK(cudaStreamSynchronize(g->st));
  return FR_OK;
}

int export_array(GenCtx* g, int which, void* buf, size_t bytes, bool import) {
  const size_t pb = g->pb;
  void* arr = nullptr;
  size_t need = 0;
  switch (which) {
    case 0: arr = g->A; need = g->sumAA * pb; break;
    case 1: arr = g->B; need = g->sumAT * pb; break;
    case 2: arr = g->C; need = g->sumAT * pb; break;
    case 3: arr = g->D; need = g->sumTT * pb; break;
    case 4: arr = g->S; need = g->sumTT * pb; break;
    case 5: arr = g->XB; need = g->sumAT * pb; break;
    case 6: arr = g->xr; need = g->sumA * 8; break;
    case 7: arr = g->te; need = g->sumT * 8; break;
    case 8: arr = g->r; need = g->sumA * 8; break;
    case 9: arr = g->s; need = g->sumT * 8; break;
    case 10: if (!import) { arr = g->tg; need = g->nh * 8; } break;
    case 11: if (!import) { arr = g->Pinv; need = g->sumP * pb; } break;
    case 64:  // the trace point of every element face point (int32); written only by checked builds
#ifndef FR_CHECKED
      if (import) break;
#endif
      arr = g->fnode;
      need = (size_t)g->nface * g->E * g->fs * sizeof(int);
      break;
  }
  if (!arr) return err(g, FR_ERR_INVALID_ARG, "hfr_export / hfr_import: unknown array");
  if (import ? bytes != need : bytes < need)
    return err(g, FR_ERR_INVALID_ARG, "hfr_export / hfr_import: buffer size");
  if (import) {
    GCK(cudaMemcpyAsync(arr, buf, need, cudaMemcpyDeviceToDevice, g->st));
  } else {
    GCK(cudaMemcpyAsync(buf, arr, need, cudaMemcpyDeviceToDevice, g->st));
  }
  GCK(cudaStreamSynchronize(g->st));
  return FR_OK;
}

static int sumsq(GenCtx* g, const double* a, size_t na, const double* b, size_t nb, double* out) {
  const int nbk = 256;
  (count_launch(), k_gen_sumsq_part<<<nbk, 256, 0, g->st>>>(a, na, b, nb, g->red));
  (count_launch(), k_gen_sumsq_final<<<1, 32, 0, g->st>>>(g->red, nbk, g->red + 1024));
  GCK(cudaGetLastError());
  GCK(cudaMemcpyAsync(out, g->red + 1024, sizeof(double), cudaMemcpyDeviceToHost, g->st));
  GCK(cudaStreamSynchronize(g->st));
  return FR_OK;
}

struct TabG {
  int s;
  double a[2][2], b[2], ah[3][3], bh[3];
};
static TabG tableau_g(int which) {
  TabG t;
  memset(&t, 0, sizeof(t));
  if (which == FR_TAB_SDIRK2) {
    const double gm = 1.0 - sqrt(2.0) / 2.0, dl = -2.0 * sqrt(2.0) / 3.0;
    t.s = 2;
    t.a[0][0] = gm;
    t.a[1][0] = 1.0 - gm;
    t.a[1][1] = gm;
    t.b[0] = 1.0 - gm;
    t.b[1] = gm;
    t.ah[1][0] = gm;
    t.ah[2][0] = dl;
    t.ah[2][1] = 1.0 - dl;
    t.bh[1] = 1.0 - gm;
    t.bh[2] = gm;
  } else {
    t.s = 1;
    t.a[0][0] = 1.0;
    t.b[0] = 1.0;
    t.ah[1][0] = 1.0;
    t.bh[1] = 1.0;
  }
  return t;
}

// ------------------------------------------------------------------ whole-stage CUDA graph
// The implicit stage as one executable graph, as on the uniform path: the Newton loop a WHILE
// node, its linear solve an IF node, the GMRES restart cycles a nested WHILE node
// (capture_gmres); small kernels take on the device the decisions the stream path takes on the
// host (same tests, same order), and the host reads the counters once after the launch.
struct GStageDev {
  double norm0, norm;
  int it, gtot, conv, err, sing, cycles;
};
__global__ void k_gs_init(GStageDev* sd) {
  sd->norm0 = -1.0;
  sd->norm = 0.0;
  sd->it = 0;
  sd->gtot = 0;
  sd->conv = 0;
  sd->err = 0;
  sd->sing = -1;
  sd->cycles = 0;
}
__global__ void k_gs_newton_check(GStageDev* sd, const double* ss, double tol, int maxit,
                                  cudaGraphConditionalHandle hn, cudaGraphConditionalHandle hs) {
  const double nrm = sqrt(*ss);
  if (sd->norm0 < 0.0) sd->norm0 = nrm;
  sd->norm = nrm;
  if (!(nrm == nrm)) sd->err |= 1;
  const int conv = (nrm <= tol * sd->norm0 || nrm == 0.0) ? 1 : 0;
  sd->conv = conv;
  const int cont = (!conv && sd->err == 0 && sd->it < maxit) ? 1 : 0;
  if (cont) sd->it += 1;
  cudaGraphSetConditional(hn, (unsigned)cont);
  cudaGraphSetConditional(hs, (unsigned)cont);
}
// a zero pivot in the condensation ends the Newton loop at its next test
__global__ void k_gs_cond_check(GStageDev* sd, const int* status) {
  if (status[0] & DEV_ERR_SINGULAR) {
    sd->err |= 8;
    if (sd->sing < 0) sd->sing = status[1];
  }
}
__global__ void k_gs_gmres_done(GStageDev* sd, const GmresGraphDev* gd) {
  sd->gtot += gd->total;
  sd->cycles += gd->cycles;
  if (gd->nan) sd->err |= 2;
}

int set_graph(GenCtx* g, int on) {
  if (on && g->Eim == 0) return err(g, FR_ERR_UNSUPPORTED, "imex_stage_set_graph: needs implicit elements");
  g->use_graph = on;
  g->gvalid = false;
  return FR_OK;
}

static int stage_graph_capture(GenCtx* g, const GenCtx::GKey& key) {
  const TabG tb = tableau_g(g->tableau);
  const int i = key.stage;
  const size_t tot = g->nstate;
  for (auto& c : g->cap)
    if (!c && cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking) != cudaSuccess)
      return err(g, FR_ERR_CUDA, "imex_stage: stream creation failed");
  if (!g->gdev) {
    int rc = FR_OK;
    g->gdev = galloc<unsigned char>(g, 256, &rc);
    if (rc) return err(g, rc, "imex_stage: out of device memory");
  }
  GStageDev* sd = reinterpret_cast<GStageDev*>(g->gdev);
  GmresGraphDev* gd = reinterpret_cast<GmresGraphDev*>(reinterpret_cast<char*>(g->gdev) + 128);
  cudaStream_t user = g->st;
  cudaGraph_t gr = nullptr, bn = nullptr, bs = nullptr;
  int depth = 0;
  auto fail = [&](cudaError_t e) {
    for (int d = depth - 1; d >= 0; --d) {
      cudaGraph_t tmp = nullptr;
      cudaStreamEndCapture(g->cap[d], &tmp);
    }
    g->st = user;
    g->capturing = false;
    if (gr) cudaGraphDestroy(gr);
    cudaGetLastError();
    return err(g, FR_ERR_CUDA, cudaGetErrorString(e));
  };
#define SK(x)                              \
  do {                                     \
    const cudaError_t e_ = (x);            \
    if (e_ != cudaSuccess) return fail(e_); \
  } while (0)
#define SR(x)                                    \
  do {                                           \
    const int r_ = (x);                          \
    if (r_ != FR_OK) return fail(cudaErrorUnknown); \
  } while (0)
  g->capturing = true;
  const unsigned long long l0 = launch_count();
  SK(cudaGraphCreate(&gr, 0));
  SK(cudaStreamBeginCaptureToGraph(g->cap[0], gr, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  depth = 1;
  g->st = g->cap[0];
  double* u_stage = const_cast<double*>(key.u_stage);
  double* uhat = const_cast<double*>(key.uhat);
  {
    StageCoefG sc;
    memset(&sc, 0, sizeof(sc));
    sc.nterm = i;
    for (int jj = 0; jj < i; ++jj) {
      sc.hi[jj] = jj;
      sc.ce[jj] = key.dt * tb.ah[i][jj];
      sc.ci[jj] = jj >= 1 ? key.dt * tb.a[i - 1][jj - 1] : 0.0;
    }
    (count_launch(), k_gen_stage_combine<<<nb256(tot), 256, 0, g->st>>>(tot, g->dof_imp, key.u_n, key.R_hist, sc,
                                                                        u_stage));
    SK(cudaGetLastError());
  }
  SK(cudaMemcpyAsync(g->Ustar, u_stage, tot * sizeof(double), cudaMemcpyDeviceToDevice, g->st));
  (count_launch(), k_gs_init<<<1, 1, 0, g->st>>>(sd));
  SK(cudaGetLastError());
  const double adt = key.dt * tb.a[i - 1][i - 1];
  SR(stage_res_prepare(g, u_stage));
  cudaGraphConditionalHandle hn, hs;
  SK(graph_conditional_handle(g->cap[0], 1u, cudaGraphCondAssignDefault, &hn));
  SK(graph_add_conditional(g->cap[0], hn, cudaGraphCondTypeWhile, &bn));
  const unsigned long long l1 = launch_count();
  // ---- Newton body: residual, right-hand sides, norm test
  SK(cudaStreamBeginCaptureToGraph(g->cap[1], bn, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  depth = 2;
  g->st = g->cap[1];
  SK(graph_conditional_handle(g->cap[1], 0u, 0u, &hs));
  SR(stage_res_newton(g, u_stage, uhat));
  SR(form_rhs(g, u_stage, g->Ustar, adt));
  {
    const int nbk = 256;
    (count_launch(), k_gen_sumsq_part<<<nbk, 256, 0, g->st>>>(g->r, g->sumA, g->gw, g->nh, g->red));
    (count_launch(), k_gen_sumsq_final<<<1, 32, 0, g->st>>>(g->red, nbk, g->red + 1024));
    (count_launch(), k_gs_newton_check<<<1, 1, 0, g->st>>>(sd, g->red + 1024, key.ntol, key.nmax, hn, hs));
    SK(cudaGetLastError());
  }
  SK(graph_add_conditional(g->cap[1], hs, cudaGraphCondTypeIf, &bs));
  const unsigned long long l2 = launch_count();
  // ---- solve body: blocks, condensation, GMRES cycles, back-substitution, update
  SK(cudaStreamBeginCaptureToGraph(g->cap[2], bs, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  depth = 3;
  g->st = g->cap[2];
  SR(jacobian_blocks(g, u_stage, uhat, adt));
  SR(condense_impl(g));
  (count_launch(), k_gs_cond_check<<<1, 1, 0, g->st>>>(sd, g->status));
  SK(cudaGetLastError());
  unsigned long long lg0 = launch_count(), lg1 = lg0;
  if (g->ntrace > 0) {
    GmresOps ops;
    ops.ctx = g;
    ops.matvec = cb_matvec_g;
    ops.gated_matvec = cb_gmatvec_g;
    ops.precond = cb_precond_g;
    const cudaStream_t sc[2] = {g->cap[3], g->cap[4]};
    lg0 = launch_count();
    SK(capture_gmres(ops, g->gm, g->tg, g->duhat, key.grtol, g->restart, key.gmax, gd, g->st, sc, &g->gl_gm));
    lg1 = launch_count();
    (count_launch(), k_gs_gmres_done<<<1, 1, 0, g->st>>>(sd, gd));
    SK(cudaGetLastError());
  } else {
    SK(cudaMemsetAsync(g->duhat, 0, std::max(g->nh, (size_t)1) * sizeof(double), g->st));
  }
  SR(backsolve_impl(g, g->duhat, g->du));
  if (g->Eim) {
    (count_launch(), k_gen_apply_du<<<nbw(g->Eim), 256, 0, g->st>>>(g->Eim, g->nv, g->imp_idx, g->deg, g->uoff, g->offr,
                                                                     g->du, u_stage));
    SK(cudaGetLastError());
  }
  if (g->nh) {
    (count_launch(), k_gen_axpy<<<nb256(g->nh), 256, 0, g->st>>>(g->nh, 1.0, g->duhat, uhat));
    SK(cudaGetLastError());
  }
  SK(cudaStreamEndCapture(g->cap[2], &bs));
  depth = 2;
  const unsigned long long l3 = launch_count();
  SK(cudaStreamEndCapture(g->cap[1], &bn));
  depth = 1;
  g->st = g->cap[0];
  SR(stage_res_finish(g, u_stage, uhat));
  SK(cudaMemcpyAsync(const_cast<double*>(key.R_hist) + (size_t)i * tot, g->Rw, tot * sizeof(double),
                     cudaMemcpyDeviceToDevice, g->st));
  SK(cudaStreamEndCapture(g->cap[0], &gr));
  depth = 0;
  const unsigned long long l4 = launch_count();
  g->st = user;
  g->capturing = false;
  cudaGraphExec_t ex = nullptr;
  {
    const cudaError_t e = cudaGraphInstantiate(&ex, gr, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(gr);
      cudaGetLastError();
      return err(g, FR_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  if (g->gexec) cudaGraphExecDestroy(g->gexec);
  if (g->graph) cudaGraphDestroy(g->graph);
  g->graph = gr;
  g->gexec = ex;
  g->gkey = key;
  g->gvalid = true;
  // the capture counted each kernel once: a replay's count follows from its loop counts
  launch_count_add(-(long long)(l4 - l0));
  g->gl_top = (int)((l1 - l0) + (l4 - l3));
  g->gl_newton = (int)(l2 - l1);
  g->gl_solve = (int)((l3 - l2) - (lg1 - lg0));
#undef SK
#undef SR
  return FR_OK;
}

static int stage_graph(GenCtx* g, const GenCtx::GKey& key, fr_stage_stats* stats) {
  if (!g->gvalid || !(g->gkey == key)) {
    const int rc = stage_graph_capture(g, key);
    if (rc) return rc;
  }
  cudaStream_t st = g->st;
  GCK(cudaGraphLaunch(g->gexec, st));
  GStageDev h;
  GCK(cudaMemcpyAsync(&h, g->gdev, sizeof(h), cudaMemcpyDeviceToHost, st));
  GCK(cudaStreamSynchronize(st));
  const int solves = g->ntrace > 0 ? h.it : 0;
  launch_count_add((long long)g->gl_top + (long long)(h.it + 1) * g->gl_newton + (long long)h.it * g->gl_solve +
                   (long long)solves * g->gl_gm.fixed + (long long)h.cycles * g->gl_gm.cycle +
                   (long long)(h.cycles - solves) * g->gl_gm.residual);
  if (stats) {
    stats->newton_iterations = h.it;
    stats->gmres_iterations = h.gtot;
    stats->residual0 = h.norm0;
    stats->residual = h.norm;
    stats->converged = h.conv;
  }
  if (h.err & 8) {
    GCK(cudaMemsetAsync(g->status, 0, sizeof(int), st));
    GCK(cudaStreamSynchronize(st));
    return err(g, FR_ERR_SINGULAR, "imex_stage: zero pivot in condensation", h.sing >= 0 ? h.sing : -1, h.it);
  }
  if (h.err & 1) return err(g, FR_ERR_DIVERGED, "imex_stage: non-finite Newton residual", -1, h.it);
  if (h.err & 2) return err(g, FR_ERR_DIVERGED, "imex_stage: non-finite GMRES residual", -1, h.it);
  if (!h.conv) return err(g, FR_ERR_NOT_CONVERGED, "imex_stage: Newton iteration limit", -1, h.it, h.norm);
  return FR_OK;
}

int stage(GenCtx* g, int stage, double dt, const double* u_n, double* u_stage, double* uhat, double* R_hist,
          double newton_tol, int newton_maxit, double gmres_rtol, int gmres_maxit, int refine, fr_stage_stats* stats) {
  if (refine != 0) return err(g, FR_ERR_UNSUPPORTED, "imex_stage: refinement sweeps are not built for general meshes");
  const TabG tb = tableau_g(g->tableau);
  if (stage < 0 || stage > tb.s + 1) return err(g, FR_ERR_INVALID_ARG, "imex_stage: stage out of range");
  const size_t tot = g->nstate;
  cudaStream_t st = g->st;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (stage == 0) {
    int rc = residual_into(g, u_n, uhat, R_hist, nullptr);
    if (rc) return rc;
    GCK(cudaStreamSynchronize(st));
    return FR_OK;
  }
  if (stage == tb.s + 1) {
    StageCoefG sc;
    memset(&sc, 0, sizeof(sc));
    sc.nterm = tb.s + 1;
    for (int jj = 0; jj <= tb.s; ++jj) {
      sc.hi[jj] = jj;
      sc.ci[jj] = jj >= 1 ? dt * tb.b[jj - 1] : 0.0;
      sc.ce[jj] = dt * tb.bh[jj];
    }
    (count_launch(), k_gen_stage_combine<<<nb256(tot), 256, 0, st>>>(tot, g->dof_imp, u_n, R_hist, sc, u_stage));
    GCK(cudaGetLastError());
    GCK(cudaStreamSynchronize(st));
    return FR_OK;
  }
  const int i = stage;
  if (g->use_graph) {
    GenCtx::GKey key;
    key.stage = i;
    key.dt = dt;
    key.u_n = u_n;
    key.u_stage = u_stage;
    key.uhat = uhat;
    key.R_hist = R_hist;
    key.ntol = newton_tol;
    key.nmax = newton_maxit;
    key.grtol = gmres_rtol;
    key.gmax = gmres_maxit;
    return stage_graph(g, key, stats);
  }
  StageCoefG sc;
  memset(&sc, 0, sizeof(sc));
  sc.nterm = i;
  for (int jj = 0; jj < i; ++jj) {
    sc.hi[jj] = jj;
    sc.ce[jj] = dt * tb.ah[i][jj];
    sc.ci[jj] = jj >= 1 ? dt * tb.a[i - 1][jj - 1] : 0.0;
  }
  (count_launch(), k_gen_stage_combine<<<nb256(tot), 256, 0, st>>>(tot, g->dof_imp, u_n, R_hist, sc, u_stage));
  GCK(cudaGetLastError());
  GCK(cudaMemcpyAsync(g->Ustar, u_stage, tot * sizeof(double), cudaMemcpyDeviceToDevice, st));
  const double adt = dt * tb.a[i - 1][i - 1];
  double norm0 = -1.0, normk = 0.0;
  int it = 0, gtot = 0;
  bool conv = false;
  {
    const int rc = stage_res_prepare(g, u_stage);
    if (rc) return rc;
  }
  for (;; ++it) {
    int rc = stage_res_newton(g, u_stage, uhat);
    const int phn = pbeg(g, 6);
    if (!rc) rc = form_rhs(g, u_stage, g->Ustar, adt);
    double ss = 0.0;
    if (!rc) rc = sumsq(g, g->r, g->sumA, g->gw, g->nh, &ss);
    pend(g, phn);
    if (rc) return rc;
    normk = sqrt(ss);
    if (!(normk == normk)) return err(g, FR_ERR_DIVERGED, "imex_stage: non-finite Newton residual", -1, it);
    if (norm0 < 0) norm0 = normk;
    if (normk <= newton_tol * norm0 || normk == 0.0) {
      conv = true;
      break;
    }
    if (it >= newton_maxit) break;
    rc = jacobian_blocks(g, u_stage, uhat, adt);
    if (!rc) rc = condense_impl(g);
    if (!rc) rc = check_status(g, "imex_stage: zero pivot in condensation");
    if (rc) return rc;
    int its = 0;
    double rel = 0.0;
    rc = gmres_impl(g, g->duhat, gmres_rtol, gmres_maxit, &its, &rel);
    gtot += its;
    if (rc && rc != FR_ERR_NOT_CONVERGED) return rc;
    rc = backsolve_impl(g, g->duhat, g->du);
    if (rc) return rc;
    const int phu = pbeg(g, 6);
    if (g->Eim) {
      (count_launch(), k_gen_apply_du<<<nbw(g->Eim), 256, 0, st>>>(g->Eim, g->nv, g->imp_idx, g->deg, g->uoff, g->offr,
                                                                   g->du, u_stage));
      GCK(cudaGetLastError());
    }
    if (g->nh) {
      (count_launch(), k_gen_axpy<<<nb256(g->nh), 256, 0, st>>>(g->nh, 1.0, g->duhat, uhat));
      GCK(cudaGetLastError());
    }
    pend(g, phu);
  }
  {
    const int rc = stage_res_finish(g, u_stage, uhat);  // R of the explicit elements at the final state
    if (rc) return rc;
  }
  GCK(cudaMemcpyAsync(R_hist + (size_t)i * tot, g->Rw, tot * sizeof(double), cudaMemcpyDeviceToDevice, st));
  GCK(cudaStreamSynchronize(st));
  if (stats) {
    stats->newton_iterations = it;
    stats->gmres_iterations = gtot;
    stats->residual0 = norm0;
    stats->residual = normk;
    stats->converged = conv ? 1 : 0;
  }
  if (!conv) return err(g, FR_ERR_NOT_CONVERGED, "imex_stage: Newton iteration limit", -1, it, normk);
  return FR_OK;
}

}  // namespace gen
}  // namespace hfr

#include "hfr_checked_unit.inc"
