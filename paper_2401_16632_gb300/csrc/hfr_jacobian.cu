// Element Jacobian blocks A, B, C, D of the hybridized stage (Pereira & Vermeire,
// arXiv 2401.16632, Sec. 3.2, eqs. elemA, elemsystem, elemsystemB), for the stage residual
// h = u - u* - a dt R(u, u^) and the element's trace-residual contribution g^k:
//     A = dh/du = I - a dt dR/du,  B = dh/du^ = -a dt dR/du^,  C = dg^k/du,  D = dg^k/du^.
//
// One CTA per implicit element.  The linearisation is organised around the structure of
// the tensor-product operators instead of differentiating the whole element residual:
//   1. exact pointwise Jacobians of the volume flux (w.r.t. the state and the reference
//      gradient) and of the common face flux (w.r.t. face state, trace, face gradient), by
//      forward-mode dual numbers, one tangent per thread;
//   2. per seed point (NV columns of the blocks), the tangent of the corrected gradient is
//      nonzero only on the two grid lines through the seeded point (or on the one line normal
//      to the seeded trace point), so the flux tangents are formed only there, by one warp;
//   3. the output columns follow from the 1D operators M, dgL, dgR along the lines: a full
//      line sum on the seed's row and column, one term elsewhere.
// Work per element is O((nA + nT)^2), not the O((nA + nT) x residual) of a dense sweep.
// T = double (plain path) or float (mixed path; blocks stored in FP32).
#include "hfr_internal.h"

namespace hfr {

// resident CTAs per SM asked of the compiler for the FP32 p = 4 kernel (register cap 65536 /
// (256 x blocks)); a build flag, for timing the register / occupancy trade
#ifndef HFR_JAC_P4_BLOCKS
#define HFR_JAC_P4_BLOCKS 4
#endif
constexpr int JAC_THREADS = 256;
constexpr int JAC_WARPS = JAC_THREADS / 32;

template <int P, int PHYS, typename T>
struct JacWork {
  static constexpr int N = P + 1, NS = N * N, NV = Phys<PHYS>::NV, NF = 4 * N;
  T U[NS][NV];
  T Uf[NF][NV];
  T ub[NF][NV];
  T un[NF][NV];
  T q[NS][2][NV];
  T qf[NF][2][NV];
  T iJ[NS];
  T Sm[NS][2][2];
  T fJ[NF], fn[NF][2];
  // pointwise Jacobians, innermost index the input variable (read NV-wide: 16-byte aligned)
  alignas(16) T KU[NS][2][NV][NV];
  alignas(16) T KQ[NS][2][2][NV][NV];
  alignas(16) T GU[NF][NV][NV];
  alignas(16) T GH[NF][NV][NV];
  alignas(16) T GQ[NF][2][NV][NV];
  T ciJ[NS];  // a dt / J at each solution point
  // per-warp tangents of one seed point, entries [v][v0] (NV seed columns innermost), rows
  // padded by 16 bytes so that lane groups reading different points hit different banks
  static constexpr int PAD = NV == 4 ? 4 : 0;
  static constexpr int LNS = 2 * NV * NV + PAD, RCS = NV * NV + PAD;
  alignas(16) T LN[JAC_WARPS][2][N][LNS];  // flux tangents [r][v][v0] on the seed's row (0) / column (1)
  alignas(16) T RC[JAC_WARPS][2][N][RCS];  // row sums sum_c M[a][c] dFx(c, b0), column sums sum_c M[b][c] dFy(a0, c)
  alignas(16) T FN[JAC_WARPS][NF][RCS];    // common face flux tangents
  T DQ[JAC_WARPS][2][N][2];                // physical gradient tangents on the two lines
  T rM[N][N], rdgL[N], rdgR[N], rlm[N], rlp[N], rw[N];  // reference operators in T
  int kf[4];
};

// NV consecutive values, 16-byte accesses where the layout allows them
template <typename T, int NV>
__device__ __forceinline__ void ldv(const T* p, T (&x)[NV]) {
  if constexpr (NV == 4 && sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
  } else if constexpr (NV == 4 && sizeof(T) == 8) {
    const double2 q0 = reinterpret_cast<const double2*>(p)[0], q1 = reinterpret_cast<const double2*>(p)[1];
    x[0] = q0.x; x[1] = q0.y; x[2] = q1.x; x[3] = q1.y;
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = p[v];
  }
}
template <typename T, int NV>
__device__ __forceinline__ void stv(T* p, const T (&x)[NV]) {
  if constexpr (NV == 4 && sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  } else if constexpr (NV == 4 && sizeof(T) == 8) {
    reinterpret_cast<double2*>(p)[0] = make_double2(x[0], x[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(x[2], x[3]);
  } else {
#pragma unroll
    for (int v = 0; v < NV; ++v) p[v] = x[v];
  }
}

// total flux F = F^c - F^v at a solution point
template <int PHYS, typename S, typename R, int NV>
__device__ __forceinline__ void vol_flux(const PhysConst<R>& pp, bool visc, const S* u, const S q[2][NV], S F[2][NV]) {
  Phys<PHYS>::template conv<S, R>(pp, u, F);
  if (visc) {
    S Fv[2][NV];
    Phys<PHYS>::template visc<S, R>(pp, u, q, Fv);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int v = 0; v < NV; ++v) F[c][v] = F[c][v] - Fv[c][v];
  }
}

// common normal flux J_f F^.n of an implicit element's face (trace or IMEX-interface face)
template <int PHYS, typename S, typename R, int NV>
__device__ __forceinline__ void imp_face_flux(const PhysConst<R>& pp, bool visc, int kf, const S* Uf, const S* ub,
                                              const S qf[2][NV], const S* un, R Jf, R n0, R n1, S* Fn) {
  S F[2][NV];
  if (kf == FK_TRACE) {
    Phys<PHYS>::template conv<S, R>(pp, ub, F);
    S s = Phys<PHYS>::template stab<S, R>(pp, ub, n0, n1);
#pragma unroll
    for (int v = 0; v < NV; ++v) Fn[v] = n0 * F[0][v] + n1 * F[1][v] + s * (Uf[v] - ub[v]);
    if (visc) {
      Phys<PHYS>::template visc<S, R>(pp, ub, qf, F);
#pragma unroll
      for (int v = 0; v < NV; ++v) Fn[v] = Fn[v] - (n0 * F[0][v] + n1 * F[1][v]);
    }
  } else {
    S G[2][NV];
    Phys<PHYS>::template conv<S, R>(pp, Uf, F);
    Phys<PHYS>::template conv<S, R>(pp, un, G);
    S lam = dmax(Phys<PHYS>::template wave<S, R>(pp, Uf, n0, n1), Phys<PHYS>::template wave<S, R>(pp, un, n0, n1));
#pragma unroll
    for (int v = 0; v < NV; ++v)
      Fn[v] = R(0.5) * (n0 * (F[0][v] + G[0][v]) + n1 * (F[1][v] + G[1][v])) + R(0.5) * lam * (Uf[v] - un[v]);
    if (visc) {
      Phys<PHYS>::template visc<S, R>(pp, Uf, qf, F);
#pragma unroll
      for (int v = 0; v < NV; ++v) Fn[v] = Fn[v] - (n0 * F[0][v] + n1 * F[1][v]);
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) Fn[v] = Jf * Fn[v];
}

template <int P, int PHYS, typename T>
__global__ void __launch_bounds__(JAC_THREADS, sizeof(T) == 4 ? (P <= 3 ? 4 : (P == 4 ? HFR_JAC_P4_BLOCKS : 2)) : 1) k_jacobian(const __grid_constant__ RefOps ref,
                                                          const __grid_constant__ PhysParams pp,
                                                          const __grid_constant__ JacArgs a) {
  using W = JacWork<P, PHYS, T>;
  using DT = Dual<T>;
  constexpr int N = W::N, NS = W::NS, NV = W::NV, NF = W::NF;
  constexpr int nA = NS * NV, nT = NF * NV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W& w = *reinterpret_cast<W*>(smem_raw);
  const int k = blockIdx.x;
  if (k >= a.Eim) return;
  const int e = a.imp_idx[k];
  const int tid = threadIdx.x;
  const bool visc = phys_viscous(pp);
  const PhysConst<T> pc = phys_const<T>(pp);
  const double* gs = a.geo_sol + (size_t)e * NS * 5;
  const double* gf = a.geo_face + (size_t)e * NF * 3;

  // ---------------------------------------------------------------- primal state (in T)
  for (int i = tid; i < nA; i += JAC_THREADS) w.U[i / NV][i % NV] = T(a.U[(size_t)e * nA + i]);
  for (int i = tid; i < NS; i += JAC_THREADS) {
    w.iJ[i] = T(gs[i * 5]);
    w.ciJ[i] = T(a.a_dt * gs[i * 5]);
    w.Sm[i][0][0] = T(gs[i * 5 + 1]);
    w.Sm[i][0][1] = T(gs[i * 5 + 2]);
    w.Sm[i][1][0] = T(gs[i * 5 + 3]);
    w.Sm[i][1][1] = T(gs[i * 5 + 4]);
  }
  for (int j = tid; j < NF; j += JAC_THREADS) {
    w.fJ[j] = T(gf[j * 3]);
    w.fn[j][0] = T(gf[j * 3 + 1]);
    w.fn[j][1] = T(gf[j * 3 + 2]);
  }
  if (tid < 4) w.kf[tid] = a.kind[e * 4 + tid];
  for (int i = tid; i < (int)(sizeof(w.LN) / sizeof(T)); i += JAC_THREADS) (&w.LN[0][0][0][0])[i] = T(0);
  for (int i = tid; i < (int)(sizeof(w.RC) / sizeof(T)); i += JAC_THREADS) (&w.RC[0][0][0][0])[i] = T(0);
  for (int i = tid; i < (int)(sizeof(w.FN) / sizeof(T)); i += JAC_THREADS) (&w.FN[0][0][0])[i] = T(0);
  for (int i = tid; i < N * N; i += JAC_THREADS) w.rM[i / N][i % N] = T(ref.M[i / N][i % N]);
  if (tid < N) {
    w.rdgL[tid] = T(ref.dgL[tid]);
    w.rdgR[tid] = T(ref.dgR[tid]);
    w.rlm[tid] = T(ref.lm[tid]);
    w.rlp[tid] = T(ref.lp[tid]);
    w.rw[tid] = T(ref.w[tid]);
  }
  __syncthreads();
  // one thread per (flux point, variable): face values, then the trace or the neighbour's state
  for (int it = tid; it < NF * NV; it += JAC_THREADS) {
    const int j = it / NV, v = it % NV;
    const int f = j / N, m = j % N, r = f >> 1;
    const T* l = (f & 1) ? w.rlp : w.rlm;
    T s = T(0);
#pragma unroll
    for (int c = 0; c < N; ++c) s += l[c] * w.U[line_pt<N>(r, m, c)][v];
    w.Uf[j][v] = s;
    if (w.kf[f] == FK_TRACE) {
      const int t = (int)FR_IDX(a.tr_of[e * 4 + f], a.ntrace, 23);
      w.ub[j][v] = T(a.uhat[((size_t)t * N + m) * NV + v]);
      w.un[j][v] = s;
    } else {  // interface face: explicit neighbour's state is the common solution
      const int en = (int)FR_IDX(a.nbr[e * 4 + f], a.E, 24), fnb = (int)FR_IDX(a.nbr_face[e * 4 + f], 4, 25);
      const T un = T(a.Uf_all[((size_t)en * NF + fnb * N + m) * NV + v]);
      w.un[j][v] = un;
      w.ub[j][v] = un;
    }
  }
  __syncthreads();
  if (visc) {
    for (int it = tid; it < NS * NV; it += JAC_THREADS) {  // one thread per (point, variable)
      const int i = it / NV, v = it % NV;
      const int ai = i % N, bi = i / N;
      T q0 = w.rdgL[ai] * w.ub[bi][v] + w.rdgR[ai] * w.ub[N + bi][v];
      T q1 = w.rdgL[bi] * w.ub[2 * N + ai][v] + w.rdgR[bi] * w.ub[3 * N + ai][v];
#pragma unroll
      for (int c = 0; c < N; ++c) {
        q0 += w.rM[ai][c] * w.U[c + N * bi][v];
        q1 += w.rM[bi][c] * w.U[ai + N * c][v];
      }
      w.q[i][0][v] = w.iJ[i] * (w.Sm[i][0][0] * q0 + w.Sm[i][1][0] * q1);
      w.q[i][1][v] = w.iJ[i] * (w.Sm[i][0][1] * q0 + w.Sm[i][1][1] * q1);
    }
    __syncthreads();
    for (int it = tid; it < NF * 2 * NV; it += JAC_THREADS) {  // (flux point, direction, variable)
      const int j = it / (2 * NV), c2 = (it / NV) % 2, v = it % NV;
      const int f = j / N, m = j % N, r = f >> 1;
      const T* l = (f & 1) ? w.rlp : w.rlm;
      T s = T(0);
#pragma unroll
      for (int c = 0; c < N; ++c) s += l[c] * w.q[line_pt<N>(r, m, c)][c2][v];
      w.qf[j][c2][v] = s;
    }
  } else {
    for (int i = tid; i < NS * 2 * NV; i += JAC_THREADS) (&w.q[0][0][0])[i] = T(0);
    for (int i = tid; i < NF * 2 * NV; i += JAC_THREADS) (&w.qf[0][0][0])[i] = T(0);
  }
  __syncthreads();

  // -------------------------------------------------- 1. pointwise Jacobians (dual numbers)
  // volume: items (point, input variable) for the state, then the same for the gradient, each
  // range padded to whole warps so that a warp takes one branch
  constexpr int NI = (NS * NV + 31) / 32 * 32;
  for (int it = tid; it < 2 * NI; it += JAC_THREADS) {
    const bool isq = it >= NI;
    const int idx = isq ? it - NI : it;
    if (idx >= NS * NV) continue;
    const int i = idx / NV, vp = idx % NV;
    DT u[NV], qd[2][NV], F[2][NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      u[v] = DT(w.U[i][v], (!isq && v == vp) ? T(1) : T(0));
      qd[0][v] = DT(w.q[i][0][v]);
      qd[1][v] = DT(w.q[i][1][v]);
    }
    if (!isq) {
      vol_flux<PHYS, DT, T, NV>(pc, visc, u, qd, F);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int v = 0; v < NV; ++v) w.KU[i][r][v][vp] = w.Sm[i][r][0] * F[0][v].d + w.Sm[i][r][1] * F[1][v].d;
    } else {
      // only the viscous flux depends on the gradient: dF/dq = -dF^v/dq
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
              T dFr = -(w.Sm[i][r][0] * F[0][v].d + w.Sm[i][r][1] * F[1][v].d);  // d F~_r / d q_{c2}
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
  // face: items (flux point, input direction) over (u_f, u^, q_f x, q_f y)
  for (int it = tid; it < NF * 4 * NV; it += JAC_THREADS) {
    const int j = it / (4 * NV), dir = it % (4 * NV);
    const int grp = dir / NV, vp = dir % NV;
    const int kf = w.kf[j / N];
    DT Uf[NV], ub[NV], un[NV], qf[2][NV], Fn[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      Uf[v] = DT(w.Uf[j][v], (grp == 0 && v == vp) ? T(1) : T(0));
      ub[v] = DT(w.ub[j][v], (grp == 1 && v == vp) ? T(1) : T(0));
      un[v] = DT(w.un[j][v]);
      qf[0][v] = DT(w.qf[j][0][v], (grp == 2 && v == vp) ? T(1) : T(0));
      qf[1][v] = DT(w.qf[j][1][v], (grp == 3 && v == vp) ? T(1) : T(0));
    }
    bool zero = (grp >= 2 && !visc) || (grp == 1 && kf != FK_TRACE);
    if (!zero) imp_face_flux<PHYS, DT, T, NV>(pc, visc, kf, Uf, ub, qf, un, w.fJ[j], w.fn[j][0], w.fn[j][1], Fn);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T d = zero ? T(0) : Fn[v].d;
      if (grp == 0) w.GU[j][v][vp] = d;
      else if (grp == 1) w.GH[j][v][vp] = d;
      else w.GQ[j][grp - 2][v][vp] = d;
    }
  }
  __syncthreads();

  // ------------------------------------------------ 2-3. columns, one seed point per warp
  // A seed point is a solution point P0 = (a0, b0) (NV columns of A and C) or a flux point j0
  // of a trace face (NV columns of B and D).  Its unit seeds move the reference gradient only on
  // the grid row b0 (dQ_xi) and the grid column a0 (dQ_eta) through P0, or on the one line of
  // points normal to the seeded face, so the flux tangents are formed on those lines alone and
  // every output follows from them and the face tangents:
  //   dR(ai, bi) = -1/J [ sum_c M[ai][c] dFx(c, bi) + M[bi][c] dFy(ai, c)
  //                       - dgL[ai] dFn(xi-, bi) + dgR[ai] dFn(xi+, bi)
  //                       - dgL[bi] dFn(eta-, ai) + dgR[bi] dFn(eta+, ai) ]
  //   dg^k(f, m) = w_m dFn(f, m)   (trace faces)
  // dFx(., bi) vanishes off the row b0 except at c = a0 and dFy(ai, .) off the column a0 except
  // at c = b0, so with the line sums RC formed once per seed point every output is two
  // one-term products and the four face terms.  Lane (v, g): output variable v, lane group g;
  // each lane carries the NV seed variables v0 of the point (NV-wide loads and stores).  The
  // warp's buffers are its own: no block barrier between seed points.
  constexpr int G = 32 / NV, LNS = W::LNS, RCS = W::RCS;
  const int lane = tid & 31, wp = tid >> 5;
  const int vv = lane % NV, g = lane / NV;
  T(*LN)[N][LNS] = w.LN[wp];
  T(*RC)[N][RCS] = w.RC[wp];
  T(*FN)[RCS] = w.FN[wp];
  T(*DQ)[N][2] = w.DQ[wp];
  T* A = reinterpret_cast<T*>(a.A) + (size_t)k * nA * nA;
  T* B = reinterpret_cast<T*>(a.B) + (size_t)k * nA * nT;
  T* C = reinterpret_cast<T*>(a.C) + (size_t)k * nT * nA;
  T* Dm = reinterpret_cast<T*>(a.D) + (size_t)k * nT * nT;
  for (int sp = wp; sp < NS + NF; sp += JAC_WARPS) {
    const bool vol = sp < NS;
    int a0, b0;
    bool has_row, has_col, active;
    const T* dgs = w.rdgL;  // weights of a trace seed along its line
    if (vol) {
      a0 = sp % N;
      b0 = sp / N;
      has_row = has_col = active = true;
    } else {
      const int f0 = (sp - NS) / N, m0 = (sp - NS) % N;
      active = w.kf[f0] == FK_TRACE;
      has_row = (f0 >> 1) == 0;  // xi faces move dQ_xi on the grid row m0
      has_col = !has_row;        // eta faces move dQ_eta on the grid column m0
      a0 = b0 = m0;
      if (f0 & 1) dgs = w.rdgR;
    }
    // reference-gradient tangents (dQ_xi, dQ_eta) at point c of line 0 (row b0) or 1 (column a0)
    auto seed_dq = [&](int line, int c, T& dQ0, T& dQ1) {
      if (line == 0) {
        dQ0 = vol ? w.rM[c][a0] : dgs[c];
        dQ1 = (vol && c == a0) ? w.rM[b0][b0] : T(0);
      } else {
        dQ1 = vol ? w.rM[c][b0] : dgs[c];
        dQ0 = (vol && c == b0) ? w.rM[a0][a0] : T(0);
      }
    };
    if (active) {
      // physical gradient tangents on the lines (independent of v0)
      if (lane < 4 * N) {
        const int line = lane / (2 * N), c = (lane >> 1) % N, c2 = lane & 1;
        if (line == 0 ? has_row : has_col) {
          const int pt = line == 0 ? c + N * b0 : a0 + N * c;
          T dQ0, dQ1;
          seed_dq(line, c, dQ0, dQ1);
          DQ[line][c][c2] = w.iJ[pt] * (w.Sm[pt][0][c2] * dQ0 + w.Sm[pt][1][c2] * dQ1);
        }
      }
      __syncwarp();
      // flux tangents on the lines, then the common face flux tangents
      for (int it = g; it < 2 * N + NF && g < G; it += G) {
        if (it < 2 * N) {
          const int line = it / N, c = it % N;
          if (!(line == 0 ? has_row : has_col)) continue;
          const int pt = line == 0 ? c + N * b0 : a0 + N * c;
          T dQ0, dQ1;
          seed_dq(line, c, dQ0, dQ1);
          const bool self = vol && pt == sp;
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            T k0[NV], k1[NV], o[NV];
            ldv<T, NV>(&w.KQ[pt][r][0][vv][0], k0);
            ldv<T, NV>(&w.KQ[pt][r][1][vv][0], k1);
#pragma unroll
            for (int x = 0; x < NV; ++x) o[x] = k0[x] * dQ0 + k1[x] * dQ1;
            if (self) {
              ldv<T, NV>(&w.KU[pt][r][vv][0], k0);
#pragma unroll
              for (int x = 0; x < NV; ++x) o[x] += k0[x];
            }
            stv<T, NV>(&LN[line][c][(r * NV + vv) * NV], o);
          }
        } else {
          const int j = it - 2 * N, f = j / N, m = j % N;
          const T* l = (f & 1) ? w.rlp : w.rlm;
          T dUf = T(0), q0 = T(0), q1 = T(0);
          if ((f >> 1) == 0) {  // xi face: flux points along the grid row m
            if (has_row && m == b0) {
#pragma unroll
              for (int c = 0; c < N; ++c) {
                q0 += l[c] * DQ[0][c][0];
                q1 += l[c] * DQ[0][c][1];
              }
            } else if (has_col) {
              q0 = l[a0] * DQ[1][m][0];
              q1 = l[a0] * DQ[1][m][1];
            }
            if (vol && m == b0) dUf = l[a0];
          } else {  // eta face: flux points along the grid column m
            if (has_col && m == a0) {
#pragma unroll
              for (int c = 0; c < N; ++c) {
                q0 += l[c] * DQ[1][c][0];
                q1 += l[c] * DQ[1][c][1];
              }
            } else if (has_row) {
              q0 = l[b0] * DQ[0][m][0];
              q1 = l[b0] * DQ[0][m][1];
            }
            if (vol && m == a0) dUf = l[b0];
          }
          T gu[NV], g0[NV], g1[NV], o[NV];
          ldv<T, NV>(&w.GU[j][vv][0], gu);
          ldv<T, NV>(&w.GQ[j][0][vv][0], g0);
          ldv<T, NV>(&w.GQ[j][1][vv][0], g1);
#pragma unroll
          for (int x = 0; x < NV; ++x) o[x] = gu[x] * dUf + g0[x] * q0 + g1[x] * q1;
          if (!vol && j == sp - NS) {
            ldv<T, NV>(&w.GH[j][vv][0], gu);
#pragma unroll
            for (int x = 0; x < NV; ++x) o[x] += gu[x];
          }
          stv<T, NV>(&FN[j][vv * NV], o);
        }
      }
      __syncwarp();
      // line sums: RC[0][ai] = sum_c M[ai][c] dFx(c, b0), RC[1][bi] = sum_c M[bi][c] dFy(a0, c)
      for (int it = g; it < 2 * N && g < G; it += G) {
        const int line = it / N, e = it % N;
        if (!(line == 0 ? has_row : has_col)) continue;
        T o[NV], t[NV];
#pragma unroll
        for (int x = 0; x < NV; ++x) o[x] = T(0);
#pragma unroll
        for (int c = 0; c < N; ++c) {
          ldv<T, NV>(&LN[line][c][(line * NV + vv) * NV], t);
          const T mc = w.rM[e][c];
#pragma unroll
          for (int x = 0; x < NV; ++x) o[x] += mc * t[x];
        }
        stv<T, NV>(&RC[line][e][vv * NV], o);
      }
      __syncwarp();
    }
    // outputs (the buffers are zeroed at entry, so a line the seed does not have reads finite
    // values that are multiplied by zero)
    for (int it = g; it < NS + NF && g < G; it += G) {
      T o[NV];
      T* dst;
      if (it < NS) {
        const int ai = it % N, bi = it / N;
#pragma unroll
        for (int x = 0; x < NV; ++x) o[x] = T(0);
        if (active) {
          T t[NV];
          const bool xrow = has_row && bi == b0, ycol = has_col && ai == a0;
          const T cx = xrow ? T(1) : (has_col ? w.rM[ai][a0] : T(0));
          const T cy = ycol ? T(1) : (has_row ? w.rM[bi][b0] : T(0));
          ldv<T, NV>(xrow ? &RC[0][ai][vv * NV] : &LN[1][bi][vv * NV], t);
#pragma unroll
          for (int x = 0; x < NV; ++x) o[x] = cx * t[x];
          ldv<T, NV>(ycol ? &RC[1][bi][vv * NV] : &LN[0][ai][(NV + vv) * NV], t);
#pragma unroll
          for (int x = 0; x < NV; ++x) o[x] += cy * t[x];
          const T cxm = -w.rdgL[ai], cxp = w.rdgR[ai], cym = -w.rdgL[bi], cyp = w.rdgR[bi];
          ldv<T, NV>(&FN[bi][vv * NV], t);
#pragma unroll
          for (int x = 0; x < NV; ++x) o[x] += cxm * t[x];
          ldv<T, NV>(&FN[N + bi][vv * NV], t);
#pragma unroll
          for (int x = 0; x < NV; ++x) o[x] += cxp * t[x];
          ldv<T, NV>(&FN[2 * N + ai][vv * NV], t);
#pragma unroll
          for (int x = 0; x < NV; ++x) o[x] += cym * t[x];
          ldv<T, NV>(&FN[3 * N + ai][vv * NV], t);
#pragma unroll
          for (int x = 0; x < NV; ++x) o[x] += cyp * t[x];
          const T cj = w.ciJ[it];
#pragma unroll
          for (int x = 0; x < NV; ++x) o[x] *= cj;  // A = I - a dt dR, B = -a dt dR
        }
        if (vol && it == sp) {
#pragma unroll
          for (int x = 0; x < NV; ++x)
            if (x == vv) o[x] += T(1);
        }
        const int i = it * NV + vv;
        dst = vol ? A + (size_t)i * nA + sp * NV : B + (size_t)i * nT + (sp - NS) * NV;
      } else {
        const int j = it - NS, m = j % N;
        if (active && w.kf[j / N] == FK_TRACE) {
          ldv<T, NV>(&FN[j][vv * NV], o);
          const T wm = w.rw[m];
#pragma unroll
          for (int x = 0; x < NV; ++x) o[x] *= wm;
        } else {
#pragma unroll
          for (int x = 0; x < NV; ++x) o[x] = T(0);
        }
        const int lr = j * NV + vv;
        dst = vol ? C + (size_t)lr * nA + sp * NV : Dm + (size_t)lr * nT + (sp - NS) * NV;
      }
      stv<T, NV>(dst, o);
    }
    __syncwarp();  // the next seed point rewrites this warp's buffers
  }
}

template <int P, int PHYS, typename T>
static cudaError_t jac_impl(const RefOps& ref, const PhysParams& pp, const JacArgs& a, cudaStream_t st) {
  size_t smem = sizeof(JacWork<P, PHYS, T>);
  auto kern = k_jacobian<P, PHYS, T>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  // several CTAs per SM: ask for the largest shared-memory carveout
  err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (err != cudaSuccess) return err;
  if (a.Eim == 0) return cudaSuccess;
  (hfr::count_launch(), kern<<<a.Eim, JAC_THREADS, smem, st>>>(ref, pp, a));
  return cudaGetLastError();
}

template <typename T>
static cudaError_t jac_dispatch(int p, const RefOps& ref, const PhysParams& pp, const JacArgs& a, cudaStream_t st) {
  if (pp.kind == 0) {
    switch (p) {
      case 1: return jac_impl<1, 0, T>(ref, pp, a, st);
      case 2: return jac_impl<2, 0, T>(ref, pp, a, st);
      case 3: return jac_impl<3, 0, T>(ref, pp, a, st);
    }
  } else if (pp.kind == 2) {
    switch (p) {
      case 2: return jac_impl<2, 2, T>(ref, pp, a, st);
      case 3: return jac_impl<3, 2, T>(ref, pp, a, st);
      case 4: return jac_impl<4, 2, T>(ref, pp, a, st);
    }
  } else {
    switch (p) {
      case 2: return jac_impl<2, 1, T>(ref, pp, a, st);
      case 3: return jac_impl<3, 1, T>(ref, pp, a, st);
      case 4: return jac_impl<4, 1, T>(ref, pp, a, st);
      case 5: return jac_impl<5, 1, T>(ref, pp, a, st);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_jacobian(int p, int prec_bytes, const RefOps& ref, const PhysParams& pp, const JacArgs& a,
                            cudaStream_t st) {
  if (prec_bytes == 8) return jac_dispatch<double>(p, ref, pp, a, st);
  return jac_dispatch<float>(p, ref, pp, a, st);
}

}  // namespace hfr

#include "hfr_checked_unit.inc"
