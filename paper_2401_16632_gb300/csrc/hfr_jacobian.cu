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
//   2. per seed (a column of the blocks), the tangent of the corrected gradient is nonzero
//      only on the two grid lines through the seeded point (or on the one line normal to
//      the seeded trace point), so the flux tangents are formed only there;
//   3. the output column follows from the 1D operators M, dgL, dgR along the lines.
// Work per element is O((nA + nT)^2 n), not the O((nA + nT) x residual) of a dense sweep.
// T = double (plain path) or float (mixed path; blocks stored in FP32).
#include "hfr_internal.h"

namespace hfr {

constexpr int JAC_THREADS = 256;
constexpr int JAC_SB = 32;  // seeds per batch

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
  T KU[NS][2][NV][NV];
  T KQ[NS][2][2][NV][NV];
  T GU[NF][NV][NV];
  T GH[NF][NV][NV];
  T GQ[NF][2][NV][NV];
  T dFt[NS][2][NV][JAC_SB];
  T dq[NS][2][JAC_SB];
  T dFn[NF][NV][JAC_SB];
  T rM[N][N], rdgL[N], rdgR[N], rlm[N], rlp[N], rw[N];  // reference operators in T
  int kf[4];
};

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
__global__ void __launch_bounds__(JAC_THREADS, sizeof(T) == 4 ? (P <= 3 ? 4 : (P == 4 ? 3 : 2)) : 1) k_jacobian(const __grid_constant__ RefOps ref,
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
  for (int i = tid; i < N * N; i += JAC_THREADS) w.rM[i / N][i % N] = T(ref.M[i / N][i % N]);
  if (tid < N) {
    w.rdgL[tid] = T(ref.dgL[tid]);
    w.rdgR[tid] = T(ref.dgR[tid]);
    w.rlm[tid] = T(ref.lm[tid]);
    w.rlp[tid] = T(ref.lp[tid]);
    w.rw[tid] = T(ref.w[tid]);
  }
  __syncthreads();
  for (int j = tid; j < NF; j += JAC_THREADS) {
    const int f = j / N, m = j % N, r = f >> 1;
    const T* l = (f & 1) ? w.rlp : w.rlm;
    const int kf = w.kf[f];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T s = T(0);
#pragma unroll
      for (int c = 0; c < N; ++c) s += l[c] * w.U[line_pt<N>(r, m, c)][v];
      w.Uf[j][v] = s;
    }
    if (kf == FK_TRACE) {
      const int t = a.tr_of[e * 4 + f];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        w.ub[j][v] = T(a.uhat[((size_t)t * N + m) * NV + v]);
        w.un[j][v] = w.Uf[j][v];
      }
    } else {  // interface face: explicit neighbour's state is the common solution
      const int en = a.nbr[e * 4 + f], fnb = a.nbr_face[e * 4 + f];
      const double* un = a.Uf_all + ((size_t)en * NF + fnb * N + m) * NV;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        w.un[j][v] = T(un[v]);
        w.ub[j][v] = T(un[v]);
      }
    }
  }
  __syncthreads();
  if (visc) {
    for (int i = tid; i < NS; i += JAC_THREADS) {
      const int ai = i % N, bi = i / N;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
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
    }
    __syncthreads();
    for (int j = tid; j < NF; j += JAC_THREADS) {
      const int f = j / N, m = j % N, r = f >> 1;
      const T* l = (f & 1) ? w.rlp : w.rlm;
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T s = T(0);
#pragma unroll
          for (int c = 0; c < N; ++c) s += l[c] * w.q[line_pt<N>(r, m, c)][c2][v];
          w.qf[j][c2][v] = s;
        }
    }
  } else {
    for (int i = tid; i < NS * 2 * NV; i += JAC_THREADS) (&w.q[0][0][0])[i] = T(0);
    for (int i = tid; i < NF * 2 * NV; i += JAC_THREADS) (&w.qf[0][0][0])[i] = T(0);
  }
  __syncthreads();

  // -------------------------------------------------- 1. pointwise Jacobians (dual numbers)
  // volume: items (point, input variable, state-or-gradient)
  for (int it = tid; it < NS * NV * 2; it += JAC_THREADS) {
    const int i = it / (2 * NV), vp = (it / 2) % NV, isq = it % 2;
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
          vol_flux<PHYS, DT, T, NV>(pc, visc, u, qd, F);
          qd[c2][vp].d = T(0);
#pragma unroll
          for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              T dFr = w.Sm[i][r][0] * F[0][v].d + w.Sm[i][r][1] * F[1][v].d;  // d F~_r / d q_{c2}
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

  // ----------------------------------------------------------- 2-3. columns in batches
  const T adt = T(a.a_dt);
  T* A = reinterpret_cast<T*>(a.A) + (size_t)k * nA * nA;
  T* B = reinterpret_cast<T*>(a.B) + (size_t)k * nA * nT;
  T* C = reinterpret_cast<T*>(a.C) + (size_t)k * nT * nA;
  T* Dm = reinterpret_cast<T*>(a.D) + (size_t)k * nT * nT;
  constexpr int NSEED = nA + nT;
  for (int s0 = 0; s0 < NSEED; s0 += JAC_SB) {
    // 2a. tangents of the reference gradient and of the transformed flux on the seed's lines
    for (int it = tid; it < NS * JAC_SB; it += JAC_THREADS) {
      const int s = it % JAC_SB, i = it / JAC_SB;
      const int sd = s0 + s;
      const int ai = i % N, bi = i / N;
      T dQ0 = T(0), dQ1 = T(0);
      int v0 = 0;
      bool self = false;
      if (sd < nA) {
        const int P0 = sd / NV;
        v0 = sd % NV;
        const int a0 = P0 % N, b0 = P0 / N;
        if (bi == b0) dQ0 = w.rM[ai][a0];
        if (ai == a0) dQ1 = w.rM[bi][b0];
        self = (i == P0);
      } else if (sd < NSEED) {
        const int l = sd - nA;
        const int f0 = l / (N * NV), m0 = (l / NV) % N;
        v0 = l % NV;
        if (w.kf[f0] == FK_TRACE) {
          const T* dg = (f0 & 1) ? w.rdgR : w.rdgL;
          if ((f0 >> 1) == 0) {
            if (bi == m0) dQ0 = dg[ai];
          } else {
            if (ai == m0) dQ1 = dg[bi];
          }
        }
      }
      w.dq[i][0][s] = w.iJ[i] * (w.Sm[i][0][0] * dQ0 + w.Sm[i][1][0] * dQ1);
      w.dq[i][1][s] = w.iJ[i] * (w.Sm[i][0][1] * dQ0 + w.Sm[i][1][1] * dQ1);
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          T d = w.KQ[i][r][0][v][v0] * dQ0 + w.KQ[i][r][1][v][v0] * dQ1;
          if (self) d += w.KU[i][r][v][v0];
          w.dFt[i][r][v][s] = d;
        }
    }
    __syncthreads();
    // 2b. tangents of the common face fluxes
    for (int it = tid; it < NF * JAC_SB; it += JAC_THREADS) {
      const int s = it % JAC_SB, j = it / JAC_SB;
      const int sd = s0 + s;
      const int f = j / N, m = j % N, r = f >> 1;
      const T* l = (f & 1) ? w.rlp : w.rlm;
      T dUf = T(0);
      int v0 = 0;
      bool selft = false;
      if (sd < nA) {
        const int P0 = sd / NV;
        v0 = sd % NV;
        const int a0 = P0 % N, b0 = P0 / N;
        const int along = r == 0 ? a0 : b0, line = r == 0 ? b0 : a0;
        if (m == line) dUf = l[along];
      } else if (sd < NSEED) {
        const int lt = sd - nA;
        v0 = lt % NV;
        selft = (lt / NV) == j && w.kf[f] == FK_TRACE;
      }
      T dqf0 = T(0), dqf1 = T(0);
#pragma unroll
      for (int c = 0; c < N; ++c) {
        const int pt = line_pt<N>(r, m, c);
        dqf0 += l[c] * w.dq[pt][0][s];
        dqf1 += l[c] * w.dq[pt][1][s];
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T d = w.GU[j][v][v0] * dUf + w.GQ[j][0][v][v0] * dqf0 + w.GQ[j][1][v][v0] * dqf1;
        if (selft) d += w.GH[j][v][v0];
        w.dFn[j][v][s] = d;
      }
    }
    __syncthreads();
    // 3. output columns.  Thread (s, v, part): seed s of the batch, variable v, and the grid rows
    // bi = part (mod NPART) and faces f = part (mod NPART) of the element.  The y-direction flux
    // tangents of the element sit in registers; each tangent loaded from shared memory feeds
    // several outputs (the 1D operators are shared-memory broadcasts):
    //   dR(ai, bi) = -iJ [ sum_c M[ai][c] dF~x(c, bi) + M[bi][c] dF~y(ai, c)
    //                      - dgL[ai] dFn(xi-, bi) + dgR[ai] dFn(xi+, bi)
    //                      - dgL[bi] dFn(eta-, ai) + dgR[bi] dFn(eta+, ai) ]
    //   dg^k(f, m) = w_m dFn(f, m)   (trace faces)
    constexpr int NPART = JAC_THREADS / (JAC_SB * NV);  // threads beyond NPART JAC_SB NV idle here
    static_assert(NPART >= 1, "phase 3 thread map");
    {
      const int s = tid % JAC_SB;
      const int v = (tid / JAC_SB) % NV;
      const int part = tid / (JAC_SB * NV);
      const int sd = s0 + s;
      if (sd < NSEED && part < NPART) {
        T dgl[N], dgr[N];
#pragma unroll
        for (int x = 0; x < N; ++x) {
          dgl[x] = w.rdgL[x];
          dgr[x] = w.rdgR[x];
        }
        T dyt[N][N];  // dF~y(ai, c) for all ai, c
#pragma unroll
        for (int ai = 0; ai < N; ++ai)
#pragma unroll
          for (int c = 0; c < N; ++c) dyt[ai][c] = w.dFt[ai + N * c][1][v][s];
        T fym[N], fyp[N];  // eta-, eta+ face tangents at every ai
#pragma unroll
        for (int ai = 0; ai < N; ++ai) {
          fym[ai] = w.dFn[2 * N + ai][v][s];
          fyp[ai] = w.dFn[3 * N + ai][v][s];
        }
        constexpr int RPP = (N + NPART - 1) / NPART;  // rows per part
        for (int rb = 0; rb < RPP; ++rb) {
          const int bi = part + NPART * rb;
          if (bi < N) {
            T dxt[N], rMb[N];
#pragma unroll
            for (int c = 0; c < N; ++c) {
              dxt[c] = w.dFt[c + N * bi][0][v][s];
              rMb[c] = w.rM[bi][c];
            }
            const T fxm = w.dFn[bi][v][s], fxp = w.dFn[N + bi][v][s];
            const T dglb = w.rdgL[bi], dgrb = w.rdgR[bi];
#pragma unroll
            for (int ai = 0; ai < N; ++ai) {
              T d = -dgl[ai] * fxm + dgr[ai] * fxp - dglb * fym[ai] + dgrb * fyp[ai];
#pragma unroll
              for (int c = 0; c < N; ++c) d += w.rM[ai][c] * dxt[c] + rMb[c] * dyt[ai][c];
              const int pt = ai + N * bi;
              const int i = pt * NV + v;
              const T dR = -w.iJ[pt] * d;
              if (sd < nA)
                A[(size_t)i * nA + sd] = (i == sd ? T(1) : T(0)) - adt * dR;
              else
                B[(size_t)i * nT + (sd - nA)] = -adt * dR;
            }
          }
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          if (f % NPART != part) continue;
          const bool tr = w.kf[f] == FK_TRACE;
#pragma unroll
          for (int m = 0; m < N; ++m) {
            const int lr = (f * N + m) * NV + v;
            const T val = tr ? w.rw[m] * w.dFn[f * N + m][v][s] : T(0);
            if (sd < nA)
              C[(size_t)lr * nA + sd] = val;
            else
              Dm[(size_t)lr * nT + (sd - nA)] = val;
          }
        }
      }
    }
    __syncthreads();
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
