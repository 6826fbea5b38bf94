// FR / hybridized-FR residual kernels (Pereira & Vermeire, arXiv 2401.16632, Sec. 2:
// eqs. freq1, hfrriemann, hfr1; transmission conditions eqs. 5treerf, hfr2; IMEX
// interface eq. hfrimex).
//
// One thread group of TPE threads per element, EPB elements per CTA; every per-element
// intermediate lives in shared memory.  The element computation is a template on the
// scalar type S: S = double gives the residual, S = Dual<double> gives the residual and its
// exact directional derivative (used for FP64 refinement residuals of the local solves).
#include "hfr_internal.h"

namespace hfr {

template <int P, int PHYS, typename S>
struct ElemWork {
  static constexpr int N = P + 1, NS = N * N, NV = Phys<PHYS>::NV, NF = 4 * N;
  S U[NS][NV];
  S Uf[NF][NV];
  S ub[NF][NV];
  S q[NS][2][NV];
  S qf[NF][2][NV];
  S Ft[NS][2][NV];
  S Fn[NF][NV];
};

template <typename S> __device__ __forceinline__ S mk(double v, double d);
template <> __device__ __forceinline__ double mk<double>(double v, double) { return v; }
template <> __device__ __forceinline__ Dual<double> mk<Dual<double>>(double v, double d) { return Dual<double>(v, d); }
__device__ __forceinline__ double tangent(double) { return 0.0; }
__device__ __forceinline__ double tangent(Dual<double> a) { return a.d; }

// Modes of the element kernel.
enum { MODE_UF = 0, MODE_QF = 1, MODE_RES = 2 };

template <int P, int PHYS, typename S, int MODE, int TPE, int EPB>
__global__ void __launch_bounds__(TPE* EPB) k_element(const __grid_constant__ RefOps ref,
                                                      const __grid_constant__ PhysParams pp,
                                                      const __grid_constant__ ResArgs a) {
  using W = ElemWork<P, PHYS, S>;
  constexpr int N = W::N, NS = W::NS, NV = W::NV, NF = W::NF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  W* works = reinterpret_cast<W*>(smem_raw);
  const int g = threadIdx.x / TPE;
  const int lt = threadIdx.x % TPE;
  const int e = blockIdx.x * EPB + g;
  const bool live = e < a.E;
  W& w = works[g];
  const bool viscous = phys_viscous(pp);
  const PhysConst<double> pc = phys_const<double>(pp);
  const bool is_imp = live ? (a.implicit[e] != 0) : false;
  const double* gs = a.geo_sol + (size_t)e * NS * 5;
  const double* gf = a.geo_face + (size_t)e * NF * 3;

  // 1. state
  if (live) {
    for (int i = lt; i < NS * NV; i += TPE) {
      double v = a.U[(size_t)e * NS * NV + i];
      double d = a.dU ? a.dU[(size_t)e * NS * NV + i] : 0.0;
      w.U[i / NV][i % NV] = mk<S>(v, d);
    }
  }
  __syncthreads();
  // 2. face states and common solution
  if (live) {
    for (int j = lt; j < NF; j += TPE) {
      const int f = j / N, m = j % N, r = f >> 1;
      const double* l = (f & 1) ? ref.lp : ref.lm;
      const int kf = a.kind[e * 4 + f];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        S s = S(0.0);
#pragma unroll
        for (int c = 0; c < N; ++c) s = s + l[c] * w.U[line_pt<N>(r, m, c)][v];
        w.Uf[j][v] = s;
      }
      if (MODE == MODE_UF) {
#pragma unroll
        for (int v = 0; v < NV; ++v) a.Uf_out[((size_t)e * NF + j) * NV + v] = dval(w.Uf[j][v]);
        continue;
      }
      if (kf == FK_TRACE) {
        const int t = (int)FR_IDX(a.tr_of[e * 4 + f], a.ntrace, 20);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          size_t ix = ((size_t)t * N + m) * NV + v;
          w.ub[j][v] = mk<S>(a.uhat[ix], a.duhat ? a.duhat[ix] : 0.0);
        }
      } else {
        const int en = (int)FR_IDX(a.nbr[e * 4 + f], a.E, 21), fn = (int)FR_IDX(a.nbr_face[e * 4 + f], 4, 22);
        const double* un = a.Uf_all + ((size_t)en * NF + fn * N + m) * NV;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if (kf == FK_FR)
            w.ub[j][v] = 0.5 * (w.Uf[j][v] + S(un[v]));
          else  // IMEX interface: explicit side's value
            w.ub[j][v] = is_imp ? S(un[v]) : w.Uf[j][v];
        }
      }
    }
  }
  if (MODE == MODE_UF) return;
  __syncthreads();
  // 3. corrected gradient at the solution points
  if (live && viscous) {
    for (int i = lt; i < NS; i += TPE) {
      const int ai = i % N, bi = i / N;
      const double* G = gs + i * 5;
      const double iJ = G[0];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        S q0 = ref.dgL[ai] * w.ub[0 * N + bi][v] + ref.dgR[ai] * w.ub[1 * N + bi][v];
        S q1 = ref.dgL[bi] * w.ub[2 * N + ai][v] + ref.dgR[bi] * w.ub[3 * N + ai][v];
#pragma unroll
        for (int c = 0; c < N; ++c) {
          q0 = q0 + ref.M[ai][c] * w.U[c + N * bi][v];
          q1 = q1 + ref.M[bi][c] * w.U[ai + N * c][v];
        }
        w.q[i][0][v] = iJ * (G[1] * q0 + G[3] * q1);
        w.q[i][1][v] = iJ * (G[2] * q0 + G[4] * q1);
      }
    }
  }
  __syncthreads();
  // 4. transformed flux at the solution points, gradient at the flux points
  if (live) {
    if (MODE == MODE_RES) {
      for (int i = lt; i < NS; i += TPE) {
        const double* G = gs + i * 5;
        S F[2][NV];
        Phys<PHYS>::template conv<S, double>(pc, w.U[i], F);
        if (viscous) {
          S Fv[2][NV];
          Phys<PHYS>::template visc<S, double>(pc, w.U[i], w.q[i], Fv);
#pragma unroll
          for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int v = 0; v < NV; ++v) F[c][v] = F[c][v] - Fv[c][v];
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          w.Ft[i][0][v] = G[1] * F[0][v] + G[2] * F[1][v];
          w.Ft[i][1][v] = G[3] * F[0][v] + G[4] * F[1][v];
        }
      }
    }
    if (viscous) {
      for (int j = lt; j < NF; j += TPE) {
        const int f = j / N, m = j % N, r = f >> 1;
        const double* l = (f & 1) ? ref.lp : ref.lm;
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            S s = S(0.0);
#pragma unroll
            for (int c = 0; c < N; ++c) s = s + l[c] * w.q[line_pt<N>(r, m, c)][c2][v];
            w.qf[j][c2][v] = s;
          }
        if (MODE == MODE_QF) {
#pragma unroll
          for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
            for (int v = 0; v < NV; ++v) a.qf_out[(((size_t)e * NF + j) * 2 + c2) * NV + v] = dval(w.qf[j][c2][v]);
        }
      }
    } else if (MODE == MODE_QF) {
      for (int j = lt; j < NF * 2 * NV; j += TPE) a.qf_out[(size_t)e * NF * 2 * NV + j] = 0.0;
    }
  }
  if (MODE == MODE_QF) return;
  __syncthreads();
  // 5. common normal flux Fn = J_f F^.n at every flux point
  if (live) {
    for (int j = lt; j < NF; j += TPE) {
      const int f = j / N, m = j % N;
      const double* G = gf + j * 3;
      const double Jf = G[0], n0 = G[1], n1 = G[2];
      const int kf = a.kind[e * 4 + f];
      S Fh[NV];
      if (kf == FK_TRACE) {
        S Fc[2][NV];
        Phys<PHYS>::template conv<S, double>(pc, w.ub[j], Fc);
        S s = Phys<PHYS>::template stab<S, double>(pc, w.ub[j], n0, n1);
#pragma unroll
        for (int v = 0; v < NV; ++v) Fh[v] = n0 * Fc[0][v] + n1 * Fc[1][v] + s * (w.Uf[j][v] - w.ub[j][v]);
        if (viscous) {
          S Fv[2][NV];
          Phys<PHYS>::template visc<S, double>(pc, w.ub[j], w.qf[j], Fv);
#pragma unroll
          for (int v = 0; v < NV; ++v) Fh[v] = Fh[v] - (n0 * Fv[0][v] + n1 * Fv[1][v]);
        }
      } else {
        const int en = (int)FR_IDX(a.nbr[e * 4 + f], a.E, 21), fn = (int)FR_IDX(a.nbr_face[e * 4 + f], 4, 22);
        const size_t nix = (size_t)en * NF + fn * N + m;
        S un[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) un[v] = S(a.Uf_all[nix * NV + v]);
        S Fa[2][NV], Fb[2][NV];
        Phys<PHYS>::template conv<S, double>(pc, w.Uf[j], Fa);
        Phys<PHYS>::template conv<S, double>(pc, un, Fb);
        S lam = dmax(Phys<PHYS>::template wave<S, double>(pc, w.Uf[j], n0, n1),
                     Phys<PHYS>::template wave<S, double>(pc, un, n0, n1));
#pragma unroll
        for (int v = 0; v < NV; ++v)
          Fh[v] = 0.5 * (n0 * (Fa[0][v] + Fb[0][v]) + n1 * (Fa[1][v] + Fb[1][v])) + 0.5 * lam * (w.Uf[j][v] - un[v]);
        if (viscous) {
          S qn[2][NV];
#pragma unroll
          for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int v = 0; v < NV; ++v) qn[c][v] = S(a.qf_all[(nix * 2 + c) * NV + v]);
          S Fv[2][NV];
          if (kf == FK_FR) {
            S Fw[2][NV];
            Phys<PHYS>::template visc<S, double>(pc, w.Uf[j], w.qf[j], Fv);
            Phys<PHYS>::template visc<S, double>(pc, un, qn, Fw);
#pragma unroll
            for (int v = 0; v < NV; ++v)
              Fh[v] = Fh[v] - 0.5 * (n0 * (Fv[0][v] + Fw[0][v]) + n1 * (Fv[1][v] + Fw[1][v]));
          } else {
            if (is_imp)
              Phys<PHYS>::template visc<S, double>(pc, w.Uf[j], w.qf[j], Fv);
            else
              Phys<PHYS>::template visc<S, double>(pc, un, qn, Fv);
#pragma unroll
            for (int v = 0; v < NV; ++v) Fh[v] = Fh[v] - (n0 * Fv[0][v] + n1 * Fv[1][v]);
          }
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) w.Fn[j][v] = Jf * Fh[v];
      if (a.gview) {  // element contribution to the trace residual (zero off trace faces)
        const double wq = kf == FK_TRACE ? ref.w[m] : 0.0;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          size_t ix = ((size_t)e * NF + j) * NV + v;
          a.gview[ix] = wq * dval(w.Fn[j][v]);
          if (a.dgview) a.dgview[ix] = wq * tangent(w.Fn[j][v]);
        }
      }
    }
  }
  __syncthreads();
  // 6. divergence: R = -(1/J) [sum_r M F~_r - dgL Fn_L + dgR Fn_R]
  if (live) {
    for (int i = lt; i < NS; i += TPE) {
      const int ai = i % N, bi = i / N;
      const double iJ = gs[i * 5];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        S d = -ref.dgL[ai] * w.Fn[0 * N + bi][v] + ref.dgR[ai] * w.Fn[1 * N + bi][v] -
              ref.dgL[bi] * w.Fn[2 * N + ai][v] + ref.dgR[bi] * w.Fn[3 * N + ai][v];
#pragma unroll
        for (int c = 0; c < N; ++c) d = d + ref.M[ai][c] * w.Ft[c + N * bi][0][v] + ref.M[bi][c] * w.Ft[ai + N * c][1][v];
        S Rv = -iJ * d;
        size_t ix = (size_t)e * NS * NV + i * NV + v;
        if (a.R) a.R[ix] = dval(Rv);
        if (a.dR) a.dR[ix] = tangent(Rv);
      }
    }
  }
}

// trace residual: g[t] = gview(side 0) + gview(side 1)
__global__ void k_trace_assemble(const double* __restrict__ gview, const int* __restrict__ sides, int ntrace,
                                 int npf, double* __restrict__ g) {
  // npf = values per face = n * nv; element face stride = 4 * n * nv
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntrace * npf) return;
  const int t = i / npf, k = i % npf;
  const int e0 = sides[t * 4 + 0], f0 = sides[t * 4 + 1], e1 = sides[t * 4 + 2], f1 = sides[t * 4 + 3];
  double s = gview[((size_t)e0 * 4 + f0) * npf + k];
  if (e1 >= 0) s += gview[((size_t)e1 * 4 + f1) * npf + k];
  g[i] = s;
}

// -------------------------------------------------------------------------------------------
template <int P, int PHYS, typename S, int MODE>
static cudaError_t launch_elem(const RefOps& ref, const PhysParams& pp, const ResArgs& a, cudaStream_t st) {
  constexpr int N = P + 1, NS = N * N;
  constexpr int TPE = NS <= 32 ? 32 : 64;
  constexpr int EPB = 4;
  size_t smem = sizeof(ElemWork<P, PHYS, S>) * EPB;
  auto kern = k_element<P, PHYS, S, MODE, TPE, EPB>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int grid = (a.E + EPB - 1) / EPB;
  if (grid == 0) return cudaSuccess;
  (hfr::count_launch(), kern<<<grid, TPE * EPB, smem, st>>>(ref, pp, a));
  return cudaGetLastError();
}

template <int P, int PHYS>
static cudaError_t residual_impl(const RefOps& ref, const PhysParams& pp, ResArgs a, bool need_nbr, bool jvp,
                                 cudaStream_t st) {
  cudaError_t err;
  if (need_nbr) {
    // neighbour face states and gradients (FR and interface faces); tangents of the
    // neighbour data are not propagated (explicit states are held fixed).
    ResArgs b = a;
    b.dU = nullptr;
    b.duhat = nullptr;
    if ((err = launch_elem<P, PHYS, double, MODE_UF>(ref, pp, b, st)) != cudaSuccess) return err;
    if ((err = launch_elem<P, PHYS, double, MODE_QF>(ref, pp, b, st)) != cudaSuccess) return err;
  }
  if (jvp) return launch_elem<P, PHYS, Dual<double>, MODE_RES>(ref, pp, a, st);
  return launch_elem<P, PHYS, double, MODE_RES>(ref, pp, a, st);
}

cudaError_t launch_residual(int p, const RefOps& ref, const PhysParams& pp, const ResArgs& a, bool need_nbr, bool jvp,
                            cudaStream_t st) {
  if (pp.kind == 0) {
    switch (p) {
      case 1: return residual_impl<1, 0>(ref, pp, a, need_nbr, jvp, st);
      case 2: return residual_impl<2, 0>(ref, pp, a, need_nbr, jvp, st);
      case 3: return residual_impl<3, 0>(ref, pp, a, need_nbr, jvp, st);
    }
  } else if (pp.kind == 2) {
    switch (p) {
      case 2: return residual_impl<2, 2>(ref, pp, a, need_nbr, jvp, st);
      case 3: return residual_impl<3, 2>(ref, pp, a, need_nbr, jvp, st);
      case 4: return residual_impl<4, 2>(ref, pp, a, need_nbr, jvp, st);
    }
  } else {
    switch (p) {
      case 2: return residual_impl<2, 1>(ref, pp, a, need_nbr, jvp, st);
      case 3: return residual_impl<3, 1>(ref, pp, a, need_nbr, jvp, st);
      case 4: return residual_impl<4, 1>(ref, pp, a, need_nbr, jvp, st);
      case 5: return residual_impl<5, 1>(ref, pp, a, need_nbr, jvp, st);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_face_states(int p, const RefOps& ref, const PhysParams& pp, const ResArgs& a, cudaStream_t st) {
  if (pp.kind == 0) {
    switch (p) {
      case 1: return launch_elem<1, 0, double, MODE_UF>(ref, pp, a, st);
      case 2: return launch_elem<2, 0, double, MODE_UF>(ref, pp, a, st);
      case 3: return launch_elem<3, 0, double, MODE_UF>(ref, pp, a, st);
    }
  } else if (pp.kind == 2) {
    switch (p) {
      case 2: return launch_elem<2, 2, double, MODE_UF>(ref, pp, a, st);
      case 3: return launch_elem<3, 2, double, MODE_UF>(ref, pp, a, st);
      case 4: return launch_elem<4, 2, double, MODE_UF>(ref, pp, a, st);
    }
  } else {
    switch (p) {
      case 2: return launch_elem<2, 1, double, MODE_UF>(ref, pp, a, st);
      case 3: return launch_elem<3, 1, double, MODE_UF>(ref, pp, a, st);
      case 4: return launch_elem<4, 1, double, MODE_UF>(ref, pp, a, st);
      case 5: return launch_elem<5, 1, double, MODE_UF>(ref, pp, a, st);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_trace_assemble(const double* gview, const int* sides, int ntrace, int npf, double* g,
                                  cudaStream_t st) {
  int total = ntrace * npf;
  if (total == 0) return cudaSuccess;
  (hfr::count_launch(), k_trace_assemble<<<(total + 255) / 256, 256, 0, st>>>(gview, sides, ntrace, npf, g));
  return cudaGetLastError();
}

}  // namespace hfr

#include "hfr_checked_unit.inc"
