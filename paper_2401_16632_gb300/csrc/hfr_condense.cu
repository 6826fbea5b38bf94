// Static condensation of the hybridized Newton system (Pereira & Vermeire, arXiv 2401.16632,
// Sec. 3.2): per implicit element k,
//     X = A_k^{-1} [B_k | r_k],   S_k = D_k - C_k X_B,   t_k = s_k - C_k x_r
// (elemental L^k and t^k of eq. assembly / assembly2).
//
// X is formed by in-place Gauss-Jordan elimination with partial pivoting on [A | B | r]
// (largest |a| among the rows not yet used as pivots, lowest row on ties).  Pivoting is
// bookkeeping only: rows never move, the pivot of step c is recorded as piv[c].  Every step is
// a rank-1 update of the whole augmented block, so each thread keeps a fixed register tile of
// it for the whole elimination.  The in-place scheme leaves (PA)^{-1} where A was (P the row
// permutation), so later FP64-refinement solves are one mat-vec: A^{-1} y = (PA)^{-1} (P y).
// Same flop count as LU plus two triangular sweeps for these shapes (nA^2 (nA + nT + 1)).
//
// Outputs per element: AinvT = ((PA)^{-1})^T (column c contiguous), piv, X_B, x_r, S, t.
// T = double (plain path) or float (mixed path).
#include <algorithm>
#include <vector>

#include "hfr_internal.h"
#include "hfr_tc.cuh"

namespace hfr {

template <typename T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

// ------------------------------------------------------------------ register-tiled kernel
// 256 threads = 16 row groups x 16 column groups; thread (rg, cg) owns physical rows
// rg + 16 s and columns cg + 16 q of the nA x (nA + nT + 1) augmented block.
constexpr int GJ_RG = 16, GJ_CG = 16, GJ_THREADS = GJ_RG * GJ_CG;

template <typename T, int NA, int NT>
struct GJShape {
  static constexpr int NC = NA + NT + 1;
  static constexpr int RT = (NA + GJ_RG - 1) / GJ_RG;
  static constexpr int CT = (NC + GJ_CG - 1) / GJ_CG;
  static constexpr int R2 = (NT + GJ_RG - 1) / GJ_RG;  // S rows per thread
  static constexpr int C2 = (NT + 1 + GJ_CG - 1) / GJ_CG;
  // shared: X (NA x (NT+1)) in logical order | W: (PA)^{-1} staging (NA x NA), later C^T
  // with leading dimension NT + 1 (NA x (NT+1), conflict-free column reads)
  static constexpr int WSZ = NA * NA > NA * (NT + 1) ? NA * NA : NA * (NT + 1);
  static constexpr size_t SMEM = sizeof(T) * ((size_t)NA * (NT + 1) + (size_t)WSZ + 2 * NC + 2 * NA);
};

template <typename T, int NA, int NT>
__global__ void __launch_bounds__(GJ_THREADS) k_condense_reg(const __grid_constant__ CondArgs a) {
  using Sh = GJShape<T, NA, NT>;
  constexpr int NC = Sh::NC, RT = Sh::RT, CT = Sh::CT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sX = reinterpret_cast<T*>(smem_raw);       // NA x (NT+1), logical rows
  T* sW = sX + (size_t)NA * (NT + 1);            // WSZ
  T* pivrow = sW + (size_t)Sh::WSZ;              // 2 x NC (double buffered)
  T* colbuf = pivrow + 2 * NC;                   // 2 x NA
  __shared__ int s_piv[2];
  __shared__ int s_ipiv[NA];
  __shared__ int s_bad;
  const int k = blockIdx.x;
  const int tid = threadIdx.x;
  const int rg = tid & (GJ_RG - 1), cg = tid >> 4;
  const T* gA = reinterpret_cast<const T*>(a.A) + (size_t)k * NA * NA;
  const T* gB = reinterpret_cast<const T*>(a.B) + (size_t)k * NA * NT;
  const double* gr = a.r + (size_t)k * NA;

  // coalesced staging of [A | B | r] (row-major, ld NC) through the X / W region
  T* stage = sX;
  for (int i = tid; i < NA * NA; i += GJ_THREADS) stage[(i / NA) * NC + (i % NA)] = gA[i];
  for (int i = tid; i < NA * NT; i += GJ_THREADS) stage[(i / NT) * NC + NA + (i % NT)] = gB[i];
  for (int i = tid; i < NA; i += GJ_THREADS) stage[i * NC + NA + NT] = T(gr[i]);
  __syncthreads();
  T m[RT][CT];
#pragma unroll
  for (int s = 0; s < RT; ++s) {
    const int r = rg + GJ_RG * s;
#pragma unroll
    for (int q = 0; q < CT; ++q) {
      const int j = cg + GJ_CG * q;
      m[s][q] = (r < NA && j < NC) ? stage[r * NC + j] : T(0);
    }
  }
  unsigned used = 0u;  // bit s: own physical row rg + 16 s already a pivot
  if (tid == 0) s_bad = 0;
  // pivot search of column c by its column group (one half-warp holds the whole column):
  // records the pivot, the factors (column c) and 1 + 1/pivot, so that the update below is a
  // single FMA per entry for every row: column c becomes f - f (1 + 1/p) = -f / p.
  auto search = [&](int c) {
    const int buf = c & 1;
    T* pr = pivrow + buf * NC;
    T* cb = colbuf + buf * NA;
    const int qc = c / GJ_CG;
    T best = T(-1), val = T(0);
    int bi = 0x7fffffff;
#pragma unroll
    for (int s = 0; s < RT; ++s) {
      const int r = rg + GJ_RG * s;
      if (r < NA) {
        T v = T(0);
#pragma unroll
        for (int q = 0; q < CT; ++q)
          if (q == qc) v = m[s][q];
        cb[r] = v;
        if (!(used >> s & 1u)) {
          const T av = tabs(v);
          if (av > best || (av == best && r < bi)) { best = av; bi = r; val = v; }
        }
      }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0x0000ffffu << (tid & 16), best, o);
      const int oi = __shfl_xor_sync(0x0000ffffu << (tid & 16), bi, o);
      const T ov = __shfl_xor_sync(0x0000ffffu << (tid & 16), val, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; val = ov; }
    }
    if (bi >= NA) bi = c;  // no candidate compared (NaN column): any row, flagged singular below
    if (rg == 0) {
      s_piv[buf] = bi;
      s_ipiv[bi] = c;
      a.piv[(size_t)k * NA + c] = bi;
      if (!(best > T(0))) s_bad = 1;
      pr[c] = T(1) + (val != T(0) ? T(1) / val : T(0));
    }
  };
  if (cg == 0) search(0);
  __syncthreads();
  for (int c = 0; c < NA; ++c) {
    const int buf = c & 1;
    T* pr = pivrow + buf * NC;
    const T* cb = colbuf + buf * NA;
    const int p = s_piv[buf];
    const T inv = pr[c] - T(1);
    const int sp = p / GJ_RG;
    const bool own_p = (p & (GJ_RG - 1)) == rg;
    // owners of the pivot row publish it, normalised (column c keeps 1 + 1/pivot)
    if (own_p) {
#pragma unroll
      for (int s = 0; s < RT; ++s)
        if (s == sp) {
#pragma unroll
          for (int q = 0; q < CT; ++q) {
            const int j = cg + GJ_CG * q;
            if (j < NC && j != c) pr[j] = m[s][q] * inv;
          }
        }
      used |= 1u << sp;
    }
    __syncthreads();
    // rank-1 update of every row (one FMA per entry), then the pivot row takes the normalised row
    T pj[CT];
#pragma unroll
    for (int q = 0; q < CT; ++q) {
      const int j = cg + GJ_CG * q;
      pj[q] = j < NC ? pr[j] : T(0);
    }
#pragma unroll
    for (int s = 0; s < RT; ++s) {
      const int r = rg + GJ_RG * s;
      const T f = r < NA ? cb[r] : T(0);
#pragma unroll
      for (int q = 0; q < CT; ++q) m[s][q] -= f * pj[q];
    }
    if (own_p) {
#pragma unroll
      for (int s = 0; s < RT; ++s)
        if (s == sp) {
#pragma unroll
          for (int q = 0; q < CT; ++q) {
            const int j = cg + GJ_CG * q;
            m[s][q] = j == c ? inv : pj[q];
          }
        }
    }
    // look-ahead: the owners of column c + 1 search its pivot right away
    if (c + 1 < NA && cg == ((c + 1) & (GJ_CG - 1))) search(c + 1);
    __syncthreads();
  }
  __syncthreads();
  if (tid == 0 && s_bad) {
    atomicOr(a.status, DEV_ERR_SINGULAR);
    atomicMin(a.status + 1, k);
  }
  // stage (PA)^{-1} transposed and X in logical row order
#pragma unroll
  for (int s = 0; s < RT; ++s) {
    const int r = rg + GJ_RG * s;
    if (r >= NA) continue;
    const int lr = s_ipiv[r];
#pragma unroll
    for (int q = 0; q < CT; ++q) {
      const int j = cg + GJ_CG * q;
      if (j >= NC) continue;
      if (j < NA)
        sW[(size_t)j * NA + lr] = m[s][q];  // (PA)^{-1}[lr][j] stored at [j][lr]
      else
        sX[(size_t)lr * (NT + 1) + (j - NA)] = m[s][q];
    }
  }
  __syncthreads();
  T* gInv = reinterpret_cast<T*>(a.LU) + (size_t)k * NA * NA;
  T* gXB = reinterpret_cast<T*>(a.XB) + (size_t)k * NA * NT;
  for (int i = tid; i < NA * NA; i += GJ_THREADS) gInv[i] = sW[i];
  for (int i = tid; i < NA * (NT + 1); i += GJ_THREADS) {
    const int r = i / (NT + 1), c = i % (NT + 1);
    if (c < NT)
      gXB[(size_t)r * NT + c] = sX[i];
    else
      a.xr[(size_t)k * NA + r] = double(sX[i]);
  }
  __syncthreads();
  // S = D - C X_B and t = s - C x_r  (C staged transposed in smem: sW[l][i], ld NT + 1)
  const T* gC = reinterpret_cast<const T*>(a.C) + (size_t)k * NT * NA;
  const T* gD = reinterpret_cast<const T*>(a.D) + (size_t)k * NT * NT;
  for (int i = tid; i < NT * NA; i += GJ_THREADS) {
    const int row = i / NA, l = i % NA;
    sW[(size_t)l * (NT + 1) + row] = gC[i];
  }
  __syncthreads();
  // thread (rg, cg): output rows i = cg + 16 s, columns j = rg + 16 q (coalesced stores)
  constexpr int R2 = Sh::R2, C2 = Sh::C2;
  T acc[R2][C2];
#pragma unroll
  for (int s = 0; s < R2; ++s)
#pragma unroll
    for (int q = 0; q < C2; ++q) acc[s][q] = T(0);
  for (int l = 0; l < NA; ++l) {
    T cv[R2], xv[C2];
#pragma unroll
    for (int s = 0; s < R2; ++s) {
      const int i = cg + GJ_CG * s;
      cv[s] = i < NT ? sW[(size_t)l * (NT + 1) + i] : T(0);
    }
#pragma unroll
    for (int q = 0; q < C2; ++q) {
      const int j = rg + GJ_RG * q;
      xv[q] = j <= NT ? sX[(size_t)l * (NT + 1) + j] : T(0);
    }
#pragma unroll
    for (int s = 0; s < R2; ++s)
#pragma unroll
      for (int q = 0; q < C2; ++q) acc[s][q] += cv[s] * xv[q];
  }
  T* gS = reinterpret_cast<T*>(a.S) + (size_t)k * NT * NT;
#pragma unroll
  for (int s = 0; s < R2; ++s) {
    const int i = cg + GJ_CG * s;
    if (i >= NT) continue;
#pragma unroll
    for (int q = 0; q < C2; ++q) {
      const int j = rg + GJ_RG * q;
      if (j < NT)
        gS[(size_t)i * NT + j] = gD[(size_t)i * NT + j] - acc[s][q];
      else if (j == NT)
        a.t[(size_t)k * NT + i] = a.s[(size_t)k * NT + i] - double(acc[s][q]);
    }
  }
}

// ------------------------------------------ two-kernel FP32 path: (PA)^{-1}, then the products
// Kernel 1 inverts A in place by Gauss-Jordan with partial pivoting, keeping the matrix in
// registers with its columns cycling: every pivot step shifts each row left by one place and
// appends the column of the inverse that the step creates, so the pivot column is always the
// first register and the nA steps run as a rolled loop over one fixed-register body (small code,
// no register indexing by step).  Rows are not normalised: each step performs
//   m_{J} <- m_{J+1} - f row_{J+1},  m_last <- [pivot row] - f,  f = m_0 / pivot
// (one FMA per entry; the pivot row uses f = 0), so a row that has served as pivot stays
// multiplied by its own pivot, and one division per row at the end restores (PA)^{-1}.  The
// cycled row is spread over a lane quad (lane h holds columns QW h .. QW h + QW-1) and each lane
// holds several rows, so every pivot-row value read from shared memory feeds several FMAs; the
// shift crosses lanes by one shuffle per row.  It writes ((PA)^{-1})^T and the interchanges.
// Kernel 2 forms X = A^{-1}[B | r] = (PA)^{-1} (P[B | r]) and S = D - C X_B, t = s - C x_r as two
// dense products with 8 x 8 register tiles over operands staged in shared memory (k-major, so
// every tile row is one broadcast float4 pair).
template <int NA>
struct InvShape {
  static constexpr int QW = (NA + 3) / 4;
  static constexpr int NCP = 4 * QW;
  static constexpr int RG = (NA + 3) / 4;
  static constexpr int THREADS = ((4 * RG + 31) / 32) * 32;
  static constexpr int NWARP = THREADS / 32;
};

template <int NA>
__global__ void __launch_bounds__(InvShape<NA>::THREADS, NA <= 64 ? 8 : 3) k_inverse_q4(const __grid_constant__ CondArgs a) {
  using Sh = InvShape<NA>;
  constexpr int QW = Sh::QW, NCP = Sh::NCP, RG = Sh::RG, NWARP = Sh::NWARP;
  __shared__ __align__(16) float pr[NCP + 4];
  __shared__ float cval[NWARP];
  __shared__ int cidx[NWARP];
  __shared__ float s_pinv;
  __shared__ int s_bad;
  __shared__ int s_step[NA];
  __shared__ float s_piv[NA];
  const int k = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int g = t >> 2, h = t & 3;
  const float* gA = reinterpret_cast<const float*>(a.A) + (size_t)k * NA * NA;
  float m[4][QW];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int r = 4 * g + s;
    const bool rok = g < RG && r < NA;
#pragma unroll
    for (int j = 0; j < QW; ++j) {
      const int J = QW * h + j;
      m[s][j] = (rok && J < NA) ? __ldg(gA + (size_t)r * NA + J) : 0.f;
    }
  }
  if (t < 4) pr[NCP + t] = 0.f;
  if (t == 0) s_bad = 0;
  unsigned used = 0u;
#pragma unroll
  for (int s = 0; s < 4; ++s)
    if (g >= RG || 4 * g + s >= NA) used |= 1u << s;
  __syncthreads();
#pragma unroll 1
  for (int c = 0; c < NA; ++c) {
    float best = -1.f;
    int bi = 0x7fffffff;
    if (h == 0) {
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const float v = fabsf(m[s][0]);
        if (!(used >> s & 1u) && (v > best)) {
          best = v;
          bi = 4 * g + s;
        }
      }
    }
#pragma unroll
    for (int o = 16; o >= 4; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (NWARP > 1 && lane == 0) {
      cval[wid] = best;
      cidx[wid] = bi;
    }
    float nxt[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) nxt[s] = __shfl_down_sync(0xffffffffu, m[s][0], 1);
    float b = best;
    int p = bi;
    if (NWARP > 1) {
      __syncthreads();
      b = cval[0];
      p = cidx[0];
#pragma unroll
      for (int w2 = 1; w2 < NWARP; ++w2) {
        const float ob = cval[w2];
        const int oi = cidx[w2];
        if (ob > b || (ob == b && oi < p)) {
          b = ob;
          p = oi;
        }
      }
    } else {
      b = __shfl_sync(0xffffffffu, b, 0);
      p = __shfl_sync(0xffffffffu, p, 0);
    }
    if (p >= NA) p = c;  // no candidate compared (NaN column): any row, flagged singular below
    const int sp = p & 3;
    if (g == (p >> 2)) {
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if (s == sp) {
#pragma unroll
          for (int j = 0; j < QW; ++j) pr[QW * h + j] = m[s][j];
          if (h == 0) {
            const float pv = m[s][0];
            s_pinv = pv != 0.f ? 1.f / pv : 0.f;
            s_piv[p] = pv;
          }
        }
      }
      if (h == 0) {
        used |= 1u << sp;
        s_step[p] = c;
        a.piv[(size_t)k * NA + c] = p;
        if (!(b > 0.f)) s_bad = 1;
      }
    }
    __syncthreads();
    const float pinv = s_pinv;
    float f[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const float fs = (h == 0 && 4 * g + s != p) ? m[s][0] * pinv : 0.f;
      f[s] = __shfl_sync(0xffffffffu, fs, lane & ~3);
    }
#pragma unroll
    for (int j = 0; j < QW; ++j) {
      const float pj = pr[QW * h + j + 1];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const float old = j < QW - 1 ? m[s][j + 1] : (h < 3 ? nxt[s] : 0.f);
        m[s][j] = old - f[s] * pj;
      }
    }
    if (h == (NA - 1) / QW) {
#pragma unroll
      for (int s = 0; s < 4; ++s) m[s][(NA - 1) % QW] = (4 * g + s == p ? 1.f : 0.f) - f[s];
    }
    if (NWARP == 1) __syncwarp();
  }
  __syncthreads();
  if (t == 0 && s_bad) {
    atomicOr(a.status, DEV_ERR_SINGULAR);
    atomicMin(a.status + 1, k);
  }
  // physical row r is row s_step[r] of (PA)^{-1}, still multiplied by its pivot
  float* gInv = reinterpret_cast<float*>(a.LU) + (size_t)k * NA * NA;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int r = 4 * g + s;
    if (g < RG && r < NA) {
      const int lr = s_step[r];
      const float pv = s_piv[r];
      const float sc = pv != 0.f ? 1.f / pv : 0.f;
#pragma unroll
      for (int j = 0; j < QW; ++j) {
        const int J = QW * h + j;
        if (J < NA) gInv[(size_t)J * NA + lr] = m[s][j] * sc;  // ((PA)^{-1})^T
      }
    }
  }
}

// Kernel 1, one warp per element (nA <= 64): lane quad q (q < 8) holds rows RPT q .. RPT q + RPT-1,
// lane h of the quad columns QW h .. QW h + QW-1 of the cycled row.  The argmax, the pivot broadcast and the shift
// stay inside the warp (no CTA barrier); each pivot-row value read from shared memory feeds RPT
// FMAs.  WPB elements (warps) per CTA share nothing but the CTA.
template <int NA>
struct InvWShape {
  static constexpr int RPT = (NA + 7) / 8;  // rows per lane
  static constexpr int QW = (NA + 3) / 4;   // columns per lane
  static constexpr int NCP = 4 * QW;
  static constexpr int WPB = 2;             // elements per CTA
};

// Pivot key of a candidate: |value| with the low six mantissa bits replaced by 63 - row, so the
// unsigned maximum over the warp (one redux.sync) picks the largest magnitude, ties (within 2^-17
// relative, where the choice does not affect stability) going to the lowest row.  0 = no candidate.
__device__ __forceinline__ unsigned inv_key(float v, int row, bool ok) {
  return ok ? ((__float_as_uint(fabsf(v)) & ~63u) | (unsigned)(63 - row)) : 0u;
}

template <int NA>
__global__ void __launch_bounds__(32 * InvWShape<NA>::WPB, 5) k_inverse_warp(const __grid_constant__ CondArgs a) {
  using Sh = InvWShape<NA>;
  constexpr int RPT = Sh::RPT, QW = Sh::QW, NCP = Sh::NCP, WPB = Sh::WPB;
  static_assert(NA <= 64 && QW >= 2 && NA == 4 * QW, "one warp per element needs nA <= 64, nA % 4 == 0");
  __shared__ __align__(16) float s_pr[WPB][NCP + 4];
  __shared__ float s_pinv[WPB];
  __shared__ int s_step[WPB][NA];
  __shared__ float s_piv[WPB][NA];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k = blockIdx.x * WPB + w;
  if (k >= a.Eim) return;  // whole warps leave; no CTA barrier follows
  const int q = lane >> 2, h = lane & 3;
  float* pr = s_pr[w];
  const float* gA = reinterpret_cast<const float*>(a.A) + (size_t)k * NA * NA;
  float m[RPT][QW];
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    const int r = RPT * q + s;
#pragma unroll
    for (int j = 0; j < QW; ++j) {
      const int J = QW * h + j;
      m[s][j] = (r < NA && J < NA) ? __ldg(gA + (size_t)r * NA + J) : 0.f;
    }
  }
  // pr[NCP] = 1: lane 3's last column slot receives the new column of the inverse in the shift
  if (lane < 4) pr[NCP + lane] = lane == 0 ? 1.f : 0.f;
  unsigned used = 0u;  // bit s once row RPT q + s has been a pivot (or is padding)
#pragma unroll
  for (int s = 0; s < RPT; ++s)
    if (RPT * q + s >= NA) used |= 1u << s;
  bool bad = false;
  // search of the first pivot (column 0 is held by lane 0 of each quad)
  auto search = [&]() {
    unsigned key = 0u;
#pragma unroll
    for (int s = 0; s < RPT; ++s) key = max(key, inv_key(m[s][0], RPT * q + s, h == 0 && !(used >> s & 1u)));
    return __reduce_max_sync(0xffffffffu, key);
  };
  unsigned kp = search();
  __syncwarp();
#pragma unroll 1
  for (int c = 0; c < NA; ++c) {
    const int p = 63 - (int)(kp & 63u);
    const int gp = p / RPT, sp = p - RPT * gp;
    float nxt[RPT];
#pragma unroll
    for (int s = 0; s < RPT; ++s) nxt[s] = __shfl_down_sync(0xffffffffu, m[s][0], 1);
    if (q == gp) {
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        if (s == sp) {
#pragma unroll
          for (int j = 0; j < QW; ++j) pr[QW * h + j] = m[s][j];
          if (h == 0) {
            const float pv = m[s][0];
            s_pinv[w] = pv != 0.f ? 1.f / pv : 0.f;
            s_piv[w][p] = pv;
            s_step[w][p] = c;
          }
        }
      }
      used |= 1u << sp;  // (read by lane 0 of the quad only)
    }
    if (lane == 0) {
      a.piv[(size_t)k * NA + c] = p;
      if ((kp & ~63u) == 0u) bad = true;  // zero pivot
    }
    __syncwarp();
    const float pinv = s_pinv[w];
    float f[RPT];
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      const float fs = (h == 0 && RPT * q + s != p) ? m[s][0] * pinv : 0.f;
      f[s] = __shfl_sync(0xffffffffu, fs, lane & ~3);
    }
    // the next pivot column first, so that the next search overlaps the rest of the update
    {
      const float pj = pr[QW * h + 1];
#pragma unroll
      for (int s = 0; s < RPT; ++s) m[s][0] = m[s][1] - f[s] * pj;
    }
    const unsigned kn = search();
#pragma unroll
    for (int j = 1; j < QW; ++j) {
      const float pj = pr[QW * h + j + 1];
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        const float old = j < QW - 1 ? m[s][j + 1] : (h < 3 ? nxt[s] : (RPT * q + s == p ? 1.f : 0.f));
        m[s][j] = old - f[s] * pj;
      }
    }
    kp = kn;
    __syncwarp();
  }
  if (lane == 0 && bad) {
    atomicOr(a.status, DEV_ERR_SINGULAR);
    atomicMin(a.status + 1, k);
  }
  float* gInv = reinterpret_cast<float*>(a.LU) + (size_t)k * NA * NA;
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    const int r = RPT * q + s;
    if (r < NA) {
      const int lr = s_step[w][r];
      const float pv = s_piv[w][r];
      const float sc = pv != 0.f ? 1.f / pv : 0.f;
#pragma unroll
      for (int j = 0; j < QW; ++j) {
        const int J = QW * h + j;
        if (J < NA) gInv[(size_t)J * NA + lr] = m[s][j] * sc;  // ((PA)^{-1})^T
      }
    }
  }
}

// Kernel 1 for larger blocks (nA > 64): the same register-tiled cycling Gauss-Jordan over a few
// warps, RPT rows per lane.  Each warp reduces its candidates' pivot keys with one redux.sync and
// the warps combine them through shared memory; the next step's keys are formed as soon as the
// next pivot column is updated, so two CTA barriers per step suffice (pivot row published; keys
// of the next step published).
template <int BITS>
__device__ __forceinline__ unsigned inv_keyb(float v, int row, bool ok) {
  constexpr unsigned MASK = (1u << BITS) - 1u;
  return ok ? ((__float_as_uint(fabsf(v)) & ~MASK) | (MASK - (unsigned)row)) : 0u;
}

constexpr int INV_RPT_LARGE = 8;  // rows per lane of the multi-warp inverse

template <int NA, int RPT>
struct InvRShape {
  static constexpr int QW = (NA + 3) / 4;
  static constexpr int NCP = 4 * QW;
  static constexpr int RG = (NA + RPT - 1) / RPT;
  static constexpr int THREADS = ((4 * RG + 31) / 32) * 32;
  static constexpr int NWARP = THREADS / 32;
  static constexpr int BITS = NA <= 64 ? 6 : (NA <= 128 ? 7 : 8);
};

template <int NA, int RPT>
__global__ void __launch_bounds__(InvRShape<NA, RPT>::THREADS) k_inverse_rq(const __grid_constant__ CondArgs a) {
  using Sh = InvRShape<NA, RPT>;
  constexpr int QW = Sh::QW, NCP = Sh::NCP, NWARP = Sh::NWARP, BITS = Sh::BITS;
  constexpr unsigned MASK = (1u << BITS) - 1u;
  static_assert(NA <= 256 && QW >= 2 && NA == 4 * QW, "shape");
  __shared__ __align__(16) float pr[2][NCP + 4];
  __shared__ float s_pinv[2];
  __shared__ unsigned s_key[2][NWARP];
  __shared__ int s_step[NA];
  __shared__ float s_piv[NA];
  const int k = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int q = t >> 2, h = t & 3;
  const float* gA = reinterpret_cast<const float*>(a.A) + (size_t)k * NA * NA;
  float m[RPT][QW];
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    const int r = RPT * q + s;
#pragma unroll
    for (int j = 0; j < QW; ++j) {
      const int J = QW * h + j;
      m[s][j] = (r < NA && J < NA) ? __ldg(gA + (size_t)r * NA + J) : 0.f;
    }
  }
  // pr[NCP] = 1: the last column slot of lane 3 then receives [pivot row] - f, the new column of
  // the inverse (nA = 4 QW), inside the shift itself
  if (t < 8) pr[t >> 2][NCP + (t & 3)] = (t & 3) == 0 ? 1.f : 0.f;
  unsigned used = 0u;
#pragma unroll
  for (int s = 0; s < RPT; ++s)
    if (RPT * q + s >= NA) used |= 1u << s;
  bool bad = false;
  auto warp_key = [&]() {
    unsigned key = 0u;
#pragma unroll
    for (int s = 0; s < RPT; ++s)
      key = max(key, inv_keyb<BITS>(m[s][0], RPT * q + s, h == 0 && !(used >> s & 1u)));
    return __reduce_max_sync(0xffffffffu, key);
  };
  {
    const unsigned wk = warp_key();
    if (lane == 0) s_key[0][wid] = wk;
  }
  __syncthreads();
#pragma unroll 1
  for (int c = 0; c < NA; ++c) {
    const int buf = c & 1;
    unsigned kp = s_key[buf][0];
#pragma unroll
    for (int w2 = 1; w2 < NWARP; ++w2) kp = max(kp, s_key[buf][w2]);
    const int p = (int)(MASK - (kp & MASK));
    const int gp = p / RPT, sp = p - RPT * gp;
    float nxt[RPT];
#pragma unroll
    for (int s = 0; s < RPT; ++s) nxt[s] = __shfl_down_sync(0xffffffffu, m[s][0], 1);
    if (q == gp) {
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        if (s == sp) {
#pragma unroll
          for (int j = 0; j < QW; ++j) pr[buf][QW * h + j] = m[s][j];
          if (h == 0) {
            const float pv = m[s][0];
            s_pinv[buf] = pv != 0.f ? 1.f / pv : 0.f;
            s_piv[p] = pv;
            s_step[p] = c;
          }
        }
      }
      used |= 1u << sp;
    }
    if (t == 0) {
      a.piv[(size_t)k * NA + c] = p;
      if ((kp & ~MASK) == 0u) bad = true;  // zero pivot
    }
    __syncthreads();
    const float pinv = s_pinv[buf];
    float f[RPT];
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
      const float fs = (h == 0 && RPT * q + s != p) ? m[s][0] * pinv : 0.f;
      f[s] = __shfl_sync(0xffffffffu, fs, lane & ~3);
    }
    {
      const float pj = pr[buf][QW * h + 1];
#pragma unroll
      for (int s = 0; s < RPT; ++s) m[s][0] = m[s][1] - f[s] * pj;
    }
    {
      const unsigned wk = warp_key();
      if (lane == 0) s_key[buf ^ 1][wid] = wk;
    }
#pragma unroll
    for (int j = 1; j < QW; ++j) {
      const float pj = pr[buf][QW * h + j + 1];
#pragma unroll
      for (int s = 0; s < RPT; ++s) {
        const float old = j < QW - 1 ? m[s][j + 1] : (h < 3 ? nxt[s] : (RPT * q + s == p ? 1.f : 0.f));
        m[s][j] = old - f[s] * pj;
      }
    }
    __syncthreads();
  }
  if (t == 0 && bad) {
    atomicOr(a.status, DEV_ERR_SINGULAR);
    atomicMin(a.status + 1, k);
  }
  float* gInv = reinterpret_cast<float*>(a.LU) + (size_t)k * NA * NA;
#pragma unroll
  for (int s = 0; s < RPT; ++s) {
    const int r = RPT * q + s;
    if (r < NA) {
      const int lr = s_step[r];
      const float pv = s_piv[r];
      const float sc = pv != 0.f ? 1.f / pv : 0.f;
#pragma unroll
      for (int j = 0; j < QW; ++j) {
        const int J = QW * h + j;
        if (J < NA) gInv[(size_t)J * NA + lr] = m[s][j] * sc;  // ((PA)^{-1})^T
      }
    }
  }
}

// ------------------------------------------- block inverse on the tensor cores (tcgen05)
// Gauss-Jordan inversion with partial pivoting, in place and without row exchanges, blocked by
// panels of 16 columns.  The matrix lives in tensor memory (lane = row, one FP32 column per
// matrix column).  For a panel J the 16 elimination steps run on the panel columns only, in the
// registers of the row owners (one CTA barrier per step: each warp publishes its best pivot
// candidate and that row's panel values); the rest of the matrix then receives the panel's
// combined transformation E A = A + W P as one rank-16 MMA on the tensor cores, with
// W = E - I on the pivot rows' columns (the panel's in-place result minus the unit entries) and
// P the pivot rows' values before the panel (zero on the panel columns, which the panel itself
// produced).  3xTF32 operands, FP32 accumulation in tensor memory.  Output as the register
// inverse: piv[c] = pivot row of step c and Wt = ((PA)^{-1})^T, Wt[c][c'] = M[piv[c']][c] for the
// in-place result M.
template <int NA>
struct InvTcShape {
  static constexpr int NC = (NA + 15) / 16 * 16;  // tensor-memory columns / MMA N
  static constexpr int NP = (NA + 15) / 16;       // panels
  static constexpr int THREADS = 128;
  static constexpr int RB = NC + 8;               // row buffer stride (conflict-free transposition)
  static constexpr uint32_t SBO = 4u * 128u;      // K = 16: four 4-element chunks per 8-row group
  static constexpr uint32_t W_BYTES = 128u * 16u * 4u, P_BYTES = (uint32_t)NC * 16u * 4u;
  static constexpr uint32_t OFF_WLO = W_BYTES, OFF_PHI = 2 * W_BYTES, OFF_PLO = 2 * W_BYTES + P_BYTES;
  static constexpr uint32_t OFF_RB = 2 * W_BYTES + 2 * P_BYTES;
  static constexpr int NQ = (NC + 31) / 32;     // 32-column groups (tensor-memory loads, output)
  static constexpr uint32_t OFF_CAND = OFF_RB + 32u * RB * 4u;
  static constexpr uint32_t OFF_KEY = OFF_CAND + 2u * 4u * 16u * 4u;
  static constexpr uint32_t OFF_MBAR = OFF_KEY + 2u * 4u * 4u;
  static constexpr uint32_t NEED = OFF_MBAR + 16u;
  // requested so that at most four CTAs share an SM: each holds 128 of its 512 tensor-memory columns
  static constexpr uint32_t SMEM = NEED > 51200u ? NEED : 51200u;
  static_assert(NA <= 112 && NA % 4 == 0 && 16 * RB >= 16 * NA, "shape");
};

template <int NA>
__global__ void __launch_bounds__(128, 4) k_inverse_tc(const __grid_constant__ CondArgs a) {
  using Sh = InvTcShape<NA>;
  using namespace tc;
  constexpr int NC = Sh::NC, NP = Sh::NP, RB = Sh::RB;
  constexpr unsigned MASK = 127u;
  extern __shared__ __align__(1024) unsigned char iv_smem[];
  unsigned char* Whi = iv_smem;
  unsigned char* Wlo = iv_smem + Sh::OFF_WLO;
  unsigned char* Phi = iv_smem + Sh::OFF_PHI;
  unsigned char* Plo = iv_smem + Sh::OFF_PLO;
  float* rowbuf = reinterpret_cast<float*>(iv_smem + Sh::OFF_RB);
  float* cand = reinterpret_cast<float*>(iv_smem + Sh::OFF_CAND);  // [2][4][16]
  unsigned* s_key = reinterpret_cast<unsigned*>(iv_smem + Sh::OFF_KEY);  // [2][4]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(iv_smem + Sh::OFF_MBAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int row = t;  // tensor-memory lane of this thread
  if (t == 0) mbar_init(smem_u32(mbar), 1);
  if (w == 0) tmem_alloc(smem_u32(tslot), 128);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t tl = tmem + ((uint32_t)(32 * w) << 16);
  uint32_t phase = 0;
  bool ok = true;
  for (int k = blockIdx.x; k < a.Eim && ok; k += gridDim.x) {
    // ---- the block into tensor memory (row = lane; columns >= NA zero)
    const float* gA = reinterpret_cast<const float*>(a.A) + (size_t)k * NA * NA;
    if (t == 0 && k + (int)gridDim.x < a.Eim)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gA + (size_t)gridDim.x * NA * NA),
                   "r"((unsigned)(NA * NA * 4)) : "memory");
    // two 16-column chunks per round: eight 16-byte loads of the row in flight
#pragma unroll 1
    for (int cc = 0; cc < NP; cc += 2) {
      float v[2][16];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int u = 0; u < 16; u += 4) {
          const int c = 16 * (cc + h) + u;
          float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
          if (row < NA && c < NA) x = __ldg(reinterpret_cast<const float4*>(gA + (size_t)row * NA + c));
          v[h][u] = x.x; v[h][u + 1] = x.y; v[h][u + 2] = x.z; v[h][u + 3] = x.w;
        }
      tmem_st16(tl + (uint32_t)(16 * cc), v[0]);
      if (cc + 1 < NP) tmem_st16(tl + (uint32_t)(16 * (cc + 1)), v[1]);
    }
    tmem_st_wait();
    bool used = row >= NA;
    int mystep = -1;
    bool bad = false;
#pragma unroll 1
    for (int p = 0; p < NP; ++p) {
      const int ns = NA - 16 * p < 16 ? NA - 16 * p : 16;
      float v[16];
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
      tmem_ld16(tl + (uint32_t)(16 * p), v);
      // pivot candidates of column 0 of the panel
      {
        const unsigned key = used ? 0u : ((__float_as_uint(fabsf(v[0])) & ~MASK) | (MASK - (unsigned)row));
        const unsigned wk = __reduce_max_sync(0xffffffffu, key);
        if (key == wk && wk != 0u) {
#pragma unroll
          for (int u = 0; u < 16; u += 4)
            *reinterpret_cast<float4*>(cand + (0 * 4 + w) * 16 + u) = make_float4(v[u], v[u + 1], v[u + 2], v[u + 3]);
        }
        if (lane == 0) s_key[0 * 4 + w] = wk;
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < 16; ++s) {
        if (s < ns) {
          const int b = s & 1;
          const uint4 kq = *reinterpret_cast<const uint4*>(s_key + b * 4);
          const unsigned km = max(max(kq.x, kq.y), max(kq.z, kq.w));
          const int r = (int)(MASK - (km & MASK));
          const int wb = r >> 5;                      // the warp that holds row r
          if ((km & 0x7F800000u) == 0u) bad = true;  // |pivot| below FLT_MIN (or no pivot left)
          float prow[16];
#pragma unroll
          for (int u = 0; u < 16; u += 4) {
            const float4 x = *reinterpret_cast<const float4*>(cand + (b * 4 + wb) * 16 + u);
            prow[u] = x.x; prow[u + 1] = x.y; prow[u + 2] = x.z; prow[u + 3] = x.w;
          }
          const float pv = prow[s];
          const float pinv = pv != 0.f ? rcp_approx(pv) : 0.f;  // 1-ulp hardware reciprocal
          if (row == r) {
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = prow[u] * pinv;
            v[s] = pinv;
            used = true;
            mystep = 16 * p + s;
          } else {
            const float g = v[s] * pinv;
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] -= g * prow[u];
            v[s] = -g;
          }
          if (s + 1 < ns) {
            const unsigned key = used ? 0u : ((__float_as_uint(fabsf(v[s + 1])) & ~MASK) | (MASK - (unsigned)row));
            const unsigned wk = __reduce_max_sync(0xffffffffu, key);
            if (key == wk && wk != 0u) {
#pragma unroll
              for (int u = 0; u < 16; u += 4)
                *reinterpret_cast<float4*>(cand + ((b ^ 1) * 4 + w) * 16 + u) =
                    make_float4(v[u], v[u + 1], v[u + 2], v[u + 3]);
            }
            if (lane == 0) s_key[(b ^ 1) * 4 + w] = wk;
            __syncthreads();
          }
        }
      }
      // ---- W = E - I on the pivot columns (rows: all), 3xTF32 split, K-major 16-byte chunks
#pragma unroll
      for (int sc = 0; sc < 4; ++sc) {
        float hs[4], ls[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int s = 4 * sc + e;
          const float x = s < ns ? v[s] - (mystep == 16 * p + s ? 1.f : 0.f) : 0.f;
          split_tf32(x, hs[e], ls[e]);
        }
        *reinterpret_cast<float4*>(Whi + kmajor_offset(row, 4 * sc, Sh::SBO)) = make_float4(hs[0], hs[1], hs[2], hs[3]);
        *reinterpret_cast<float4*>(Wlo + kmajor_offset(row, 4 * sc, Sh::SBO)) = make_float4(ls[0], ls[1], ls[2], ls[3]);
      }
      // ---- P: the pivot rows before the panel (panel columns zero) into the row buffer; only
      // warps that hold one of the panel's pivot rows read tensor memory
      const bool prow_here = used && mystep >= 16 * p && mystep < 16 * p + ns;
      if (__any_sync(0xffffffffu, prow_here)) {
        for (int cq = 0; cq < Sh::NQ; ++cq) {
          float x[32];
          tmem_ld32(tl + (uint32_t)(32 * cq), x);
          if (prow_here) {
            float* dst = rowbuf + (mystep - 16 * p) * RB + 32 * cq;
#pragma unroll
            for (int u = 0; u < 32; u += 4) {
              const int c = 32 * cq + u;
              if (c < NC)
                *reinterpret_cast<float4*>(dst + u) = (c >= 16 * p && c < 16 * p + 16)
                                                          ? make_float4(0.f, 0.f, 0.f, 0.f)
                                                          : make_float4(x[u], x[u + 1], x[u + 2], x[u + 3]);
            }
          }
        }
      }
      if (ns < 16)
        for (int e = t; e < (16 - ns) * NC; e += Sh::THREADS) rowbuf[(ns + e / NC) * RB + e % NC] = 0.f;
      // the panel's in-place result replaces its columns (the MMA adds zero there)
      tmem_st16(tl + (uint32_t)(16 * p), v);
      tmem_st_wait();
      __syncthreads();
      // ---- row buffer -> P operand (rows = matrix columns j, K = pivot index), 3xTF32 split
      for (int e = t; e < NC * 4; e += Sh::THREADS) {
        const int j = e % NC, sc = e / NC;  // lanes along j: conflict-free reads, 16-byte stores
        float hs[4], ls[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) split_tf32(rowbuf[(4 * sc + q) * RB + j], hs[q], ls[q]);
        *reinterpret_cast<float4*>(Phi + kmajor_offset(j, 4 * sc, Sh::SBO)) = make_float4(hs[0], hs[1], hs[2], hs[3]);
        *reinterpret_cast<float4*>(Plo + kmajor_offset(j, 4 * sc, Sh::SBO)) = make_float4(ls[0], ls[1], ls[2], ls[3]);
      }
      fence_proxy_async();
      fence_before_sync();
      __syncthreads();
      if (t == 0) {
        fence_after_sync();
        constexpr uint32_t idesc = idesc_tf32(128, NC);
        const uint32_t wh = smem_u32(Whi), wl = smem_u32(Wlo), ph = smem_u32(Phi), pl = smem_u32(Plo);
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const uint32_t off = (uint32_t)kk * 256u;
          mma_tf32(tmem, desc_noswizzle(wh + off, 128, Sh::SBO), desc_noswizzle(ph + off, 128, Sh::SBO), idesc, 1);
          if (a.tc_mode != 3) {  // 3xTF32; mode 3 keeps the single TF32 pass
            mma_tf32(tmem, desc_noswizzle(wh + off, 128, Sh::SBO), desc_noswizzle(pl + off, 128, Sh::SBO), idesc, 1);
            mma_tf32(tmem, desc_noswizzle(wl + off, 128, Sh::SBO), desc_noswizzle(ph + off, 128, Sh::SBO), idesc, 1);
          }
        }
        mma_commit(smem_u32(mbar));
      }
      ok = mbar_wait(smem_u32(mbar), phase, tc::TIMEOUT_NS);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        ok = false;
        break;
      }
      fence_after_sync();
    }
    if (!ok) break;
    if (__syncthreads_or(bad) && t == 0) {
      atomicOr(a.status, DEV_ERR_SINGULAR);
      atomicMin(a.status + 1, k);
    }
    // pivot row of each step, written once by its owner
    if (row < NA && mystep >= 0) a.piv[(size_t)k * NA + mystep] = row;
    // ---- output: Wt[c][c'] = M[piv[c']][c], through the row buffer 32 columns at a time
    float* gWt = reinterpret_cast<float*>(a.LU) + (size_t)k * NA * NA;
#pragma unroll 1
    for (int cq = 0; cq < Sh::NQ; ++cq) {
      float x[32];
      tmem_ld32(tl + (uint32_t)(32 * cq), x);
      if (row < NA && mystep >= 0)
#pragma unroll
        for (int u = 0; u < 32; ++u)
          if (32 * cq + u < NA) rowbuf[u * RB + mystep] = x[u];
      __syncthreads();
      const int nrow = NA - 32 * cq < 32 ? NA - 32 * cq : 32;
      for (int e = t; e < nrow * (NA / 4); e += Sh::THREADS) {
        const int u = e / (NA / 4), i4 = e % (NA / 4);
        *reinterpret_cast<float4*>(gWt + (size_t)(32 * cq + u) * NA + 4 * i4) =
            *reinterpret_cast<const float4*>(rowbuf + u * RB + 4 * i4);
      }
      __syncthreads();
    }
  }
  if (!ok) {
    if (t == 0) atomicOr(a.status, DEV_ERR_TIMEOUT);
    mbar_wait(smem_u32(mbar), phase ^ 1u, tc::TIMEOUT_NS);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (w == 0) tmem_dealloc(tmem, 128);
}

template <int NA>
static cudaError_t launch_inverse_tc(const CondArgs& a, cudaStream_t st) {
  using Sh = InvTcShape<NA>;
  static int grid = 0, nsm = 0;
  if (grid == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_inverse_tc<NA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_inverse_tc<NA>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    // resident CTAs per SM from the shared-memory arithmetic (at most four: tensor memory)
    int dev = 0, smem_sm = 0, resv = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess) return e;
    int fit = smem_sm / (int)(Sh::SMEM + (uint32_t)resv);
    grid = nsm * (fit < 1 ? 1 : (fit > 4 ? 4 : fit));
  }
  int gr = grid;
  if (a.inv_ctas > 0 && a.inv_ctas * nsm < grid) gr = a.inv_ctas * nsm;
  const int g = a.Eim < gr ? a.Eim : gr;
  (hfr::count_launch(), k_inverse_tc<NA><<<g, Sh::THREADS, Sh::SMEM, st>>>(a));
  return cudaGetLastError();
}

template <int NA, int NT>
struct ProdShape {
  static constexpr int TI = (NA + 7) / 8;  // row tiles of X
  static constexpr int TJ = NT / 8;        // column tiles of X_B and S
  static constexpr int NAP = 8 * TI;
  static constexpr int LDW = (NAP > NT ? NAP : NT) + 4;  // ((PA)^{-1})^T rows, then C^T rows
  static constexpr int LDB = NT + 4;       // P[B | r] rows, then X rows (NT + 1 used)
  static constexpr int NTILE = TI * TJ > TJ * TJ ? TI * TJ : TJ * TJ;
  static constexpr int THREADS = ((NTILE + 31) / 32) * 32 < 64 ? 64 : ((NTILE + 31) / 32) * 32;
  static constexpr int WROWS = NA;         // k extent of both products
  static constexpr size_t SMEM = sizeof(float) * ((size_t)WROWS * LDW + (size_t)NAP * LDB);
  static_assert(NT % 8 == 0, "nT must be a multiple of 8");
};

template <int NA, int NT>
__global__ void __launch_bounds__(ProdShape<NA, NT>::THREADS) k_condense_products(const __grid_constant__ CondArgs a) {
  using Sh = ProdShape<NA, NT>;
  constexpr int TI = Sh::TI, TJ = Sh::TJ, LDW = Sh::LDW, LDB = Sh::LDB, THREADS = Sh::THREADS;
  extern __shared__ __align__(16) float sm[];
  float* W = sm;                    // NA x LDW: k-major left operand
  float* Bs = sm + (size_t)NA * LDW;  // NAP x LDB: k-major right operand
  const int k = blockIdx.x, t = threadIdx.x;
  const float* gWt = reinterpret_cast<const float*>(a.LU) + (size_t)k * NA * NA;
  const float* gB = reinterpret_cast<const float*>(a.B) + (size_t)k * NA * NT;
  const int* piv = a.piv + (size_t)k * NA;
  // W[c][i] = (PA)^{-1}[i][c] (stored transposed), Bs[c][:] = [B | r][piv[c]][:]; the pivots
  // first (the B rows they select are the only dependent loads), every copy float4-wide and
  // unrolled so that all of a thread's loads are in flight together
  __shared__ int s_pv[NA];
  for (int c = t; c < NA; c += THREADS) s_pv[c] = __ldg(piv + c);
  static_assert(NA % 4 == 0 || NA * NA % 4 == 0, "W copy");
  constexpr int W4 = NA * NA / 4;  // float4 of ((PA)^{-1})^T
  constexpr int B4 = NA * NT / 4;
  constexpr int C4 = NT * NA / 4;
#pragma unroll
  for (int u = 0; u < (W4 + THREADS - 1) / THREADS; ++u) {
    const int e4 = t + THREADS * u;
    if (e4 < W4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(gWt) + e4);
      const int e = 4 * e4;
      const int c = e / NA, i = e % NA;  // NA % 4 == 0: the four values share a row
      *reinterpret_cast<float4*>(W + c * LDW + i) = v;
    }
  }
  for (int e = t; e < NA * (LDW - NA); e += THREADS) {
    const int c = e / (LDW - NA), i = NA + e % (LDW - NA);
    W[c * LDW + i] = 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < (B4 + THREADS - 1) / THREADS; ++u) {
    const int e4 = t + THREADS * u;
    if (e4 < B4) {
      const int c = (4 * e4) / NT, j = (4 * e4) % NT;
      const float4 v = __ldg(reinterpret_cast<const float4*>(gB + (size_t)s_pv[c] * NT + j));
      *reinterpret_cast<float4*>(Bs + c * LDB + j) = v;
    }
  }
  for (int c = t; c < NA; c += THREADS) Bs[c * LDB + NT] = float(a.r[(size_t)k * NA + s_pv[c]]);
  // C and D are pulled into L2 while the first product runs
  const float* gC = reinterpret_cast<const float*>(a.C) + (size_t)k * NT * NA;
  const float* gD = reinterpret_cast<const float*>(a.D) + (size_t)k * NT * NT;
  for (int off = 32 * t; off < NT * NA; off += 32 * THREADS)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(gC + off));
  for (int off = 32 * t; off < NT * NT; off += 32 * THREADS)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(gD + off));
  __syncthreads();
  // X = W^T Bs: thread tile rows 8 ti .. 8 ti + 7, columns 8 tj .. 8 tj + 7 of X_B
  float acc[8][8];
  const bool t1 = t < TI * TJ;
  const int ti = t1 ? t / TJ : 0, tj = t1 ? t % TJ : 0;
  if (t1) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
#pragma unroll 2
    for (int c = 0; c < NA; ++c) {
      const float4 w0 = *reinterpret_cast<const float4*>(W + c * LDW + 8 * ti);
      const float4 w1 = *reinterpret_cast<const float4*>(W + c * LDW + 8 * ti + 4);
      const float4 b0 = *reinterpret_cast<const float4*>(Bs + c * LDB + 4 * tj);
      const float4 b1 = *reinterpret_cast<const float4*>(Bs + c * LDB + NT / 2 + 4 * tj);
      const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] += wv[u] * bv[v];
    }
  }
  // x_r = W^T (P r): one row per thread
  float xrv = 0.f;
  if (t < NA) {
#pragma unroll 8
    for (int c = 0; c < NA; ++c) xrv += W[c * LDW + t] * Bs[c * LDB + NT];
  }
  __syncthreads();
  // X_B and x_r out, X into Bs (rows = k of the second product), C^T into W
  float* gXB = reinterpret_cast<float*>(a.XB) + (size_t)k * NA * NT;
  if (t1) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = 8 * ti + u;
      if (i < NA) {
        const float4 x0 = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
        const float4 x1 = make_float4(acc[u][4], acc[u][5], acc[u][6], acc[u][7]);
        *reinterpret_cast<float4*>(gXB + (size_t)i * NT + 4 * tj) = x0;
        *reinterpret_cast<float4*>(gXB + (size_t)i * NT + NT / 2 + 4 * tj) = x1;
        *reinterpret_cast<float4*>(Bs + i * LDB + 4 * tj) = x0;
        *reinterpret_cast<float4*>(Bs + i * LDB + NT / 2 + 4 * tj) = x1;
      }
    }
  }
  if (t < NA) {
    a.xr[(size_t)k * NA + t] = double(xrv);
    Bs[t * LDB + NT] = xrv;
  }
#pragma unroll
  for (int u = 0; u < (C4 + THREADS - 1) / THREADS; ++u) {
    const int e4 = t + THREADS * u;
    if (e4 < C4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(gC) + e4);
      const int i = (4 * e4) / NA, l = (4 * e4) % NA;  // C row i, columns l .. l+3
      W[l * LDW + i] = v.x;
      W[(l + 1) * LDW + i] = v.y;
      W[(l + 2) * LDW + i] = v.z;
      W[(l + 3) * LDW + i] = v.w;
    }
  }
  __syncthreads();
  // S = D - C X_B (tiles over nT x nT), t = s - C x_r
  if (t < TJ * TJ) {
    const int si = t / TJ, sj = t % TJ;
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
#pragma unroll 2
    for (int l = 0; l < NA; ++l) {
      const float4 c0 = *reinterpret_cast<const float4*>(W + l * LDW + 8 * si);
      const float4 c1 = *reinterpret_cast<const float4*>(W + l * LDW + 8 * si + 4);
      const float4 x0 = *reinterpret_cast<const float4*>(Bs + l * LDB + 4 * sj);
      const float4 x1 = *reinterpret_cast<const float4*>(Bs + l * LDB + NT / 2 + 4 * sj);
      const float cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
      const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] += cv[u] * xv[v];
    }
    float* gS = reinterpret_cast<float*>(a.S) + (size_t)k * NT * NT;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const size_t o0 = (size_t)(8 * si + u) * NT + 4 * sj, o1 = o0 + NT / 2;
      const float4 d0 = __ldg(reinterpret_cast<const float4*>(gD + o0));
      const float4 d1 = __ldg(reinterpret_cast<const float4*>(gD + o1));
      *reinterpret_cast<float4*>(gS + o0) =
          make_float4(d0.x - acc[u][0], d0.y - acc[u][1], d0.z - acc[u][2], d0.w - acc[u][3]);
      *reinterpret_cast<float4*>(gS + o1) =
          make_float4(d1.x - acc[u][4], d1.y - acc[u][5], d1.z - acc[u][6], d1.w - acc[u][7]);
    }
  }
  for (int i = t; i < NT; i += THREADS) {
    float v = 0.f;
#pragma unroll 8
    for (int l = 0; l < NA; ++l) v += W[l * LDW + i] * Bs[l * LDB + NT];
    a.t[(size_t)k * NT + i] = a.s[(size_t)k * NT + i] - double(v);
  }
}

// ---------------------------------------- products in two streaming kernels (larger blocks)
// For nA > 64 the single products kernel needs both whole operands in shared memory (two CTAs per
// SM).  Here each product streams its k dimension through shared memory in chunks of KC rows
// with cp.async double buffering, so a CTA holds two small chunks and the next chunk's copy
// overlaps the current chunk's FMAs:
//   k_products_x:  X_B = (PA)^{-1} P B and x_r = (PA)^{-1} P r (4 x 8 register tiles, the tiles
//                  of column block 0 also carry x_r), written to global memory;
//   k_products_s:  S = D - C X_B and t = s - C x_r, C staged row-major with an odd row stride
//                  (4-byte copies, conflict-free column reads), X_B rows with 16-byte copies.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int NA, int NT>
struct StreamShape {
  static constexpr int KC = NA % 20 == 0 ? 20 : (NA % 16 == 0 ? 16 : (NA % 12 == 0 ? 12 : 4));
  static constexpr int NCH = NA / KC;
  static constexpr int TIX = NA / 4, TJ = NT / 8;  // X_B tiles
  static constexpr int TIS = NT / 4;               // S tiles
  static constexpr int TX = ((TIX * TJ + 31) / 32) * 32;
  static constexpr int TSS = ((TIS * TJ + 31) / 32) * 32;
  static constexpr int LDW = NA + 4, LDB = NT + 4;  // k-major chunk rows (16-byte aligned)
  static constexpr int LDC = KC + 1;               // C chunk rows (odd: conflict-free columns)
  static_assert(NA % 4 == 0 && NT % 8 == 0 && NA % KC == 0, "shape");
  // a thread's eight columns are 4 tj .. 4 tj + 3 and nT/2 + 4 tj .. nT/2 + 4 tj + 3: the eight
  // lanes of a float4 phase then read 128 contiguous bytes (no bank conflict)
};

template <int NA, int NT>
__global__ void __launch_bounds__(StreamShape<NA, NT>::TX) k_products_x(const __grid_constant__ CondArgs a) {
  using Sh = StreamShape<NA, NT>;
  constexpr int KC = Sh::KC, NCH = Sh::NCH, TJ = Sh::TJ, LDW = Sh::LDW, LDB = Sh::LDB, TH = Sh::TX;
  __shared__ __align__(16) float Wc[2][KC * LDW];
  __shared__ __align__(16) float Bc[2][KC * LDB];
  __shared__ float rc[2][KC];
  __shared__ int s_pv[NA];
  const int k = blockIdx.x, t = threadIdx.x;
  const float* gWt = reinterpret_cast<const float*>(a.LU) + (size_t)k * NA * NA;
  const float* gB = reinterpret_cast<const float*>(a.B) + (size_t)k * NA * NT;
  const double* gr = a.r + (size_t)k * NA;
  for (int c = t; c < NA; c += TH) s_pv[c] = a.piv[(size_t)k * NA + c];
  __syncthreads();
  auto stage = [&](int ch, int buf) {
    const int c0 = ch * KC;
    for (int e = t; e < KC * (NA / 4); e += TH) {
      const int rr = e / (NA / 4), q4 = e % (NA / 4);
      cp_async16(&Wc[buf][rr * LDW + 4 * q4], gWt + (size_t)(c0 + rr) * NA + 4 * q4);
    }
    for (int e = t; e < KC * (NT / 4); e += TH) {
      const int rr = e / (NT / 4), q4 = e % (NT / 4);
      cp_async16(&Bc[buf][rr * LDB + 4 * q4], gB + (size_t)s_pv[c0 + rr] * NT + 4 * q4);
    }
    cp_async_commit();
    for (int rr = t; rr < KC; rr += TH) rc[buf][rr] = float(gr[s_pv[c0 + rr]]);
  };
  const bool act = t < Sh::TIX * TJ;
  const int ti = act ? t / TJ : 0, tj = act ? t % TJ : 0;
  float acc[4][8], accr[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    accr[u] = 0.f;
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
  }
  stage(0, 0);
  for (int ch = 0; ch < NCH; ++ch) {
    const int buf = ch & 1;
    if (ch + 1 < NCH) {
      stage(ch + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    if (act) {
      const float* W = Wc[buf];
      const float* Bm = Bc[buf];
#pragma unroll 4
      for (int c = 0; c < KC; ++c) {
        const float4 w0 = *reinterpret_cast<const float4*>(W + c * LDW + 4 * ti);
        const float4 b0 = *reinterpret_cast<const float4*>(Bm + c * LDB + 4 * tj);
        const float4 b1 = *reinterpret_cast<const float4*>(Bm + c * LDB + NT / 2 + 4 * tj);
        const float wv[4] = {w0.x, w0.y, w0.z, w0.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 8; ++v) acc[u][v] += wv[u] * bv[v];
        if (tj == 0) {
          const float rv = rc[buf][c];
#pragma unroll
          for (int u = 0; u < 4; ++u) accr[u] += wv[u] * rv;
        }
      }
    }
    __syncthreads();
  }
  if (!act) return;
  float* gXB = reinterpret_cast<float*>(a.XB) + (size_t)k * NA * NT;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = 4 * ti + u;
    *reinterpret_cast<float4*>(gXB + (size_t)i * NT + 4 * tj) = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
    *reinterpret_cast<float4*>(gXB + (size_t)i * NT + NT / 2 + 4 * tj) =
        make_float4(acc[u][4], acc[u][5], acc[u][6], acc[u][7]);
    if (tj == 0) a.xr[(size_t)k * NA + i] = double(accr[u]);
  }
}

template <int NA, int NT>
__global__ void __launch_bounds__(StreamShape<NA, NT>::TSS) k_products_s(const __grid_constant__ CondArgs a) {
  using Sh = StreamShape<NA, NT>;
  constexpr int KC = Sh::KC, NCH = Sh::NCH, TJ = Sh::TJ, LDB = Sh::LDB, LDC = Sh::LDC, TH = Sh::TSS;
  __shared__ __align__(16) float Cc[2][NT * LDC];
  __shared__ __align__(16) float Xc[2][KC * LDB];
  __shared__ float xc[2][KC];
  const int k = blockIdx.x, t = threadIdx.x;
  const float* gC = reinterpret_cast<const float*>(a.C) + (size_t)k * NT * NA;
  const float* gX = reinterpret_cast<const float*>(a.XB) + (size_t)k * NA * NT;
  const double* gxr = a.xr + (size_t)k * NA;
  const float* gD = reinterpret_cast<const float*>(a.D) + (size_t)k * NT * NT;
  for (int off = 32 * t; off < NT * NT; off += 32 * TH) asm volatile("prefetch.global.L2 [%0];" ::"l"(gD + off));
  auto stage = [&](int ch, int buf) {
    const int l0 = ch * KC;
    for (int e = t; e < NT * KC; e += TH) {
      const int i = e / KC, l = e % KC;
      cp_async4(&Cc[buf][i * LDC + l], gC + (size_t)i * NA + l0 + l);
    }
    for (int e = t; e < KC * (NT / 4); e += TH) {
      const int rr = e / (NT / 4), q4 = e % (NT / 4);
      cp_async16(&Xc[buf][rr * LDB + 4 * q4], gX + (size_t)(l0 + rr) * NT + 4 * q4);
    }
    cp_async_commit();
    for (int rr = t; rr < KC; rr += TH) xc[buf][rr] = float(gxr[l0 + rr]);
  };
  const bool act = t < Sh::TIS * TJ;
  const int si = act ? t / TJ : 0, sj = act ? t % TJ : 0;
  float acc[4][8], acct[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    acct[u] = 0.f;
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
  }
  stage(0, 0);
  for (int ch = 0; ch < NCH; ++ch) {
    const int buf = ch & 1;
    if (ch + 1 < NCH) {
      stage(ch + 1, buf ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    if (act) {
      const float* Cm = Cc[buf];
      const float* Xm = Xc[buf];
#pragma unroll 4
      for (int l = 0; l < KC; ++l) {
        float cv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cv[u] = Cm[(4 * si + u) * LDC + l];
        const float4 x0 = *reinterpret_cast<const float4*>(Xm + l * LDB + 4 * sj);
        const float4 x1 = *reinterpret_cast<const float4*>(Xm + l * LDB + NT / 2 + 4 * sj);
        const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 8; ++v) acc[u][v] += cv[u] * xv[v];
        if (sj == 0) {
          const float xrv = xc[buf][l];
#pragma unroll
          for (int u = 0; u < 4; ++u) acct[u] += cv[u] * xrv;
        }
      }
    }
    __syncthreads();
  }
  if (!act) return;
  float* gS = reinterpret_cast<float*>(a.S) + (size_t)k * NT * NT;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = 4 * si + u;
    const size_t o0 = (size_t)i * NT + 4 * sj, o1 = o0 + NT / 2;
    const float4 d0 = __ldg(reinterpret_cast<const float4*>(gD + o0));
    const float4 d1 = __ldg(reinterpret_cast<const float4*>(gD + o1));
    *reinterpret_cast<float4*>(gS + o0) =
        make_float4(d0.x - acc[u][0], d0.y - acc[u][1], d0.z - acc[u][2], d0.w - acc[u][3]);
    *reinterpret_cast<float4*>(gS + o1) =
        make_float4(d1.x - acc[u][4], d1.y - acc[u][5], d1.z - acc[u][6], d1.w - acc[u][7]);
    if (sj == 0) a.t[(size_t)k * NT + i] = a.s[(size_t)k * NT + i] - double(acct[u]);
  }
}

// ------------------------------------------------ products on the tensor cores (tcgen05)
// Both products of the condensation as two transposed GEMMs per element on the fifth-generation
// tensor cores, in 3xTF32 (each FP32 operand split into a TF32 high part and the TF32 remainder;
// hi*hi + hi*lo + lo*hi accumulated in FP32 in tensor memory, about 2^-21 relative per product):
//   GEMM 1:  [X_B | x_r]^T (M = nT + 1 rows, padded to 128)  =  [P B | P r]^T  *  ((PA)^{-1})^T
//   GEMM 2:  [C X_B | C x_r]^T                               =  [X_B | x_r]^T  *  C^T
// then S = D - C X_B and t = s - C x_r.  Transposing puts the trace index j on the tensor-memory
// lanes, so that each thread of the epilogues owns one j: X_B[i][j], S[i][j] and D[i][j] are
// read and written with the 32 lanes of a warp on 32 consecutive j (coalesced), and the thread's
// run of consecutive i is one 16-byte chunk of GEMM 2's K-major A operand (conflict-free).
// Operands are staged K-major without swizzle (see hfr_tc.cuh); the staging maps the 32 lanes of
// a warp to 8 rows x 4 k, which the layout spreads over all 32 banks.  One CTA of 256 threads per
// element in a persistent loop; thread 0 issues the MMAs; the next element's blocks are prefetched
// into L2 while the current one is processed.
template <int NA, int NT>
struct TcShape {
  static constexpr int K1 = (NA + 7) / 8 * 8;     // GEMM K (both GEMMs), padded with zeros
  static constexpr int N1 = (NA + 15) / 16 * 16;  // GEMM 1 N (the i index of X_B)
  static constexpr int N2 = (NT + 15) / 16 * 16;  // GEMM 2 N (the i index of S)
  static constexpr int M = 128;
  static constexpr int NB = N1 > N2 ? N1 : N2;
  static constexpr int KG = K1 / 4;               // 4-element k chunks
  // 8-row groups padded by 16 bytes: with SBO = 16 (mod 128) the 4-byte stores of a float4 read
  // along the rows (lanes = 4 k x 8 row quads) fall in 32 distinct banks
  static constexpr uint32_t SBO = (uint32_t)KG * 128u + 16u;
  static constexpr uint32_t A_BYTES = (uint32_t)(M / 8) * SBO;   // one of hi / lo
  static constexpr uint32_t B_BYTES = (uint32_t)(NB / 8) * SBO;
  static constexpr uint32_t SMEM = 2u * A_BYTES + 2u * B_BYTES + 16u + 128u + 2u * NA * 4u + 1024u;
  // 8 warps: warps 0-6 stage operands, warp 7 (lanes 96-127 of tensor memory, rows the epilogues
  // do not need while nT < 96) allocates tensor memory and issues the MMAs
  static constexpr int THREADS = 256, WARPS = 7, ISSUER = 7;
  // GEMM 1 staging: slots of one float4 (four consecutive rows of one k), enumerated k mod 4
  // fastest, then the row quad, then k / 4
  static constexpr int AQ = NT / 4, BQ = NA / 4;  // row quads of the A and B operands
  static constexpr int A_SLOTS = AQ * K1, B_SLOTS = BQ * K1;
  static constexpr int A_PER = (A_SLOTS + WARPS * 32 - 1) / (WARPS * 32);
  static constexpr int B_PER = (B_SLOTS + WARPS * 32 - 1) / (WARPS * 32);
  static constexpr int R_PER = (K1 + THREADS - 1) / THREADS;
  // C staging: warp task = 8 rows x 4 chunks of 4 k (one float4 per lane)
  static constexpr int CG = (KG + 3) / 4;
  static constexpr int C_TASKS = (NT / 8) * CG, C_PER = (C_TASKS + WARPS - 1) / WARPS;
  static constexpr int NCH1 = N1 / 16, H1 = (NCH1 + 1) / 2;  // epilogue column chunks, split in halves
  static constexpr int NCH2 = N2 / 16, H2 = (NCH2 + 1) / 2;
  static constexpr uint32_t TMEM_COLS = 256, D2_COL = 128;
  static_assert(NT < 96 && N1 <= 128 && N2 <= 128, "trace block too large for one 128-row tile");
  static_assert(NA % 4 == 0 && NT % 8 == 0, "shape");
  static_assert(SMEM <= 232448, "shared memory");
};

// slot -> (k, first row) of the float4 staging of a GEMM 1 operand with NQ row quads
template <int NQ>
__device__ __forceinline__ void tc_slot(int slot, int& c, int& r0) {
  const int c_lo = slot & 3, rest = slot >> 2;
  r0 = 4 * (rest % NQ);
  c = 4 * (rest / NQ) + c_lo;
}

// GEMM 1 operands of one element held in registers between their load and their store
template <int NA, int NT>
struct TcStage {
  float4 av[TcShape<NA, NT>::A_PER];
  float4 bv[TcShape<NA, NT>::B_PER];
  float rv[TcShape<NA, NT>::R_PER];
};

// all loads first (one memory latency per element), 16 bytes per lane along the contiguous
// dimension, pivots from shared memory
template <int NA, int NT>
__device__ __forceinline__ void tc_load_stage(TcStage<NA, NT>& g, const CondArgs& a, int k, const int* pv, int t) {
  using Sh = TcShape<NA, NT>;
  const float* gWt = reinterpret_cast<const float*>(a.LU) + (size_t)k * NA * NA;
  const float* gB = reinterpret_cast<const float*>(a.B) + (size_t)k * NA * NT;
  const double* gr = a.r + (size_t)k * NA;
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int u = 0; u < Sh::A_PER; ++u) {
    const int slot = t + Sh::WARPS * 32 * u;
    int c, j0;
    tc_slot<Sh::AQ>(slot, c, j0);
    g.av[u] = (slot < Sh::A_SLOTS && c < NA) ? __ldg(reinterpret_cast<const float4*>(gB + (size_t)pv[c] * NT + j0)) : z;
  }
#pragma unroll
  for (int u = 0; u < Sh::B_PER; ++u) {
    const int slot = t + Sh::WARPS * 32 * u;
    int c, i0;
    tc_slot<Sh::BQ>(slot, c, i0);
    g.bv[u] = (slot < Sh::B_SLOTS && c < NA) ? __ldg(reinterpret_cast<const float4*>(gWt + (size_t)c * NA + i0)) : z;
  }
#pragma unroll
  for (int u = 0; u < Sh::R_PER; ++u) {
    const int c = t + Sh::THREADS * u;
    g.rv[u] = c < NA ? float(gr[pv[c]]) : 0.f;
  }
}

// A: row jj < NT is column jj of P B, row NT is P r; B: row i is row i of (PA)^{-1} (column i of
// Wt); K padding zero.  Four 4-byte stores per float4, conflict-free with the padded row groups.
template <int NA, int NT>
__device__ __forceinline__ void tc_store_stage(const TcStage<NA, NT>& g, unsigned char* Ahi, unsigned char* Alo,
                                               unsigned char* Bhi, unsigned char* Blo, int t) {
  using Sh = TcShape<NA, NT>;
  using namespace tc;
#pragma unroll
  for (int u = 0; u < Sh::A_PER; ++u) {
    const int slot = t + Sh::WARPS * 32 * u;
    if (slot < Sh::A_SLOTS) {
      int c, j0;
      tc_slot<Sh::AQ>(slot, c, j0);
      const float x[4] = {g.av[u].x, g.av[u].y, g.av[u].z, g.av[u].w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float h, l;
        split_tf32(x[e], h, l);
        *reinterpret_cast<float*>(Ahi + kmajor_offset(j0 + e, c, Sh::SBO)) = h;
        *reinterpret_cast<float*>(Alo + kmajor_offset(j0 + e, c, Sh::SBO)) = l;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < Sh::B_PER; ++u) {
    const int slot = t + Sh::WARPS * 32 * u;
    if (slot < Sh::B_SLOTS) {
      int c, i0;
      tc_slot<Sh::BQ>(slot, c, i0);
      const float x[4] = {g.bv[u].x, g.bv[u].y, g.bv[u].z, g.bv[u].w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float h, l;
        split_tf32(x[e], h, l);
        *reinterpret_cast<float*>(Bhi + kmajor_offset(i0 + e, c, Sh::SBO)) = h;
        *reinterpret_cast<float*>(Blo + kmajor_offset(i0 + e, c, Sh::SBO)) = l;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < Sh::R_PER; ++u) {
    const int c = t + Sh::THREADS * u;
    if (c < Sh::K1) {
      float h, l;
      split_tf32(g.rv[u], h, l);
      *reinterpret_cast<float*>(Ahi + kmajor_offset(NT, c, Sh::SBO)) = h;
      *reinterpret_cast<float*>(Alo + kmajor_offset(NT, c, Sh::SBO)) = l;
    }
  }
}

template <int NA, int NT>
__device__ __forceinline__ void tc_issue(uint32_t td, unsigned char* Ahi, unsigned char* Alo, unsigned char* Bhi,
                                         unsigned char* Blo, uint32_t idesc, uint32_t mbar, bool three) {
  using Sh = TcShape<NA, NT>;
  using namespace tc;
  fence_after_sync();
  const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll 1
  for (int kk = 0; kk < Sh::K1 / 8; ++kk) {
    const uint32_t off = (uint32_t)kk * 256u;  // two core matrices along k per instruction
    mma_tf32(td, desc_noswizzle(ah + off, 128, Sh::SBO), desc_noswizzle(bh + off, 128, Sh::SBO), idesc, kk > 0);
    if (three) {  // 3xTF32 (single TF32 pass otherwise)
      mma_tf32(td, desc_noswizzle(ah + off, 128, Sh::SBO), desc_noswizzle(bl + off, 128, Sh::SBO), idesc, 1);
      mma_tf32(td, desc_noswizzle(al + off, 128, Sh::SBO), desc_noswizzle(bh + off, 128, Sh::SBO), idesc, 1);
    }
  }
  mma_commit(mbar);
}

template <int NA, int NT>
__global__ void __launch_bounds__(256, 1) k_products_tc(const __grid_constant__ CondArgs a) {
  using Sh = TcShape<NA, NT>;
  using namespace tc;
  constexpr int K1 = Sh::K1, NA4 = NA / 4;
  constexpr uint32_t SBO = Sh::SBO;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* Ahi = tc_smem;
  unsigned char* Alo = Ahi + Sh::A_BYTES;
  unsigned char* Bhi = Alo + Sh::A_BYTES;
  unsigned char* Blo = Bhi + Sh::B_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Blo + Sh::B_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  float* s_row = reinterpret_cast<float*>(mbar + 2);  // row NT (x_r / C x_r): 2 halves x 16
  int* s_pv = reinterpret_cast<int*>(s_row + 32);     // two buffers of NA pivots
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const bool issuer = w == Sh::ISSUER;
  const int q = w & 3, hh = w >> 2;  // tensor-memory lane quarter, column half
  const int j = 32 * q + lane;       // this thread's row of both accumulators (trace index)
  const bool epi = q < 3;            // warps whose lanes hold rows j <= NT
  const bool rowNT = q == NT / 32;   // warps whose lane NT % 32 holds row NT
  if (t == 0) mbar_init(smem_u32(mbar), 1);
  if (issuer) tmem_alloc(smem_u32(tslot), Sh::TMEM_COLS);
  const int G = gridDim.x;
  int k = blockIdx.x;
  if (k < a.Eim)
    for (int c = t; c < NA; c += blockDim.x) s_pv[c] = a.piv[(size_t)k * NA + c];
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t tlane = (uint32_t)(32 * q) << 16;
  bool ok = true;
  uint32_t pend = 0;  // parity of the phase being waited for
  TcStage<NA, NT> g;
  if (k < a.Eim && !issuer) tc_load_stage<NA, NT>(g, a, k, s_pv, t);
  static_assert(NA <= Sh::THREADS, "one pivot per thread");
  if (issuer && lane == 0 && k + G < a.Eim) {  // the first iteration loads element k + G
    const size_t o = (size_t)k + G;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const float*>(a.LU) + o * NA * NA),
                 "r"((unsigned)(NA * NA * 4)) : "memory");
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const float*>(a.B) + o * NA * NT),
                 "r"((unsigned)(NA * NT * 4)) : "memory");
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const float*>(a.C) + o * NT * NA),
                 "r"((unsigned)(NT * NA * 4)) : "memory");
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const float*>(a.D) + o * NT * NT),
                 "r"((unsigned)(NT * NT * 4)) : "memory");
  }
  int pv_next = (k + G < a.Eim && t < NA) ? __ldg(a.piv + (size_t)(k + G) * NA + t) : 0;
  for (int it = 0; k < a.Eim; k += G, ++it) {
    const int buf = it & 1;
    const int kn = k + G;
    if (!issuer) tc_store_stage<NA, NT>(g, Ahi, Alo, Bhi, Blo, t);
    // the next element's pivots, read one iteration ahead (this buffer's last reader was two
    // iterations ago)
    if (kn < a.Eim && t < NA) s_pv[(buf ^ 1) * NA + t] = pv_next;
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    if (issuer && lane == 0) {
      tc_issue<NA, NT>(tmem, Ahi, Alo, Bhi, Blo, idesc_tf32(128, Sh::N1), smem_u32(mbar), a.tc_mode != 3);
      // L2 prefetch of the operands one load-phase ahead: the factor and B two elements ahead (the
      // next element's are loaded into registers in this iteration), C and D one element ahead
      // (this element's are read in this iteration); farther ahead overflows the L2 (measured)
      if (kn + G < a.Eim) {
        const size_t o = (size_t)kn + G;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const float*>(a.LU) + o * NA * NA),
                     "r"((unsigned)(NA * NA * 4)) : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const float*>(a.B) + o * NA * NT),
                     "r"((unsigned)(NA * NT * 4)) : "memory");
      }
      if (kn < a.Eim) {
        const size_t o = (size_t)kn;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const float*>(a.C) + o * NT * NA),
                     "r"((unsigned)(NT * NA * 4)) : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<const float*>(a.D) + o * NT * NT),
                     "r"((unsigned)(NT * NT * 4)) : "memory");
      }
    }
    // C for GEMM 2, read while GEMM 1 runs
    const float* gC = reinterpret_cast<const float*>(a.C) + (size_t)k * NT * NA;
    float4 creg[Sh::C_PER];
#pragma unroll
    for (int u = 0; u < Sh::C_PER; ++u) {
      const int task = w + Sh::WARPS * u;
      const int i = 8 * (task / Sh::CG) + (lane & 7), ch = 4 * (task % Sh::CG) + (lane >> 3);
      creg[u] = (w < Sh::WARPS && task < Sh::C_TASKS && ch < NA4)
                    ? __ldg(reinterpret_cast<const float4*>(gC + (size_t)i * NA) + ch)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // the next element's GEMM 1 operands, in flight during GEMM 1, epilogue 1 and GEMM 2
    if (kn < a.Eim && !issuer) tc_load_stage<NA, NT>(g, a, kn, s_pv + (buf ^ 1) * NA, t);
    pend = 0;
    ok = mbar_wait(smem_u32(mbar), 0, tc::TIMEOUT_NS);
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    fence_after_sync();
    // ---- epilogue 1: X_B, x_r out; [X_B | x_r]^T as GEMM 2's A operand; C as its B operand
    if (epi) {
      float* gXB = reinterpret_cast<float*>(a.XB) + (size_t)k * NA * NT;
      double* gxr = a.xr + (size_t)k * NA;
      const int cb = hh == 0 ? 0 : Sh::H1, ce = hh == 0 ? Sh::H1 : Sh::NCH1;
      for (int cc = cb; cc < ce; ++cc) {
        float v[16];
        tmem_ld16(tmem + tlane + (uint32_t)(16 * cc), v);
        if (rowNT) {  // row NT is x_r: its lane hands the 16 values over through shared memory
          if (lane == (NT & 31))
#pragma unroll
            for (int u = 0; u < 16; u += 4)
              *reinterpret_cast<float4*>(s_row + 16 * hh + u) = make_float4(v[u], v[u + 1], v[u + 2], v[u + 3]);
          __syncwarp();
          if (lane < 16 && 16 * cc + lane < NA) gxr[16 * cc + lane] = double(s_row[16 * hh + lane]);
          __syncwarp();
        }
        if (j <= NT) {
          if (j < NT) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              const int i = 16 * cc + u;
              if (i < NA) gXB[(size_t)i * NT + j] = v[u];
            }
          }
#pragma unroll
          for (int u = 0; u < 16; u += 4) {
            const int i = 16 * cc + u;
            if (i < K1) {
              float hs[4], ls[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) split_tf32(i + e < NA ? v[u + e] : 0.f, hs[e], ls[e]);
              *reinterpret_cast<float4*>(Ahi + kmajor_offset(j, i, SBO)) = make_float4(hs[0], hs[1], hs[2], hs[3]);
              *reinterpret_cast<float4*>(Alo + kmajor_offset(j, i, SBO)) = make_float4(ls[0], ls[1], ls[2], ls[3]);
            }
          }
        }
      }
    }
    if (w < Sh::WARPS) {
#pragma unroll
      for (int u = 0; u < Sh::C_PER; ++u) {
        const int task = w + Sh::WARPS * u;
        const int i = 8 * (task / Sh::CG) + (lane & 7), ch = 4 * (task % Sh::CG) + (lane >> 3);
        if (task < Sh::C_TASKS && ch < Sh::KG) {
          float hs[4], ls[4];
          split_tf32(creg[u].x, hs[0], ls[0]);
          split_tf32(creg[u].y, hs[1], ls[1]);
          split_tf32(creg[u].z, hs[2], ls[2]);
          split_tf32(creg[u].w, hs[3], ls[3]);
          *reinterpret_cast<float4*>(Bhi + kmajor_offset(i, 4 * ch, SBO)) = make_float4(hs[0], hs[1], hs[2], hs[3]);
          *reinterpret_cast<float4*>(Blo + kmajor_offset(i, 4 * ch, SBO)) = make_float4(ls[0], ls[1], ls[2], ls[3]);
        }
      }
    }
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    if (issuer && lane == 0)
      tc_issue<NA, NT>(tmem + Sh::D2_COL, Ahi, Alo, Bhi, Blo, idesc_tf32(128, Sh::N2), smem_u32(mbar), a.tc_mode != 3);
    if (kn + G < a.Eim && t < NA) pv_next = __ldg(a.piv + (size_t)(kn + G) * NA + t);
    // while GEMM 2 runs: this element's D and s
    const int cb2 = hh == 0 ? 0 : Sh::H2, ce2 = hh == 0 ? Sh::H2 : Sh::NCH2;
    const float* gD = reinterpret_cast<const float*>(a.D) + (size_t)k * NT * NT;
    float dreg[16 * Sh::H2];
#pragma unroll
    for (int u = 0; u < 16 * Sh::H2; ++u) {
      const int i = 16 * cb2 + u;
      dreg[u] = (epi && j < NT && i < 16 * ce2 && i < NT) ? __ldg(gD + (size_t)i * NT + j) : 0.f;
    }
    double sreg[Sh::H2];  // lane u of a row-NT warp stores t[16 cc + u]
#pragma unroll
    for (int u = 0; u < Sh::H2; ++u) {
      const int i = 16 * (cb2 + u) + lane;
      sreg[u] = (rowNT && lane < 16 && cb2 + u < ce2 && i < NT) ? __ldg(a.s + (size_t)k * NT + i) : 0.0;
    }
    pend = 1;
    ok = mbar_wait(smem_u32(mbar), 1, tc::TIMEOUT_NS);
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    fence_after_sync();
    // ---- epilogue 2: S = D - C X_B, t = s - C x_r
    if (epi) {
      float* gS = reinterpret_cast<float*>(a.S) + (size_t)k * NT * NT;
      for (int cc = cb2; cc < ce2; ++cc) {
        float v[16];
        tmem_ld16(tmem + tlane + Sh::D2_COL + (uint32_t)(16 * cc), v);
        if (j < NT) {
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int i = 16 * cc + u;
            if (i < NT) gS[(size_t)i * NT + j] = dreg[16 * (cc - cb2) + u] - v[u];
          }
        }
        if (rowNT) {
          if (lane == (NT & 31))
#pragma unroll
            for (int u = 0; u < 16; u += 4)
              *reinterpret_cast<float4*>(s_row + 16 * hh + u) = make_float4(v[u], v[u + 1], v[u + 2], v[u + 3]);
          __syncwarp();
          double sv = 0.0;
#pragma unroll
          for (int u = 0; u < Sh::H2; ++u)
            if (cc - cb2 == u) sv = sreg[u];
          if (lane < 16 && 16 * cc + lane < NT) a.t[(size_t)k * NT + 16 * cc + lane] = sv - double(s_row[16 * hh + lane]);
          __syncwarp();
        }
      }
    }
    fence_before_sync();
  }
  if (!ok) {
    if (t == 0) atomicOr(a.status, DEV_ERR_TIMEOUT);
    mbar_wait(smem_u32(mbar), pend, tc::TIMEOUT_NS);  // let MMAs in flight finish before freeing
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (issuer) tmem_dealloc(tmem, Sh::TMEM_COLS);
}

template <int NA, int NT>
static cudaError_t launch_products_tc(const CondArgs& a, cudaStream_t st) {
  using Sh = TcShape<NA, NT>;
  static int grid = 0;
  if (grid == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_products_tc<NA, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Sh::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_products_tc<NA, NT>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, occ = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_products_tc<NA, NT>, Sh::THREADS, Sh::SMEM)) !=
        cudaSuccess)
      return e;
    // at most two resident CTAs per SM: each holds 256 of the SM's 512 tensor-memory columns
    grid = nsm * (occ < 1 ? 1 : (occ > 2 ? 2 : occ));
  }
  const int g = a.Eim < grid ? a.Eim : grid;
  (hfr::count_launch(), k_products_tc<NA, NT><<<g, Sh::THREADS, Sh::SMEM, st>>>(a));
  return cudaGetLastError();
}

template <int NA, int NT>
static cudaError_t cond_two_kernel(const CondArgs& a, cudaStream_t st, int part) {
  using P = ProdShape<NA, NT>;
  if (part == 0) {
    if (a.tc_mode >= 2) return launch_inverse_tc<NA>(a, st);
    if constexpr (NA <= 64) {
      constexpr int WPB = InvWShape<NA>::WPB;
      (hfr::count_launch(), k_inverse_warp<NA><<<(a.Eim + WPB - 1) / WPB, 32 * WPB, 0, st>>>(a));
    } else {
      constexpr int RPT = INV_RPT_LARGE;
      (hfr::count_launch(), k_inverse_rq<NA, RPT><<<a.Eim, InvRShape<NA, RPT>::THREADS, 0, st>>>(a));
    }
    return cudaGetLastError();
  }
  if (a.tc_mode >= 1) return launch_products_tc<NA, NT>(a, st);
  if constexpr (NA > 64) {
    using SS = StreamShape<NA, NT>;
    (hfr::count_launch(), k_products_x<NA, NT><<<a.Eim, SS::TX, 0, st>>>(a));
    (hfr::count_launch(), k_products_s<NA, NT><<<a.Eim, SS::TSS, 0, st>>>(a));
    return cudaGetLastError();
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_condense_products<NA, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)P::SMEM);
    if (e != cudaSuccess) return e;
    (hfr::count_launch(), k_condense_products<NA, NT><<<a.Eim, P::THREADS, P::SMEM, st>>>(a));
    return cudaGetLastError();
  }
}

// ------------------------------------------------------------- generic shared-memory kernel
// Same algorithm and outputs for any (nA, nT) and either precision; the augmented block lives
// in shared memory.  Used where the register tile does not fit (e.g. FP64 with nA >= 100).
constexpr int GJS_THREADS = 256;

// One element's blocks and outputs (row-major, the layouts of CondArgs) for the shared-memory
// condensation: used by the uniform launch (fixed strides) and by the uneven-shape launch (offsets).
template <typename T>
struct CondElem {
  int nA, nT, id;
  const T *A, *B, *C, *D;
  const double *r, *s;
  T* LU;  // ((PA)^{-1})^T
  int* piv;
  T* XB;
  double* xr;
  T* S;
  double* t;
};

// barrier of one thread group (id 0 with the whole CTA is __syncthreads)
__device__ __forceinline__ void grp_sync(int id, int nth) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nth) : "memory");
}

// Gauss-Jordan on [A | B | r] in shared memory with partial pivoting (rows not exchanged), then
// S = D - C X_B and t = s - C x_r, by a group of nth threads (a multiple of 32; tid is the thread's
// index in the group, bar its named barrier).  Ends with a group barrier, so the group may reuse
// its memory.
template <typename T>
__device__ void condense_smem_elem(const CondElem<T>& e, unsigned char* smem_raw, int* status, int tid, int nth,
                                   int bar) {
  const int nA = e.nA, nT = e.nT, nc = nA + nT + 1;
  const int big = nA > nT ? nA : nT;
  T* M = reinterpret_cast<T*>(smem_raw);  // nA x nc, physical rows
  T* W = M + (size_t)nA * nc;             // big x nA
  T* pr = W + (size_t)big * nA;           // nc
  T* cb = pr + nc;                        // nA
  int* ipiv = reinterpret_cast<int*>(cb + nA);  // physical row -> elimination step
  int* lpiv = ipiv + nA;                          // elimination step -> physical row
  int* sflag = lpiv + nA;  // [0] pivot row of the step, [1] zero pivot seen
  unsigned char* used = reinterpret_cast<unsigned char*>(sflag + 2);
  const int lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
  int& s_p = sflag[0];
  int& s_bad = sflag[1];
  for (int i = tid; i < nA * nc; i += nth) {
    const int r = i / nc, j = i % nc;
    M[i] = j < nA ? e.A[(size_t)r * nA + j] : (j < nA + nT ? e.B[(size_t)r * nT + (j - nA)] : T(e.r[r]));
  }
  for (int i = tid; i < nA; i += nth) used[i] = 0;
  if (tid == 0) s_bad = 0;
  grp_sync(bar, nth);
  for (int c = 0; c < nA; ++c) {
    if (tid < 32) {
      T best = T(-1);
      int bi = 0x7fffffff;
      for (int r = tid; r < nA; r += 32) {
        if (used[r]) continue;
        const T v = tabs(M[(size_t)r * nc + c]);
        if (v > best || (v == best && r < bi)) { best = v; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (bi >= nA) bi = c;  // no candidate compared (NaN column): any row, flagged singular
      if (tid == 0) {
        s_p = bi;
        used[bi] = 1;
        ipiv[bi] = c;
        lpiv[c] = bi;
        e.piv[c] = bi;
        if (!(best > T(0))) s_bad = 1;
      }
    }
    grp_sync(bar, nth);
    const int p = s_p;
    const T pv = M[(size_t)p * nc + c];
    const T inv = pv != T(0) ? T(1) / pv : T(0);
    for (int j = tid; j < nc; j += nth) pr[j] = j == c ? inv : M[(size_t)p * nc + j] * inv;
    for (int r = tid; r < nA; r += nth) cb[r] = M[(size_t)r * nc + c];
    grp_sync(bar, nth);
    // one warp per row, lanes along the row
    for (int r = wid; r < nA; r += nw) {
      T* Mr = M + (size_t)r * nc;
      if (r == p) {
        for (int j = lane; j < nc; j += 32) Mr[j] = pr[j];
      } else {
        const T l = cb[r];
        for (int j = lane; j < nc; j += 32) Mr[j] = (j == c ? T(0) : Mr[j]) - l * pr[j];
      }
    }
    grp_sync(bar, nth);
  }
  if (tid == 0 && s_bad) {
    atomicOr(status, DEV_ERR_SINGULAR);
    atomicMin(status + 1, e.id);
  }
  for (int i = tid; i < nA * nc; i += nth) {
    const int r = i / nc, j = i % nc;
    const int lr = ipiv[r];
    if (j < nA)
      e.LU[(size_t)j * nA + lr] = M[i];
    else if (j < nA + nT)
      e.XB[(size_t)lr * nT + (j - nA)] = M[i];
    else
      e.xr[lr] = double(M[i]);
  }
  // C into W; X rows in logical order are read through the pivot sequence
  for (int i = tid; i < nT * nA; i += nth) W[i] = e.C[i];
  grp_sync(bar, nth);
  // [S | t] = [D | s] - C [X_B | x_r]: 4 x 4 outputs per thread (rows i0.., columns j0..)
  const int ni = (nT + 3) >> 2, nj = (nT + 4) >> 2;
  for (int it = tid; it < ni * nj; it += nth) {
    const int i0 = (it / nj) * 4, j0 = (it % nj) * 4;
    T acc[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[q][u] = T(0);
    const T* Wr[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) Wr[q] = W + (size_t)min(i0 + q, nT - 1) * nA;
    int jc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) jc[u] = nA + min(j0 + u, nT);
    for (int l = 0; l < nA; ++l) {
      const T* Xl = M + (size_t)lpiv[l] * nc;
      T a4[4], b4[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) a4[q] = Wr[q][l];
#pragma unroll
      for (int u = 0; u < 4; ++u) b4[u] = Xl[jc[u]];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[q][u] += a4[q] * b4[u];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + q;
      if (i >= nT) continue;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + u;
        if (j < nT)
          e.S[(size_t)i * nT + j] = e.D[(size_t)i * nT + j] - acc[q][u];
        else if (j == nT)
          e.t[i] = e.s[i] - double(acc[q][u]);
      }
    }
  }
  grp_sync(bar, nth);
}

template <typename T>
__global__ void __launch_bounds__(GJS_THREADS) k_condense_smem(const __grid_constant__ CondArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = blockIdx.x, nA = a.nA, nT = a.nT;
  CondElem<T> e;
  e.nA = nA;
  e.nT = nT;
  e.id = k;
  e.A = reinterpret_cast<const T*>(a.A) + (size_t)k * nA * nA;
  e.B = reinterpret_cast<const T*>(a.B) + (size_t)k * nA * nT;
  e.C = reinterpret_cast<const T*>(a.C) + (size_t)k * nT * nA;
  e.D = reinterpret_cast<const T*>(a.D) + (size_t)k * nT * nT;
  e.r = a.r + (size_t)k * nA;
  e.s = a.s + (size_t)k * nT;
  e.LU = reinterpret_cast<T*>(a.LU) + (size_t)k * nA * nA;
  e.piv = a.piv + (size_t)k * nA;
  e.XB = reinterpret_cast<T*>(a.XB) + (size_t)k * nA * nT;
  e.xr = a.xr + (size_t)k * nA;
  e.S = reinterpret_cast<T*>(a.S) + (size_t)k * nT * nT;
  e.t = a.t + (size_t)k * nT;
  condense_smem_elem<T>(e, smem_raw, a.status, (int)threadIdx.x, GJS_THREADS, 0);
}

// Elements of uneven block shapes (e.g. several polynomial degrees) condensed in one persistent
// launch: the CTAs walk a list of bundles ordered by decreasing element cost.  A bundle holds up to
// `groups` elements of one shape; the CTA splits into that many thread groups, each condensing one
// element in its own slice of shared memory (stride bytes apart) with its own named barrier, so
// small elements run several to a CTA while the dynamic shared memory is sized for the largest.
// Element k has shape shape[2 k], shape[2 k + 1] and its blocks at the offsets off[5 k ..] into
// the packed arrays (A-sized: A, LU; B-sized: B, C, X_B; D-sized: D, S; nA-sized: r, x_r, piv;
// nT-sized: s, t).
constexpr int UNEVEN_THREADS = 1024, UNEVEN_MAX_GROUPS = 8;
struct UnevenArgs {
  int nb;
  const int* bundle;  // per bundle: first position in order, elements, groups, stride (bytes)
  const int* order;
  const int* shape;
  const long long* off;
  const void *A, *B, *C, *D;
  const double *r, *s;
  void* LU;
  int* piv;
  void* XB;
  double* xr;
  void* S;
  double* t;
  int* status;
  int colmajor = 0;  // A, B, C, D stored column-major (global-memory kernel only)
};

template <typename T>
__global__ void __launch_bounds__(UNEVEN_THREADS) k_condense_uneven(const __grid_constant__ UnevenArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int b = blockIdx.x; b < a.nb; b += gridDim.x) {
    const int* bd = a.bundle + 4 * (size_t)b;
    const int start = bd[0], cnt = bd[1], groups = bd[2], stride = bd[3];
    const int nth = UNEVEN_THREADS / groups;
    const int g = (int)threadIdx.x / nth;
    if (g < cnt) {
      const int k = a.order[start + g];
      const long long* o = a.off + 5 * (size_t)k;
      CondElem<T> e;
      e.nA = a.shape[2 * k];
      e.nT = a.shape[2 * k + 1];
      e.id = k;
      e.A = reinterpret_cast<const T*>(a.A) + o[0];
      e.LU = reinterpret_cast<T*>(a.LU) + o[0];
      e.B = reinterpret_cast<const T*>(a.B) + o[1];
      e.C = reinterpret_cast<const T*>(a.C) + o[1];
      e.XB = reinterpret_cast<T*>(a.XB) + o[1];
      e.D = reinterpret_cast<const T*>(a.D) + o[2];
      e.S = reinterpret_cast<T*>(a.S) + o[2];
      e.r = a.r + o[3];
      e.xr = a.xr + o[3];
      e.piv = a.piv + o[3];
      e.s = a.s + o[4];
      e.t = a.t + o[4];
      condense_smem_elem<T>(e, smem_raw + (size_t)g * stride, a.status, (int)threadIdx.x - g * nth, nth,
                            groups == 1 ? 0 : 1 + g);
    }
    __syncthreads();  // the next bundle reuses the memory
  }
}

static size_t smem_elem_bytes(size_t tb, int nA, int nT) {
  const int nc = nA + nT + 1, big = nA > nT ? nA : nT;
  return tb * ((size_t)nA * nc + (size_t)big * nA + nc + nA) + sizeof(int) * (2 * (size_t)nA + 2) + nA;
}

}  // namespace hfr
#include "hfr_bigblock.cuh"
namespace hfr {

bool uneven_fits_smem(int prec_bytes, int nA, int nT) {
  return smem_elem_bytes((size_t)prec_bytes, nA, nT) <= 227 * 1024;
}

// largest nA of an uneven batch that goes to the shared-memory Gauss-Jordan bundles; larger blocks
// take the blocked LU with the column-block solve and batched GEMMs.  Measured on 10 000 FP32
// blocks per shape (call wall time): nA = 144, nT = 96: 40.3 ms in the bundles (shared-memory
// bound rank-1 steps), 26.0 ms blocked; nA = 100, nT = 80: 23.0 / 18.6 ms; nA = 64, nT = 64: 13.4
// / 13.2 ms (even).  FP64 blocks keep the bundles up to nA = 128 (both forms on the FP64 pipe).
// Build flags, for timing the two forms against each other.
#ifndef HFR_UNEVEN_SMEM_MAX_NA
#define HFR_UNEVEN_SMEM_MAX_NA 64
#endif
#ifndef HFR_UNEVEN_SMEM_MAX_NA_FP64
#define HFR_UNEVEN_SMEM_MAX_NA_FP64 128
#endif
static bool uneven_route_smem(int prec_bytes, int nA, int nT) {
  return uneven_fits_smem(prec_bytes, nA, nT) &&
         nA <= (prec_bytes == 8 ? HFR_UNEVEN_SMEM_MAX_NA_FP64 : HFR_UNEVEN_SMEM_MAX_NA);
}

// Host tables of an uneven launch: per element offsets (A, B/C, D, nA-, nT-vectors), shapes, the
// shared-memory elements' order (most expensive first) and bundles, and the elements too large for
// shared memory (global-memory kernel).
int uneven_tables(int prec_bytes, int n, const int* nA, const int* nT, UnevenTables* tb, const unsigned char* skip) {
  tb->off.assign(5 * (size_t)n, 0);
  tb->shape.assign(2 * (size_t)n, 0);
  tb->order.clear();
  tb->bundle.clear();
  tb->global.clear();
  tb->smem = 0;
  long long oa = 0, ob = 0, od = 0, ova = 0, ovt = 0;
  for (int k = 0; k < n; ++k) {
    if (nA[k] < 1 || nT[k] < 1 || nT[k] > 16384) return -1;
    tb->shape[2 * k] = nA[k];
    tb->shape[2 * k + 1] = nT[k];
    long long* o = &tb->off[5 * (size_t)k];
    o[0] = oa;
    o[1] = ob;
    o[2] = od;
    o[3] = ova;
    o[4] = ovt;
    oa += (long long)nA[k] * nA[k];
    ob += (long long)nA[k] * nT[k];
    od += (long long)nT[k] * nT[k];
    ova += nA[k];
    ovt += nT[k];
    if (skip && skip[k]) continue;  // condensed elsewhere: offsets only
    if (uneven_route_smem(prec_bytes, nA[k], nT[k])) {
      tb->order.push_back(k);
      const size_t sb = smem_elem_bytes(prec_bytes, nA[k], nT[k]);
      tb->smem = sb > tb->smem ? sb : tb->smem;
    } else {
      tb->global.push_back(k);
      tb->gmax_nA = nA[k] > tb->gmax_nA ? nA[k] : tb->gmax_nA;
      tb->gmax_nT = nT[k] > tb->gmax_nT ? nT[k] : tb->gmax_nT;
    }
  }
  auto cost = [&](int k) {
    const double x = nA[k], y = nT[k];
    return x * x * (x + y) + y * y * x;
  };
  std::stable_sort(tb->order.begin(), tb->order.end(), [&](int x, int y) { return cost(x) > cost(y); });
  std::stable_sort(tb->global.begin(), tb->global.end(), [&](int x, int y) { return cost(x) > cost(y); });
  const int m = (int)tb->order.size();
  for (int i = 0; i < m;) {
    const int k0 = tb->order[i];
    int j = i;
    while (j < m && nA[tb->order[j]] == nA[k0] && nT[tb->order[j]] == nT[k0]) ++j;
    const size_t stride = (smem_elem_bytes(prec_bytes, nA[k0], nT[k0]) + 15) / 16 * 16;
    int groups = 1;
    while (groups < UNEVEN_MAX_GROUPS && (size_t)(2 * groups) * stride <= tb->smem) groups *= 2;
    for (int q = i; q < j; q += groups) {
      tb->bundle.push_back(q);
      tb->bundle.push_back(j - q < groups ? j - q : groups);
      tb->bundle.push_back(groups);
      tb->bundle.push_back((int)stride);
    }
    i = j;
  }
  return 0;
}

size_t uneven_dev_bytes(const UnevenTables& tb) {
  return sizeof(long long) * tb.off.size() +
         sizeof(int) * (tb.order.size() + tb.shape.size() + tb.bundle.size() + tb.global.size()) + 64;
}

cudaError_t uneven_upload(const UnevenTables& tb, void* dbuf, UnevenDev* dv, cudaStream_t st) {
  long long* d_off = reinterpret_cast<long long*>(dbuf);
  int* d_order = reinterpret_cast<int*>(d_off + tb.off.size());
  int* d_shape = d_order + tb.order.size();
  int* d_bund = d_shape + tb.shape.size();
  int* d_glob = d_bund + tb.bundle.size();
  cudaError_t e;
  if (!tb.off.empty() &&
      (e = cudaMemcpyAsync(d_off, tb.off.data(), sizeof(long long) * tb.off.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  if (!tb.order.empty() &&
      (e = cudaMemcpyAsync(d_order, tb.order.data(), sizeof(int) * tb.order.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  if (!tb.shape.empty() &&
      (e = cudaMemcpyAsync(d_shape, tb.shape.data(), sizeof(int) * tb.shape.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  if (!tb.bundle.empty() &&
      (e = cudaMemcpyAsync(d_bund, tb.bundle.data(), sizeof(int) * tb.bundle.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  if (!tb.global.empty() &&
      (e = cudaMemcpyAsync(d_glob, tb.global.data(), sizeof(int) * tb.global.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  dv->off = d_off;
  dv->order = d_order;
  dv->shape = d_shape;
  dv->bundle = d_bund;
  dv->global = d_glob;
  dv->nb = (int)(tb.bundle.size() / 4);
  dv->nglobal = (int)tb.global.size();
  dv->smem = tb.smem;
  dv->gmax_nA = tb.gmax_nA;
  dv->gmax_nT = tb.gmax_nT;
  return cudaSuccess;
}

cudaError_t launch_condense_uneven_dev(int prec_bytes, const UnevenDev& dv, const void* A, const void* B, const void* C,
                                       const void* D, const double* r, const double* s, void* LU, int* piv, void* XB,
                                       double* xr, void* S, double* t, int* status, cudaStream_t st) {
  UnevenArgs ua{dv.nb, dv.bundle, dv.order, dv.shape, dv.off, A, B, C, D, r, s, LU, piv, XB, xr, S, t, status,
                dv.colmajor};
  if (dv.colmajor && dv.nb > 0) return cudaErrorInvalidValue;  // column-major blocks: global kernel only
  int dev = 0, nsm = 0, occ = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (dv.nb > 0) {
    const size_t smem = dv.smem;
    if (prec_bytes == 8) {
      if ((e = cudaFuncSetAttribute(k_condense_uneven<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_condense_uneven<double>, UNEVEN_THREADS, smem);
    } else {
      if ((e = cudaFuncSetAttribute(k_condense_uneven<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_condense_uneven<float>, UNEVEN_THREADS, smem);
    }
    if (e != cudaSuccess) return e;
    int grid = nsm * (occ < 1 ? 1 : occ);
    grid = dv.nb < grid ? dv.nb : grid;
    if (prec_bytes == 8)
      (hfr::count_launch(), k_condense_uneven<double><<<grid, UNEVEN_THREADS, smem, st>>>(ua));
    else
      (hfr::count_launch(), k_condense_uneven<float><<<grid, UNEVEN_THREADS, smem, st>>>(ua));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (dv.nglobal > 0) {
    e = prec_bytes == 8 ? big::condense_big<double>(ua, dv.global, dv.nglobal, 0, 0, dv.gmax_nA, dv.gmax_nT, st)
                        : big::condense_big<float>(ua, dv.global, dv.nglobal, 0, 0, dv.gmax_nA, dv.gmax_nT, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ------------------------------------------- one shape class of a packed uneven batch
// Elements of one shape (nA, nT) scattered through the packed arrays of an uneven batch, condensed
// by the fixed-shape kernels of that shape (e.g. the tensor-core inverse and products) through a
// contiguous scratch batch: gather, launch_condense, scatter, in chunks of at most `cap` elements.
struct ClassScratch {
  size_t a, b, d, va, vt;  // values per chunk: nA^2, nA nT, nT^2, nA, nT (times cap)
  float *A, *B, *C, *D, *LU, *XB, *S;
  double *r, *s, *xr, *t;
  int* piv;
  int* status;  // two words: the chunk's own status (DEV_ERR_*, first failing chunk element)
};
size_t class_scratch_bytes(int nA, int nT, int cap) {
  const size_t c = (size_t)cap, a = c * nA * nA, b = c * nA * nT, d = c * nT * nT;
  return 4 * (2 * a + 3 * b + 2 * d) + 8 * (2 * c * nA + 2 * c * nT) + 4 * c * nA + 64 + 8 * 16;
}
static ClassScratch class_scratch(void* buf, int nA, int nT, int cap) {
  ClassScratch cs;
  const size_t c = (size_t)cap;
  cs.a = c * nA * nA;
  cs.b = c * nA * nT;
  cs.d = c * nT * nT;
  cs.va = c * nA;
  cs.vt = c * nT;
  cs.status = reinterpret_cast<int*>(buf);  // first 16 bytes: the same place for every shape
  double* dp = reinterpret_cast<double*>(reinterpret_cast<char*>(buf) + 16);
  cs.r = dp;
  cs.xr = cs.r + cs.va;
  cs.s = cs.xr + cs.va;
  cs.t = cs.s + cs.vt;
  float* fp = reinterpret_cast<float*>(cs.t + cs.vt);
  cs.A = fp;
  cs.LU = cs.A + cs.a;
  cs.B = cs.LU + cs.a;
  cs.C = cs.B + cs.b;
  cs.XB = cs.C + cs.b;
  cs.D = cs.XB + cs.b;
  cs.S = cs.D + cs.d;
  cs.piv = reinterpret_cast<int*>(cs.S + cs.d);
  return cs;
}

// copies of n values (16-byte vectors where both sides allow them)
__device__ __forceinline__ void class_copy(const float* __restrict__ src, float* __restrict__ dst, size_t n) {
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0) {
    const size_t n4 = n / 4;
    for (size_t i = threadIdx.x; i < n4; i += blockDim.x)
      reinterpret_cast<float4*>(dst)[i] = reinterpret_cast<const float4*>(src)[i];
    for (size_t i = 4 * n4 + threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
  } else {
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
  }
}
template <typename V>
__device__ __forceinline__ void class_copy_v(const V* __restrict__ src, V* __restrict__ dst, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// chunk element i (one CTA each) <- packed element list[i]
__global__ void __launch_bounds__(256) k_class_gather(const int* __restrict__ list, const long long* __restrict__ off,
                                                      int nA, int nT, const float* A, const float* B, const float* C,
                                                      const float* D, const double* r, const double* s,
                                                      ClassScratch cs) {
  const int i = blockIdx.x, k = list[i];
  const long long* o = off + 5 * (size_t)k;
  const size_t a = (size_t)nA * nA, b = (size_t)nA * nT, d = (size_t)nT * nT;
  class_copy(A + o[0], cs.A + i * a, a);
  class_copy(B + o[1], cs.B + i * b, b);
  class_copy(C + o[1], cs.C + i * b, b);
  class_copy(D + o[2], cs.D + i * d, d);
  class_copy_v(r + o[3], cs.r + (size_t)i * nA, nA);
  class_copy_v(s + o[4], cs.s + (size_t)i * nT, nT);
}

// packed element list[i] <- chunk element i: factors, pivots, X_B, x_r, S, t
__global__ void __launch_bounds__(256) k_class_scatter(const int* __restrict__ list, const long long* __restrict__ off,
                                                       int nA, int nT, ClassScratch cs, float* LU, int* piv, float* XB,
                                                       double* xr, float* S, double* t) {
  const int i = blockIdx.x, k = list[i];
  const long long* o = off + 5 * (size_t)k;
  const size_t a = (size_t)nA * nA, b = (size_t)nA * nT, d = (size_t)nT * nT;
  class_copy(cs.LU + i * a, LU + o[0], a);
  class_copy(cs.XB + i * b, XB + o[1], b);
  class_copy(cs.S + i * d, S + o[2], d);
  class_copy_v(cs.piv + (size_t)i * nA, piv + o[3], nA);
  class_copy_v(cs.xr + (size_t)i * nA, xr + o[3], nA);
  class_copy_v(cs.t + (size_t)i * nT, t + o[4], nT);
}

// the chunk's status into the batch's (its first failing element as a packed element id)
__global__ void k_class_status(int* cstatus, const int* __restrict__ list, int k0, int cnt, int* status) {
  if (cstatus[0] != 0) {
    atomicOr(status, cstatus[0]);
    const int i = cstatus[1];
    atomicMin(status + 1, (i >= 0 && i < cnt) ? (list ? list[i] : k0 + i) : -1);
  }
  cstatus[0] = 0;
  cstatus[1] = 0x7fffffff;
}

cudaError_t launch_condense_class(const int* list, int count, int nA, int nT, const long long* off, const void* A,
                                  const void* B, const void* C, const void* D, const double* r, const double* s,
                                  void* LU, int* piv, void* XB, double* xr, void* S, double* t, int* status,
                                  void* scratch, int cap, int tc_mode, cudaStream_t st, int contig_k0,
                                  const long long* contig_off) {
  if (count <= 0) return cudaSuccess;
  if (!condense_feasible(4, nA, nT)) return cudaErrorInvalidValue;
  cudaError_t e;
  if (contig_k0 >= 0) {  // consecutive elements of one shape: uniform strides, condensed in place
    const long long* o = contig_off;
    CondArgs ca;
    ca.Eim = count;
    ca.nA = nA;
    ca.nT = nT;
    ca.A = static_cast<const float*>(A) + o[0];
    ca.B = static_cast<const float*>(B) + o[1];
    ca.C = static_cast<const float*>(C) + o[1];
    ca.D = static_cast<const float*>(D) + o[2];
    ca.r = r + o[3];
    ca.s = s + o[4];
    ca.LU = static_cast<float*>(LU) + o[0];
    ca.piv = piv + o[3];
    ca.XB = static_cast<float*>(XB) + o[1];
    ca.xr = xr + o[3];
    ca.S = static_cast<float*>(S) + o[2];
    ca.t = t + o[4];
    ca.status = reinterpret_cast<int*>(scratch);  // the scratch buffer's leading status words
    ca.tc_mode = tc_mode;
    if ((e = launch_condense(4, ca, st)) != cudaSuccess) return e;
    (hfr::count_launch(), k_class_status<<<1, 1, 0, st>>>(ca.status, nullptr, contig_k0, count, status));
    return cudaGetLastError();
  }
  if (cap <= 0) return cudaErrorInvalidValue;
  const ClassScratch cs = class_scratch(scratch, nA, nT, cap);
  for (int base = 0; base < count; base += cap) {
    const int cnt = count - base < cap ? count - base : cap;
    (hfr::count_launch(), k_class_gather<<<cnt, 256, 0, st>>>(list + base, off, nA, nT, (const float*)A,
                                                               (const float*)B, (const float*)C, (const float*)D, r, s,
                                                               cs));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    CondArgs ca;
    ca.Eim = cnt;
    ca.nA = nA;
    ca.nT = nT;
    ca.A = cs.A;
    ca.B = cs.B;
    ca.C = cs.C;
    ca.D = cs.D;
    ca.r = cs.r;
    ca.s = cs.s;
    ca.LU = cs.LU;
    ca.piv = cs.piv;
    ca.XB = cs.XB;
    ca.xr = cs.xr;
    ca.S = cs.S;
    ca.t = cs.t;
    ca.status = cs.status;
    ca.tc_mode = tc_mode;
    if ((e = launch_condense(4, ca, st)) != cudaSuccess) return e;
    (hfr::count_launch(), k_class_scatter<<<cnt, 256, 0, st>>>(list + base, off, nA, nT, cs, (float*)LU, piv,
                                                                (float*)XB, xr, (float*)S, t));
    (hfr::count_launch(), k_class_status<<<1, 1, 0, st>>>(cs.status, list + base, 0, cnt, status));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t class_scratch_init_status(void* scratch, cudaStream_t st) {
  const int init[2] = {0, 0x7fffffff};
  cudaError_t e = cudaMemcpyAsync(scratch, init, sizeof(init), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

cudaError_t launch_condense_uneven(int prec_bytes, int n, const int* nA, const int* nT, const void* A, const void* B,
                                   const void* C, const void* D, const double* r, const double* s, void* LU, int* piv,
                                   void* XB, double* xr, void* S, double* t, int* status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  UnevenTables tb;
  if (uneven_tables(prec_bytes, n, nA, nT, &tb) != 0) return cudaErrorInvalidValue;
  void* dbuf = nullptr;
  cudaError_t e = cudaMallocAsync(&dbuf, uneven_dev_bytes(tb), st);
  if (e != cudaSuccess) return e;
  UnevenDev dv;
  e = uneven_upload(tb, dbuf, &dv, st);
  if (e == cudaSuccess)
    e = launch_condense_uneven_dev(prec_bytes, dv, A, B, C, D, r, s, LU, piv, XB, xr, S, t, status, st);
  // the host tables must outlive their copies; the work buffer is freed in stream order
  cudaStreamSynchronize(st);
  cudaFreeAsync(dbuf, st);
  cudaStreamSynchronize(st);
  return e;
}

// y = A^{-1} b = (PA)^{-1} (P b), in place on b.  One warp per element; lane owns rows
// lane + 32 q; the stored transpose makes each step a coalesced row read.
constexpr int INV_SLOTS = 5;  // nA <= 160
template <typename T>
__global__ void k_inv_apply(int Eim, int nA, const T* __restrict__ AinvT, const int* __restrict__ piv,
                            double* __restrict__ b) {
  // arithmetic in the block precision T: the result is a correction, T-accurate is enough
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= Eim) return;
  const T* W = AinvT + (size_t)k * nA * nA;
  const int* pv = piv + (size_t)k * nA;
  double* bk = b + (size_t)k * nA;
  T pb[INV_SLOTS], y[INV_SLOTS];
#pragma unroll
  for (int q = 0; q < INV_SLOTS; ++q) {
    const int j = lane + 32 * q;
    pb[q] = j < nA ? T(bk[pv[j]]) : T(0);  // (P b)_j
    y[q] = T(0);
  }
#pragma unroll
  for (int q = 0; q < INV_SLOTS; ++q) {
    if (32 * q >= nA) break;
    for (int jj = 0; jj < 32; ++jj) {
      const int j = 32 * q + jj;
      if (j >= nA) break;
      const T bj = __shfl_sync(0xffffffffu, pb[q], jj);
#pragma unroll
      for (int qq = 0; qq < INV_SLOTS; ++qq) {
        const int c = lane + 32 * qq;
        if (c < nA) y[qq] += W[(size_t)j * nA + c] * bj;
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < INV_SLOTS; ++q) {
    const int c = lane + 32 * q;
    if (c < nA) bk[c] = double(y[q]);
  }
}

// ---------------------------------------------------------------- LU kernel (FP64 path)
// LU with partial pivoting (full-row interchanges) of A applied to [B | r] in shared memory,
// then back substitution: X = A^{-1}[B | r] with nA^3/3 + nA^2 (nT+1) multiply-adds, ~25 % fewer
// than Gauss-Jordan, which is what counts where the FP64 pipe is the roof.  Keeps LU + piv.
constexpr int LU_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(LU_THREADS) k_condense_lu(const __grid_constant__ CondArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nA = a.nA, nT = a.nT, ldx = nT + 1;
  const int k = blockIdx.x;
  const int tid = threadIdx.x;
  const int rows2 = nA > nT ? nA : nT;
  T* sA = reinterpret_cast<T*>(smem_raw);  // rows2 x nA (A, later C)
  T* sX = sA + (size_t)rows2 * nA;          // nA x (nT + 1)
  __shared__ int s_piv;
  __shared__ int s_bad;
  const T* gA = reinterpret_cast<const T*>(a.A) + (size_t)k * nA * nA;
  const T* gB = reinterpret_cast<const T*>(a.B) + (size_t)k * nA * nT;
  const T* gC = reinterpret_cast<const T*>(a.C) + (size_t)k * nT * nA;
  const T* gD = reinterpret_cast<const T*>(a.D) + (size_t)k * nT * nT;
  for (int i = tid; i < nA * nA; i += LU_THREADS) sA[i] = gA[i];
  for (int i = tid; i < nA * ldx; i += LU_THREADS) {
    const int r = i / ldx, c = i % ldx;
    sX[i] = c < nT ? gB[(size_t)r * nT + c] : T(a.r[(size_t)k * nA + r]);
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  int* piv = a.piv + (size_t)k * nA;
  for (int c = 0; c < nA; ++c) {
    if (tid < 32) {
      T best = T(-1);
      int bi = c;
      for (int i = c + tid; i < nA; i += 32) {
        T v = tabs(sA[i * nA + c]);
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        T ov = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (tid == 0) {
        s_piv = bi;
        piv[c] = bi;
        if (!(best > T(0)) || best != best) s_bad = 1;
      }
    }
    __syncthreads();
    const int p = s_piv;
    if (p != c) {
      for (int j = tid; j < nA; j += LU_THREADS) {
        T t0 = sA[c * nA + j];
        sA[c * nA + j] = sA[p * nA + j];
        sA[p * nA + j] = t0;
      }
      for (int j = tid; j < ldx; j += LU_THREADS) {
        T t0 = sX[c * ldx + j];
        sX[c * ldx + j] = sX[p * ldx + j];
        sX[p * ldx + j] = t0;
      }
    }
    __syncthreads();
    const T pv = sA[c * nA + c];
    const T inv = pv != T(0) ? T(1) / pv : T(0);
    for (int i = c + 1 + tid; i < nA; i += LU_THREADS) sA[i * nA + c] *= inv;
    __syncthreads();
    const int nr = nA - c - 1;
    const int ncA = nA - c - 1;
    const int ncols = ncA + ldx;
    for (int it = tid; it < nr * ncols; it += LU_THREADS) {
      const int i = c + 1 + it / ncols;
      const int jj = it % ncols;
      const T l = sA[i * nA + c];
      if (jj < ncA) {
        const int j = c + 1 + jj;
        sA[i * nA + j] -= l * sA[c * nA + j];
      } else {
        const int j = jj - ncA;
        sX[i * ldx + j] -= l * sX[c * ldx + j];
      }
    }
    __syncthreads();
  }
  // back substitution with U
  for (int c = nA - 1; c >= 0; --c) {
    const T pv = sA[c * nA + c];
    const T inv = pv != T(0) ? T(1) / pv : T(0);
    for (int j = tid; j < ldx; j += LU_THREADS) sX[c * ldx + j] *= inv;
    __syncthreads();
    for (int it = tid; it < c * ldx; it += LU_THREADS) {
      const int i = it / ldx, j = it % ldx;
      sX[i * ldx + j] -= sA[i * nA + c] * sX[c * ldx + j];
    }
    __syncthreads();
  }
  if (tid == 0 && s_bad) {
    atomicOr(a.status, DEV_ERR_SINGULAR);
    atomicMin(a.status + 1, k);
  }
  // outputs: LU, X_B, x_r
  T* gLU = reinterpret_cast<T*>(a.LU) + (size_t)k * nA * nA;
  T* gXB = reinterpret_cast<T*>(a.XB) + (size_t)k * nA * nT;
  for (int i = tid; i < nA * nA; i += LU_THREADS) gLU[i] = sA[i];
  for (int i = tid; i < nA * ldx; i += LU_THREADS) {
    const int r = i / ldx, c = i % ldx;
    if (c < nT)
      gXB[(size_t)r * nT + c] = sX[i];
    else
      a.xr[(size_t)k * nA + r] = double(sX[i]);
  }
  __syncthreads();
  // C into the freed A region, then S = D - C X_B and t = s - C x_r
  for (int i = tid; i < nT * nA; i += LU_THREADS) sA[i] = gC[i];
  __syncthreads();
  T* gS = reinterpret_cast<T*>(a.S) + (size_t)k * nT * nT;
  for (int it = tid; it < nT * ldx; it += LU_THREADS) {
    const int i = it / ldx, j = it % ldx;
    T acc = T(0);
    for (int l = 0; l < nA; ++l) acc += sA[i * nA + l] * sX[l * ldx + j];
    if (j < nT)
      gS[(size_t)i * nT + j] = gD[(size_t)i * nT + j] - acc;
    else
      a.t[(size_t)k * nT + i] = a.s[(size_t)k * nT + i] - double(acc);
  }
}

// x = A^{-1} b with stored LU factors and row interchanges (FP64 path), in place on b.
// One warp per element; x distributed over lanes (row i in lane i % 32, slot i / 32).
template <typename T>
__global__ void k_lu_solve(int Eim, int nA, const T* __restrict__ LU, const int* __restrict__ piv,
                           double* __restrict__ b) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= Eim) return;
  const T* L = LU + (size_t)k * nA * nA;
  const int* pv = piv + (size_t)k * nA;
  double* bk = b + (size_t)k * nA;
  double x[INV_SLOTS];
#pragma unroll
  for (int q = 0; q < INV_SLOTS; ++q) {
    const int i = lane + 32 * q;
    x[q] = i < nA ? bk[i] : 0.0;
  }
  for (int c = 0; c < nA; ++c) {  // row interchanges in order
    const int p = pv[c];
    if (p == c) continue;
    const int qc = c >> 5, lc = c & 31, qp = p >> 5, lp = p & 31;
    double vc = 0.0, vp = 0.0;
#pragma unroll
    for (int q = 0; q < INV_SLOTS; ++q) {
      const double tc = __shfl_sync(0xffffffffu, x[q], lc);
      const double tp = __shfl_sync(0xffffffffu, x[q], lp);
      if (q == qc) vc = tc;
      if (q == qp) vp = tp;
    }
#pragma unroll
    for (int q = 0; q < INV_SLOTS; ++q) {
      if (q == qc && lane == lc) x[q] = vp;
      if (q == qp && lane == lp) x[q] = vc;
    }
  }
  for (int c = 0; c < nA - 1; ++c) {  // unit lower
    const int qc = c >> 5, lc = c & 31;
    double xc = 0.0;
#pragma unroll
    for (int q = 0; q < INV_SLOTS; ++q) {
      const double t = __shfl_sync(0xffffffffu, x[q], lc);
      if (q == qc) xc = t;
    }
#pragma unroll
    for (int q = 0; q < INV_SLOTS; ++q) {
      const int i = lane + 32 * q;
      if (i > c && i < nA) x[q] -= double(L[(size_t)i * nA + c]) * xc;
    }
  }
  for (int c = nA - 1; c >= 0; --c) {  // upper
    const int qc = c >> 5, lc = c & 31;
    const double d = double(L[(size_t)c * nA + c]);
#pragma unroll
    for (int q = 0; q < INV_SLOTS; ++q)
      if (q == qc && lane == lc) x[q] = x[q] / d;
    double xc = 0.0;
#pragma unroll
    for (int q = 0; q < INV_SLOTS; ++q) {
      const double t = __shfl_sync(0xffffffffu, x[q], lc);
      if (q == qc) xc = t;
    }
#pragma unroll
    for (int q = 0; q < INV_SLOTS; ++q) {
      const int i = lane + 32 * q;
      if (i < c) x[q] -= double(L[(size_t)i * nA + c]) * xc;
    }
  }
#pragma unroll
  for (int q = 0; q < INV_SLOTS; ++q) {
    const int i = lane + 32 * q;
    if (i < nA) bk[i] = x[q];
  }
}

template <typename T, int NA, int NT>
static cudaError_t cond_reg(const CondArgs& a, cudaStream_t st) {
  const size_t smem = GJShape<T, NA, NT>::SMEM;
  cudaError_t err = cudaFuncSetAttribute(k_condense_reg<T, NA, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  (hfr::count_launch(), k_condense_reg<T, NA, NT><<<a.Eim, GJ_THREADS, smem, st>>>(a));
  return cudaGetLastError();
}

template <typename T>
static cudaError_t cond_global_uniform(const CondArgs& a, cudaStream_t st) {
  UnevenArgs ua{0, nullptr, nullptr, nullptr, nullptr, a.A, a.B, a.C, a.D, a.r, a.s, a.LU, a.piv, a.XB, a.xr, a.S, a.t,
                a.status, 0};
  int dev = 0, nsm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  (void)nsm;
  return big::condense_big<T>(ua, nullptr, a.Eim, a.nA, a.nT, a.nA, a.nT, st);
}

template <typename T>
static cudaError_t cond_smem(const CondArgs& a, cudaStream_t st) {
  const size_t smem = smem_elem_bytes(sizeof(T), a.nA, a.nT);
  if (smem > 227 * 1024) return cond_global_uniform<T>(a, st);  // LU factors and pivots
  cudaError_t err = cudaFuncSetAttribute(k_condense_smem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  (hfr::count_launch(), k_condense_smem<T><<<a.Eim, GJS_THREADS, smem, st>>>(a));
  return cudaGetLastError();
}

// part 0: the factorisation (or the whole condensation where it is one kernel); part 1: the
// products of the two-kernel FP32 path (nothing elsewhere)
template <typename T>
static cudaError_t cond_dispatch(const CondArgs& a, cudaStream_t st, int part) {
  if (a.Eim == 0) return cudaSuccess;
  const int nA = a.nA, nT = a.nT;
  if (sizeof(T) == 4) {
    if (nA == 64 && nT == 64) return cond_two_kernel<64, 64>(a, st, part);
    if (nA == 36 && nT == 48) return cond_two_kernel<36, 48>(a, st, part);
    if (nA == 100 && nT == 80) return cond_two_kernel<100, 80>(a, st, part);
  }
  if (part != 0) return cudaSuccess;
  if (nA == 9 && nT == 12) return cond_reg<T, 9, 12>(a, st);
  if (nA == 16 && nT == 16) return cond_reg<T, 16, 16>(a, st);
  if (nA == 36 && nT == 48) return cond_reg<T, 36, 48>(a, st);
  if (nA == 64 && nT == 64) return cond_reg<T, 64, 64>(a, st);
  if (nA == 100 && nT == 80) return cond_reg<T, 100, 80>(a, st);
  return cond_smem<T>(a, st);
}

template <typename T>
static cudaError_t cond_lu(const CondArgs& a, cudaStream_t st) {
  const int rows2 = a.nA > a.nT ? a.nA : a.nT;
  size_t smem = sizeof(T) * ((size_t)rows2 * a.nA + (size_t)a.nA * (a.nT + 1));
  if (smem > 227 * 1024) return cond_dispatch<T>(a, st, 0);
  cudaError_t err = cudaFuncSetAttribute(k_condense_lu<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (a.Eim == 0) return cudaSuccess;
  (hfr::count_launch(), k_condense_lu<T><<<a.Eim, LU_THREADS, smem, st>>>(a));
  return cudaGetLastError();
}

// FP64: LU factors (fewest FP64 operations); FP32: in-place Gauss-Jordan (register tiles).
int condense_tc_available(int prec_bytes, int nA, int nT) {
  return prec_bytes == 4 && ((nA == 100 && nT == 80) || (nA == 64 && nT == 64) || (nA == 36 && nT == 48)) ? 2 : 0;
}

static bool lu_fits_smem(int prec_bytes, int nA, int nT) {
  const int rows2 = nA > nT ? nA : nT;
  return prec_bytes == 8 && sizeof(double) * ((size_t)rows2 * nA + (size_t)nA * (nT + 1)) <= 227 * 1024;
}
static bool reg_shape(int nA, int nT) {
  return (nA == 9 && nT == 12) || (nA == 16 && nT == 16) || (nA == 36 && nT == 48) || (nA == 64 && nT == 64) ||
         (nA == 100 && nT == 80);
}
// the condensation of this shape runs the global-memory kernel (LU factors, not an inverse)
static bool needs_global(int prec_bytes, int nA, int nT) {
  return !lu_fits_smem(prec_bytes, nA, nT) && !condense_tc_available(prec_bytes, nA, nT) && !reg_shape(nA, nT) &&
         smem_elem_bytes((size_t)prec_bytes, nA, nT) > 227 * 1024;
}

bool condense_uses_lu(int prec_bytes, int nA, int nT) {
  return lu_fits_smem(prec_bytes, nA, nT) || needs_global(prec_bytes, nA, nT);
}

bool condense_feasible(int prec_bytes, int nA, int nT) {
  return nA >= 1 && nT >= 1 && nA <= 32 * INV_SLOTS && nT <= 16384 && (prec_bytes == 4 || prec_bytes == 8);
}

cudaError_t launch_condense_part(int prec_bytes, const CondArgs& a, cudaStream_t st, int part) {
  if (lu_fits_smem(prec_bytes, a.nA, a.nT)) return part == 0 ? cond_lu<double>(a, st) : cudaSuccess;
  return prec_bytes == 8 ? cond_dispatch<double>(a, st, part) : cond_dispatch<float>(a, st, part);
}

cudaError_t launch_condense(int prec_bytes, const CondArgs& a, cudaStream_t st) {
  cudaError_t e = launch_condense_part(prec_bytes, a, st, 0);
  if (e != cudaSuccess) return e;
  return launch_condense_part(prec_bytes, a, st, 1);
}

cudaError_t launch_lu_solve(int prec_bytes, int Eim, int nA, int nT_of_last, const void* LU, const int* piv,
                            double* b, cudaStream_t st) {
  if (Eim == 0) return cudaSuccess;
  if (nA > 32 * INV_SLOTS) return cudaErrorInvalidValue;
  const int threads = 128;
  const int grid = (Eim * 32 + threads - 1) / threads;
  if (condense_uses_lu(prec_bytes, nA, nT_of_last) && prec_bytes == 8)
    (hfr::count_launch(), k_lu_solve<double><<<grid, threads, 0, st>>>(Eim, nA, (const double*)LU, piv, b));
  else if (condense_uses_lu(prec_bytes, nA, nT_of_last))
    (hfr::count_launch(), k_lu_solve<float><<<grid, threads, 0, st>>>(Eim, nA, (const float*)LU, piv, b));
  else if (prec_bytes == 8)
    (hfr::count_launch(), k_inv_apply<double><<<grid, threads, 0, st>>>(Eim, nA, (const double*)LU, piv, b));
  else
    (hfr::count_launch(), k_inv_apply<float><<<grid, threads, 0, st>>>(Eim, nA, (const float*)LU, piv, b));
  return cudaGetLastError();
}

}  // namespace hfr
