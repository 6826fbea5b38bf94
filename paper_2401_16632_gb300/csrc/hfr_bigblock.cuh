// Condensation of element blocks too large for one CTA's shared memory (FP64 p = 5 quadrilaterals,
// hexahedra: nA = 320, nT = 480), as a sequence of batched kernels over all such elements:
//   1. blocked right-looking LU with partial pivoting of A in place, panel by panel of LB columns:
//      the panel (all its rows) factorised in shared memory by one CTA per element (largest |a|,
//      lowest row on ties), its row interchanges applied to the columns left and right of it and
//      the block row right of it solved with the panel's unit lower triangle (same kernel); then
//      the trailing matrix updated by the batched GEMM;
//   2-3. X = A^{-1} P B: one CTA per block of 32 columns of one element, the block whole in shared
//      memory (permuted columns of B in, forward and back substitution by factor panels staged in
//      shared memory, X out once); where the block does not fit: the row interchanges applied to
//      the right-hand sides, then forward / back substitution blocked by NB rows (a small
//      triangular solve of the diagonal block, the rest of the rows updated by a batched GEMM);
//   4. S = D - C X_B by the same batched GEMM;
//   5. t = s - C x_r with FP64 accumulation (one CTA per element); x_r is the right-hand side's
//      column of the column-block solve, or, on the blocked path, A^{-1} r by FP64 substitution.
// The batched GEMM is a register-tiled CUDA-core kernel: 128 x 128 output tiles in FP32 (64 x 64 in
// FP64), 256 threads with 8 x 8 (4 x 4) outputs each, K staged through two shared-memory buffers 8
// at a time; arithmetic in the block precision T.  Included by hfr_condense.cu (uses UnevenArgs and DEV_ERR_*).
#pragma once

// FP32 batched GEMMs on the tensor cores (1) or the CUDA cores (0): a build flag for timing
#ifndef HFR_BIG_GEMM_TC
#define HFR_BIG_GEMM_TC 1
#endif

namespace hfr {
namespace big {

constexpr int NB = 32;       // rows per diagonal block of the triangular solves
constexpr int BT = 256;      // threads per CTA
// LU panel width: the panel of up to 1024 rows stays in shared memory (128 KB at most)
template <typename T>
__host__ __device__ constexpr int lu_panel() {
  return sizeof(T) == 8 ? 16 : 32;
}
template <typename T>
size_t lu_panel_smem(int max_nA) {
  return (size_t)max_nA * (lu_panel<T>() + 1) * sizeof(T);
}

// element of list position li: its id, five offsets and shape (tables, or one uniform shape)
struct Elem {
  int k, nA, nT;
  long long o[5];
};
__device__ __forceinline__ Elem elem_of(const UnevenArgs& a, const int* list, int li, int uni_nA, int uni_nT) {
  Elem e;
  e.k = list ? list[li] : li;
  if (uni_nA > 0) {
    e.nA = uni_nA;
    e.nT = uni_nT;
    e.o[0] = (long long)e.k * e.nA * e.nA;
    e.o[1] = (long long)e.k * e.nA * e.nT;
    e.o[2] = (long long)e.k * e.nT * e.nT;
    e.o[3] = (long long)e.k * e.nA;
    e.o[4] = (long long)e.k * e.nT;
  } else {
#pragma unroll
    for (int q = 0; q < 5; ++q) e.o[q] = a.off[5 * (size_t)e.k + q];
    e.nA = a.shape[2 * e.k];
    e.nT = a.shape[2 * e.k + 1];
  }
  return e;
}

// 1a. A copied into the LU slot (transposed when stored column-major); identity pivots
template <typename T>
__global__ void __launch_bounds__(BT) k_big_lu_init(const __grid_constant__ UnevenArgs a, const int* __restrict__ list,
                                                    int nlist, int uni_nA, int uni_nT) {
  for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
    const Elem E = elem_of(a, list, li, uni_nA, uni_nT);
    const int nA = E.nA;
    const T* A = reinterpret_cast<const T*>(a.A) + E.o[0];
    T* L = reinterpret_cast<T*>(a.LU) + E.o[0];
    const bool cm = a.colmajor != 0;
    for (size_t i = threadIdx.x; i < (size_t)nA * nA; i += BT) L[i] = cm ? A[(i % nA) * nA + i / nA] : A[i];
    for (int i = threadIdx.x; i < nA; i += BT) a.piv[E.o[3] + i] = i;
  }
}

// 1b. panel jb (columns [j0, j0 + w), rows [j0, nA)) of every element: factorised in shared memory
// (row stride LB + 1), pivots recorded as global rows, the interchanges applied to the other
// columns, and the block row U12 = L11^{-1} A12 right of the panel solved (one thread per column)
template <typename T>
__global__ void __launch_bounds__(BT) k_big_lu_panel(const __grid_constant__ UnevenArgs a, const int* __restrict__ list,
                                                     int nlist, int uni_nA, int uni_nT, int jb) {
  constexpr int LB = lu_panel<T>(), PS = LB + 1;
  extern __shared__ __align__(16) unsigned char lu_smem[];
  T* P = reinterpret_cast<T*>(lu_smem);
  __shared__ T rkey_v[BT / 32];
  __shared__ int rkey_i[BT / 32];
  __shared__ int spiv[LB];
  __shared__ int s_bad;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
    const Elem E = elem_of(a, list, li, uni_nA, uni_nT);
    const int nA = E.nA, j0 = jb * LB;
    if (j0 >= nA) continue;  // uniform over the CTA
    const int w = min(LB, nA - j0), R = nA - j0;
    T* L = reinterpret_cast<T*>(a.LU) + E.o[0];
    int* piv = a.piv + E.o[3];
    __syncthreads();  // the previous element's panel is free
    for (int i = tid; i < R * w; i += BT) {
      const int r = i / w, c = i % w;
      P[r * PS + c] = L[(size_t)(j0 + r) * nA + j0 + c];
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int c = 0; c < w; ++c) {
      T bv = T(-1);
      int bi = 0x7fffffff;
      for (int r = c + tid; r < R; r += BT) {
        const T v = fabs(P[r * PS + c]);
        if (v > bv || (v == bv && r < bi)) {
          bv = v;
          bi = r;
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, bv, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ov > bv || (ov == bv && oi < bi)) {
          bv = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        rkey_v[wid] = bv;
        rkey_i[wid] = bi;
      }
      __syncthreads();
      if (tid == 0) {
        T v = rkey_v[0];
        int ii = rkey_i[0];
        for (int q = 1; q < BT / 32; ++q)
          if (rkey_v[q] > v || (rkey_v[q] == v && rkey_i[q] < ii)) {
            v = rkey_v[q];
            ii = rkey_i[q];
          }
        spiv[c] = ii;
        if (!(v > T(0))) s_bad = 1;
      }
      __syncthreads();
      if (s_bad) break;
      const int pr = spiv[c];
      if (pr != c)
        for (int x = tid; x < w; x += BT) {
          const T u = P[c * PS + x];
          P[c * PS + x] = P[pr * PS + x];
          P[pr * PS + x] = u;
        }
      __syncthreads();
      const T inv = T(1) / P[c * PS + c];
      for (int r = c + 1 + tid; r < R; r += BT) {
        const T l = P[r * PS + c] * inv;
        P[r * PS + c] = l;
        for (int x = c + 1; x < w; ++x) P[r * PS + x] -= l * P[c * PS + x];
      }
      __syncthreads();
    }
    if (s_bad) {
      if (tid == 0) {
        atomicOr(a.status, DEV_ERR_SINGULAR);
        atomicMin(a.status + 1, E.k);
      }
      continue;  // the element's factors are left unfinished; its pivots stay in range
    }
    for (int i = tid; i < R * w; i += BT) {
      const int r = i / w, c = i % w;
      L[(size_t)(j0 + r) * nA + j0 + c] = P[r * PS + c];
    }
    for (int c = tid; c < w; c += BT) piv[j0 + c] = j0 + spiv[c];
    // the interchanges on the columns outside the panel; U12 on those right of it
    for (int col = tid; col < nA - w; col += BT) {
      const int cc = col < j0 ? col : col + w;
      for (int q = 0; q < w; ++q) {
        const int pr = spiv[q];
        if (pr != q) {
          const T u = L[(size_t)(j0 + q) * nA + cc];
          L[(size_t)(j0 + q) * nA + cc] = L[(size_t)(j0 + pr) * nA + cc];
          L[(size_t)(j0 + pr) * nA + cc] = u;
        }
      }
      if (cc >= j0 + w) {
        T x[LB];
#pragma unroll
        for (int q = 0; q < LB; ++q) {
          if (q < w) {
            T v = L[(size_t)(j0 + q) * nA + cc];
#pragma unroll
            for (int s2 = 0; s2 < q; ++s2) v -= P[q * PS + s2] * x[s2];
            x[q] = v;
            L[(size_t)(j0 + q) * nA + cc] = v;
          }
        }
      }
    }
  }
}

// 2. X = P B (rows in the order the interchanges leave them; B transposed when column-major)
template <typename T>
__global__ void __launch_bounds__(BT) k_big_rhs(const __grid_constant__ UnevenArgs a, const int* __restrict__ list,
                                                int nlist, int uni_nA, int uni_nT) {
  __shared__ int perm[1024], pvs[1024];
  for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
    const Elem E = elem_of(a, list, li, uni_nA, uni_nT);
    const int nA = E.nA, nT = E.nT;
    const T* B = reinterpret_cast<const T*>(a.B) + E.o[1];
    T* X = reinterpret_cast<T*>(a.XB) + E.o[1];
    const int* piv = a.piv + E.o[3];
    __syncthreads();
    for (int i = threadIdx.x; i < nA; i += BT) {
      pvs[i] = piv[i];
      perm[i] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int j = 0; j < nA; ++j) {
        const int p = pvs[j];
        if (p >= 0 && p < nA && p != j) {
          const int u = perm[j];
          perm[j] = perm[p];
          perm[p] = u;
        }
      }
    }
    __syncthreads();
    const bool cm = a.colmajor != 0;
    for (size_t i = threadIdx.x; i < (size_t)nA * nT; i += BT) {
      const int row = (int)(i / nT), col = (int)(i % nT), src = perm[row];
      X[i] = cm ? B[(size_t)col * nA + src] : B[(size_t)src * nT + col];
    }
  }
}

// 3a. diagonal block jb of the triangular solves: rows [r0, r1) of X, one thread per column
// (lower: unit lower factor, forward; upper: upper factor, backward)
template <typename T>
__global__ void __launch_bounds__(128) k_big_trsm_diag(const __grid_constant__ UnevenArgs a, const int* __restrict__ list,
                                                      int base, int nlist, int uni_nA, int uni_nT, int jb, int upper) {
  if ((int)blockIdx.y >= nlist) return;
  const int li = base + blockIdx.y;
  const Elem E = elem_of(a, list, li, uni_nA, uni_nT);
  const int nA = E.nA, nT = E.nT;
  const int r0 = jb * NB;
  if (r0 >= nA) return;
  const int r1 = min(nA, r0 + NB);
  const int col = blockIdx.x * 128 + threadIdx.x;
  if (col >= nT) return;
  const T* L = reinterpret_cast<const T*>(a.LU) + E.o[0];
  T* X = reinterpret_cast<T*>(a.XB) + E.o[1];
  T x[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) x[q] = (r0 + q < r1) ? X[(size_t)(r0 + q) * nT + col] : T(0);
  if (!upper) {
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      if (r0 + q >= r1) break;
#pragma unroll
      for (int c = 0; c < q; ++c) x[q] -= L[(size_t)(r0 + q) * nA + r0 + c] * x[c];
    }
  } else {
#pragma unroll
    for (int q = NB - 1; q >= 0; --q) {
      if (r0 + q >= r1) continue;
      T s = x[q];
#pragma unroll
      for (int c = q + 1; c < NB; ++c)
        if (r0 + c < r1) s -= L[(size_t)(r0 + q) * nA + r0 + c] * x[c];
      x[q] = s / L[(size_t)(r0 + q) * nA + r0 + q];
    }
  }
#pragma unroll
  for (int q = 0; q < NB; ++q)
    if (r0 + q < r1) X[(size_t)(r0 + q) * nT + col] = x[q];
}

// 2'-3'. X = A^{-1} P B for a block of SC columns per CTA, whole in shared memory: the permuted
// columns of B loaded once, forward substitution with the unit lower factor and back substitution
// with the upper factor by panels of SP pivots (the factor's panel staged in shared memory: an
// in-panel solve of SP steps, then one register-tiled update of every row outside the panel), X
// written once.  Replaces the row interchange copy and the blocked triangular solves when the two
// tiles fit shared memory.
constexpr int SC = 32;  // columns of X per CTA (the lanes of a warp)
constexpr int SP = 32;  // pivots per factor panel
template <typename T>
size_t solve_smem(int max_nA) {
  return ((size_t)max_nA * SC + (size_t)max_nA * SP) * sizeof(T) + (size_t)max_nA * sizeof(int);
}
// Lp[r][j] = L[r0 + r][p0 + j] for r < nrows, j < w (zero for w <= j < SP); SU loads per thread in
// flight before their stores.  A full panel (w = SP) of a factor whose rows start on 16-byte
// boundaries moves in 16-byte vectors: a quarter (FP32) of the dependent rounds of loads.
template <typename T>
__device__ __forceinline__ void solve_stage_panel(T* Lp, const T* L, int nA, int r0, int nrows, int p0, int w,
                                                  int tid) {
  constexpr int SU = 8;
  constexpr int V = 16 / sizeof(T);  // values per 16-byte vector
  using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  if (w == SP && nA % V == 0 && (reinterpret_cast<uintptr_t>(L) & 15) == 0) {
    // rows r0 .. r0 + nrows - 1 < nA, columns p0 .. p0 + SP - 1 < nA (full panel); p0 % SP == 0
    constexpr int VR = SP / V;  // vectors per panel row
    const int cnt = nrows * VR;
    for (int b = tid; b < cnt; b += BT * SU) {
      VT v[SU];
#pragma unroll
      for (int u = 0; u < SU; ++u) {
        const int idx = b + BT * u, r = idx / VR, q = idx % VR;
        if (idx < cnt) v[u] = *reinterpret_cast<const VT*>(L + (size_t)(r0 + r) * nA + p0 + q * V);
      }
#pragma unroll
      for (int u = 0; u < SU; ++u) {
        const int idx = b + BT * u;
        if (idx < cnt) *reinterpret_cast<VT*>(Lp + (size_t)(idx / VR) * SP + (idx % VR) * V) = v[u];
      }
    }
    return;
  }
  const int cnt = nrows * SP;
  for (int b = tid; b < cnt; b += BT * SU) {
    T v[SU];
#pragma unroll
    for (int u = 0; u < SU; ++u) {
      const int idx = b + BT * u, r = idx / SP, j = idx % SP;
      v[u] = (idx < cnt && j < w) ? L[(size_t)(r0 + r) * nA + p0 + j] : T(0);
    }
#pragma unroll
    for (int u = 0; u < SU; ++u)
      if (b + BT * u < cnt) Lp[b + BT * u] = v[u];
  }
}

// Xs rows [ra, rb) -= (factor panel rows, staged at Lp row r - lbase) x (solved panel rows of Xs,
// p0 .. p0 + w - 1): eight rows per warp pass, four pivots per step (one 16-byte broadcast of the
// factor per row, four values of the solved rows per lane); the factor panel is zero beyond w
template <typename T>
__device__ __forceinline__ void solve_update(T* Xs, const T* Lp, int p0, int w, int ra, int rb, int lbase, int lane,
                                             int wid) {
  constexpr int NW = BT / 32;
  for (int r0 = ra + 8 * wid; r0 < rb; r0 += 8 * NW) {
    T acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = T(0);
    for (int j = 0; j < w; j += 4) {
      T xv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[u] = j + u < w ? Xs[(p0 + j + u) * SC + lane] : T(0);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (r0 + q < rb) {
          const T* lr = Lp + (size_t)(r0 + q - lbase) * SP + j;  // 16-byte aligned (j % 4 == 0)
          if constexpr (sizeof(T) == 4) {
            const float4 l4 = *reinterpret_cast<const float4*>(lr);
            acc[q] += l4.x * xv[0] + l4.y * xv[1] + l4.z * xv[2] + l4.w * xv[3];
          } else {
            const double2 la = reinterpret_cast<const double2*>(lr)[0], lb = reinterpret_cast<const double2*>(lr)[1];
            acc[q] += la.x * xv[0] + la.y * xv[1] + lb.x * xv[2] + lb.y * xv[3];
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (r0 + q < rb) Xs[(r0 + q) * SC + lane] -= acc[q];
  }
}

template <typename T>
__global__ void __launch_bounds__(BT, 2) k_big_solve(const __grid_constant__ UnevenArgs a, const int* __restrict__ list,
                                                  int base, int nlist, int uni_nA, int uni_nT) {
  extern __shared__ __align__(16) unsigned char sv_smem[];
  if ((int)blockIdx.y >= nlist) return;
  const Elem E = elem_of(a, list, base + blockIdx.y, uni_nA, uni_nT);
  const int nA = E.nA, nT = E.nT, c0 = blockIdx.x * SC;
  if (c0 > nT) return;  // uniform over the CTA (column nT is r: x_r)
  T* Xs = reinterpret_cast<T*>(sv_smem);  // nA x SC
  T* Lp = Xs + (size_t)nA * SC;            // nA x SP: rows of the current factor panel
  int* perm = reinterpret_cast<int*>(Lp + (size_t)nA * SP);
  const T* L = reinterpret_cast<const T*>(a.LU) + E.o[0];
  const T* B = reinterpret_cast<const T*>(a.B) + E.o[1];
  T* X = reinterpret_cast<T*>(a.XB) + E.o[1];
  const int* piv = a.piv + E.o[3];
  const bool cm = a.colmajor != 0;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int NW = BT / 32;
  // rows in the order the interchanges leave them: the pivots staged in shared memory (the factor
  // panel's space, free until the forward sweep), then applied in sequence by one thread
  int* pvs = reinterpret_cast<int*>(Lp);
  for (int i = tid; i < nA; i += BT) {
    pvs[i] = piv[i];
    perm[i] = i;
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < nA; ++j) {
      const int p = pvs[j];
      if (p >= 0 && p < nA && p != j) {
        const int u = perm[j];
        perm[j] = perm[p];
        perm[p] = u;
      }
    }
  }
  __syncthreads();
  const int c = c0 + lane;
  const bool live = c < nT;
  const double* rv = a.r + E.o[3];
  // global loads in batches of SU per thread, all in flight before their shared-memory stores
  constexpr int SU = 8;
  for (int i0 = wid; i0 < nA; i0 += NW * SU) {
    T v[SU];
#pragma unroll
    for (int u = 0; u < SU; ++u) {
      const int i = i0 + NW * u;
      v[u] = T(0);
      if (i < nA) {
        const int src = perm[i];
        v[u] = live ? (cm ? B[(size_t)c * nA + src] : B[(size_t)src * nT + c]) : (c == nT ? T(rv[src]) : T(0));
      }
    }
#pragma unroll
    for (int u = 0; u < SU; ++u)
      if (i0 + NW * u < nA) Xs[(i0 + NW * u) * SC + lane] = v[u];
  }
  // ---- forward: unit lower factor, panels top to bottom
  for (int p0 = 0; p0 < nA; p0 += SP) {
    const int w = min(SP, nA - p0);
    __syncthreads();  // the previous panel's readers are done
    solve_stage_panel<T>(Lp, L, nA, p0, nA - p0, p0, w, tid);
    __syncthreads();
    if (wid == 0) {  // in-panel solve: one warp, lane = column, the panel's rows in registers
      T x[SP];
#pragma unroll
      for (int r = 0; r < SP; ++r) x[r] = r < w ? Xs[(p0 + r) * SC + lane] : T(0);
#pragma unroll
      for (int j = 0; j < SP; ++j)
#pragma unroll
        for (int r = j + 1; r < SP; ++r) x[r] -= Lp[r * SP + j] * x[j];  // zero beyond w
#pragma unroll
      for (int r = 0; r < SP; ++r)
        if (r < w) Xs[(p0 + r) * SC + lane] = x[r];
    }
    __syncthreads();
    // rows below the panel: X[r] -= L[r, panel] X[panel]
    solve_update<T>(Xs, Lp, p0, w, p0 + w, nA, p0, lane, wid);
  }
  // ---- backward: upper factor, panels bottom to top
  const int np = (nA + SP - 1) / SP;
  for (int pb = np - 1; pb >= 0; --pb) {
    const int p0 = pb * SP, w = min(SP, nA - p0);
    __syncthreads();
    solve_stage_panel<T>(Lp, L, nA, 0, p0 + w, p0, w, tid);
    __syncthreads();
    if (wid == 0) {
      T x[SP];
#pragma unroll
      for (int r = 0; r < SP; ++r) x[r] = r < w ? Xs[(p0 + r) * SC + lane] : T(0);
#pragma unroll
      for (int j = SP - 1; j >= 0; --j) {
        if (j < w) {
          x[j] = x[j] / Lp[(p0 + j) * SP + j];
#pragma unroll
          for (int r = 0; r < j; ++r) x[r] -= Lp[(p0 + r) * SP + j] * x[j];
        }
      }
#pragma unroll
      for (int r = 0; r < SP; ++r)
        if (r < w) Xs[(p0 + r) * SC + lane] = x[r];
    }
    __syncthreads();
    solve_update<T>(Xs, Lp, p0, w, 0, p0, 0, lane, wid);  // rows above the panel
  }
  __syncthreads();
  if (live)
    for (int i = wid; i < nA; i += NW) X[(size_t)i * nT + c] = Xs[i * SC + lane];
  else if (c == nT)
    for (int i = wid; i < nA; i += NW) a.xr[E.o[3] + i] = double(Xs[i * SC + lane]);
}

// 3b / 4. batched GEMM Out -= A B, per element:
//   phase 0: rows [r1, nA) of X -= L[r1:, r0:r1] X[r0:r1, :]     (forward, block jb)
//   phase 1: rows [0, r0) of X  -= L[:r0, r0:r1] X[r0:r1, :]     (backward, block jb)
//   phase 2: S = D - C X_B (C, D column-major when the blocks are)
//   phase 3: L[j1:, j1:] -= L[j1:, j0:j1] L[j0:j1, j1:]          (LU trailing update, panel jb)
// 16 x 16 threads, each with TM x TM outputs in two TM/2-wide halves of rows and of columns (so
// that its shared-memory operands are two 16-byte vectors per k), GKK values of k per stage, two
// shared-memory stages with the next stage's global values held in registers meanwhile.
template <typename T>
struct GemmCfg {
  static constexpr int TM = sizeof(T) == 8 ? 4 : 8;  // outputs per thread and dimension
  static constexpr int H = TM / 2;                   // one 16-byte vector
  static constexpr int BM = 16 * TM;                 // output tile (rows = columns)
  static constexpr int GKK = 8;                      // k per stage
  static constexpr int PAD = 16 / sizeof(T);
  static constexpr int LD = BM * GKK / BT;           // values of each operand a thread loads per stage
};
template <typename T>
__device__ __forceinline__ void gemm_vec_ld(const T* p, T (&v)[GemmCfg<T>::H]) {
  if constexpr (sizeof(T) == 8) {
    const double2 x = *reinterpret_cast<const double2*>(p);
    v[0] = x.x;
    v[1] = x.y;
  } else {
    const float4 x = *reinterpret_cast<const float4*>(p);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
  }
}
template <typename T>
__global__ void __launch_bounds__(BT) k_big_gemm(const __grid_constant__ UnevenArgs a, const int* __restrict__ list,
                                                 int base, int nlist, int uni_nA, int uni_nT, int phase, int jb) {
  using C = GemmCfg<T>;
  constexpr int TM = C::TM, H = C::H, BM = C::BM, GKK = C::GKK, LDN = C::LD;
  __shared__ __align__(16) T As[2][GKK][BM + C::PAD];  // [k][m]
  __shared__ __align__(16) T Bs[2][GKK][BM + C::PAD];  // [k][n]
  if ((int)blockIdx.z >= nlist) return;
  const int li = base + blockIdx.z;
  const Elem E = elem_of(a, list, li, uni_nA, uni_nT);
  const int nA = E.nA, nT = E.nT;
  const bool cm = a.colmajor != 0;
  int M, N, K, m_off = 0, k_off = 0, n_off = 0;
  T* L = reinterpret_cast<T*>(a.LU) + E.o[0];
  T* X = reinterpret_cast<T*>(a.XB) + E.o[1];
  const T* Cm = reinterpret_cast<const T*>(a.C) + E.o[1];
  const T* Dm = reinterpret_cast<const T*>(a.D) + E.o[2];
  T* S = reinterpret_cast<T*>(a.S) + E.o[2];
  if (phase == 0) {
    const int r0 = jb * NB, r1 = min(nA, r0 + NB);
    M = nA - r1;
    N = nT;
    K = r1 - r0;
    m_off = r1;
    k_off = r0;
  } else if (phase == 1) {
    const int r0 = jb * NB, r1 = min(nA, r0 + NB);
    M = r0;
    N = nT;
    K = r1 - r0;
    k_off = r0;
  } else if (phase == 2) {
    M = nT;
    N = nT;
    K = nA;
  } else {
    const int j0 = jb * lu_panel<T>(), j1 = min(nA, j0 + lu_panel<T>());
    M = nA - j1;
    N = nA - j1;
    K = j1 - j0;
    m_off = j1;
    n_off = j1;
    k_off = j0;
  }
  const int tm0 = blockIdx.y * BM, tn0 = blockIdx.x * BM;
  if (M <= 0 || K <= 0 || tm0 >= M || tn0 >= N) return;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  // operand A element (m, k) of the tile: k contiguous in memory except column-major C
  const bool a_mfast = phase == 2 && cm;
  auto lda = [&](int m, int k) -> T {
    if (m >= M || k >= K) return T(0);
    if (phase != 2) return L[(size_t)(m_off + m) * nA + k_off + k];
    return cm ? Cm[(size_t)k * nT + m] : Cm[(size_t)m * nA + k];
  };
  auto ldb = [&](int k, int n) -> T {
    if (n >= N || k >= K) return T(0);
    return phase == 3 ? L[(size_t)(k_off + k) * nA + n_off + n] : X[(size_t)(k_off + k) * nT + n];
  };
  // thread's load slots: A (m, k) with k fastest (or m fastest), B (k, n) with n fastest
  T ra[LDN], rb[LDN];
  auto gload = [&](int k0) {
#pragma unroll
    for (int q = 0; q < LDN; ++q) {
      const int idx = tid + q * BT;
      if (a_mfast)
        ra[q] = lda(tm0 + idx % BM, k0 + idx / BM);
      else
        ra[q] = lda(tm0 + idx / GKK, k0 + idx % GKK);
      rb[q] = ldb(k0 + idx / BM, tn0 + idx % BM);
    }
  };
  auto sstore = [&](int st) {
#pragma unroll
    for (int q = 0; q < LDN; ++q) {
      const int idx = tid + q * BT;
      if (a_mfast)
        As[st][idx / BM][idx % BM] = ra[q];
      else
        As[st][idx % GKK][idx / GKK] = ra[q];
      Bs[st][idx / BM][idx % BM] = rb[q];
    }
  };
  T acc[TM][TM];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc[i][j] = T(0);
  gload(0);
  sstore(0);
  __syncthreads();
  int st = 0;
  for (int k0 = 0; k0 < K; k0 += GKK) {
    const bool more = k0 + GKK < K;
    if (more) gload(k0 + GKK);
#pragma unroll
    for (int kk = 0; kk < GKK; ++kk) {
      T av[TM], bv[TM];
      gemm_vec_ld<T>(&As[st][kk][ty * H], *reinterpret_cast<T(*)[H]>(&av[0]));
      gemm_vec_ld<T>(&As[st][kk][BM / 2 + ty * H], *reinterpret_cast<T(*)[H]>(&av[H]));
      gemm_vec_ld<T>(&Bs[st][kk][tx * H], *reinterpret_cast<T(*)[H]>(&bv[0]));
      gemm_vec_ld<T>(&Bs[st][kk][BM / 2 + tx * H], *reinterpret_cast<T(*)[H]>(&bv[H]));
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) acc[i][j] += av[i] * bv[j];
    }
    if (more) {
      sstore(st ^ 1);
      __syncthreads();
      st ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = tm0 + (i < H ? ty * H + i : BM / 2 + ty * H + i - H);
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      const int n = tn0 + (j < H ? tx * H + j : BM / 2 + tx * H + j - H);
      if (n >= N) continue;
      if (phase <= 1) {
        X[(size_t)(m_off + m) * nT + n] -= acc[i][j];
      } else if (phase == 3) {
        L[(size_t)(m_off + m) * nA + n_off + n] -= acc[i][j];
      } else {
        const T d = cm ? Dm[(size_t)n * nT + m] : Dm[(size_t)m * nT + n];
        S[(size_t)m * nT + n] = d - acc[i][j];
      }
    }
  }
}

// 3b' / 4'. the same batched GEMMs for FP32 blocks on the tensor cores (tcgen05, 3xTF32: each
// operand split into a TF32 high part and the remainder, hi*hi + hi*lo + lo*hi accumulated in FP32
// in tensor memory).  One CTA per output tile of 256 rows (m) x 128 columns (n) of one element,
// computed transposed: the tensor-memory lanes hold the 128 columns n and its 256 FP32 columns the
// rows m, so that in the epilogue the 32 lanes of a warp read and write 32 consecutive n of one
// row (coalesced).  K runs in chunks of 32, staged K-major without swizzle (hfr_tc.cuh) in two
// shared-memory buffers, one mbarrier per buffer; the next chunk's global loads are in flight
// while the tensor core works on the current one.  Thread 0 issues the MMAs; in the epilogue warp
// w reads lanes 32 (w % 4).. and the column half w / 4 of the accumulator.
namespace btc {
constexpr int TM = 256, TN = 128, KC = 32, THREADS = 256;
constexpr uint32_t SBO = (KC / 4) * 128u + 16u;  // 8-row groups padded by 16 bytes
constexpr uint32_t N_BYTES = (TN / 8) * SBO;     // the n-rows operand (MMA A, 128 rows), hi or lo
constexpr uint32_t M_BYTES = (TM / 8) * SBO;     // the m-rows operand (MMA B, 256 rows), hi or lo
constexpr uint32_t STAGE = 2 * N_BYTES + 2 * M_BYTES;
constexpr uint32_t SMEM = 2 * STAGE + 64;
constexpr int A_PER = TM * KC / THREADS, B_PER = TN * KC / THREADS;  // values a thread stages per chunk
static_assert(SMEM <= 232448, "shared memory");
}  // namespace btc

__global__ void __launch_bounds__(btc::THREADS, 1) k_big_gemm_tc(const __grid_constant__ UnevenArgs a,
                                                                const int* __restrict__ list, int base, int nlist,
                                                                int uni_nA, int uni_nT, int phase, int jb) {
  using namespace tc;
  using namespace btc;
  extern __shared__ __align__(1024) unsigned char btc_smem[];
  if ((int)blockIdx.z >= nlist) return;
  const Elem E = elem_of(a, list, base + blockIdx.z, uni_nA, uni_nT);
  const int nA = E.nA, nT = E.nT;
  const bool cm = a.colmajor != 0;
  int M, N, K, m_off = 0, k_off = 0, n_off = 0;
  float* L = reinterpret_cast<float*>(a.LU) + E.o[0];
  float* X = reinterpret_cast<float*>(a.XB) + E.o[1];
  const float* Cm = reinterpret_cast<const float*>(a.C) + E.o[1];
  const float* Dm = reinterpret_cast<const float*>(a.D) + E.o[2];
  float* S = reinterpret_cast<float*>(a.S) + E.o[2];
  if (phase == 0) {
    const int r0 = jb * NB, r1 = min(nA, r0 + NB);
    M = nA - r1;
    N = nT;
    K = r1 - r0;
    m_off = r1;
    k_off = r0;
  } else if (phase == 1) {
    const int r0 = jb * NB, r1 = min(nA, r0 + NB);
    M = r0;
    N = nT;
    K = r1 - r0;
    k_off = r0;
  } else if (phase == 2) {
    M = nT;
    N = nT;
    K = nA;
  } else {
    const int j0 = jb * lu_panel<float>(), j1 = min(nA, j0 + lu_panel<float>());
    M = nA - j1;
    N = nA - j1;
    K = j1 - j0;
    m_off = j1;
    n_off = j1;
    k_off = j0;
  }
  const int tm0 = blockIdx.y * TM, tn0 = blockIdx.x * TN;
  if (M <= 0 || K <= 0 || tm0 >= M || tn0 >= N) return;  // uniform over the CTA
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(btc_smem + 2 * STAGE);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  if (t == 0) {
    mbar_init(smem_u32(mbar), 1);
    mbar_init(smem_u32(mbar + 1), 1);
  }
  if (w == 0) tmem_alloc(smem_u32(tslot), 256);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const bool a_mfast = phase == 2 && cm;  // A(m, k) contiguous in m (column-major C)
  // staging slots of this thread: A (m, k) with k fastest: rows (t >> 3) + 32 u, k 4 (t & 7) + e;
  // m fastest: row 32 w + lane, k = u; B (k, n): column t & 127, k (t >> 7) + 2 u
  float ra[A_PER], rb[B_PER];
  auto gload = [&](int k0) {
#pragma unroll
    for (int u = 0; u < A_PER; ++u) {
      const int m = tm0 + (a_mfast ? 32 * w + lane : (t >> 3) + 32 * (u >> 2));
      const int k = k0 + (a_mfast ? u : 4 * (t & 7) + (u & 3));
      float v = 0.f;
      if (m < M && k < K) {
        if (phase != 2)
          v = L[(size_t)(m_off + m) * nA + k_off + k];
        else
          v = cm ? Cm[(size_t)k * nT + m] : Cm[(size_t)m * nA + k];
      }
      ra[u] = v;
    }
#pragma unroll
    for (int u = 0; u < B_PER; ++u) {
      const int n = tn0 + (t & 127), k = k0 + (t >> 7) + 2 * u;
      float v = 0.f;
      if (n < N && k < K) v = phase == 3 ? L[(size_t)(k_off + k) * nA + n_off + n] : X[(size_t)(k_off + k) * nT + n];
      rb[u] = v;
    }
  };
  auto sstore = [&](int b) {
    unsigned char* Nhi = btc_smem + b * STAGE;
    unsigned char* Nlo = Nhi + N_BYTES;
    unsigned char* Mhi = Nlo + N_BYTES;
    unsigned char* Mlo = Mhi + M_BYTES;
    if (a_mfast) {
#pragma unroll
      for (int u = 0; u < A_PER; ++u) {
        float h, l;
        split_tf32(ra[u], h, l);
        const uint32_t o = kmajor_offset(32 * w + lane, u, SBO);
        *reinterpret_cast<float*>(Mhi + o) = h;
        *reinterpret_cast<float*>(Mlo + o) = l;
      }
    } else {
#pragma unroll
      for (int u = 0; u < A_PER; u += 4) {
        float h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_tf32(ra[u + e], h[e], l[e]);
        const uint32_t o = kmajor_offset((t >> 3) + 32 * (u >> 2), 4 * (t & 7), SBO);
        *reinterpret_cast<float4*>(Mhi + o) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(Mlo + o) = make_float4(l[0], l[1], l[2], l[3]);
      }
    }
#pragma unroll
    for (int u = 0; u < B_PER; ++u) {
      float h, l;
      split_tf32(rb[u], h, l);
      const uint32_t o = kmajor_offset(t & 127, (t >> 7) + 2 * u, SBO);
      *reinterpret_cast<float*>(Nhi + o) = h;
      *reinterpret_cast<float*>(Nlo + o) = l;
    }
  };
  const int nch = (K + KC - 1) / KC;
  const uint32_t idesc = idesc_tf32(TN, TM);  // M = 128 (n on the lanes), N = 256 (m)
  bool ok = true;
  gload(0);
  for (int c = 0; c < nch; ++c) {
    const int b = c & 1;
    if (c >= 2) {  // the MMAs of chunk c - 2 read this buffer
      ok = mbar_wait(smem_u32(mbar + b), (uint32_t)(((c - 2) >> 1) & 1), TIMEOUT_NS);
      if (__syncthreads_or(!ok)) {
        ok = false;
        break;
      }
      fence_after_sync();
    }
    sstore(b);
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    if (t == 0) {
      fence_after_sync();
      const uint32_t nh = smem_u32(btc_smem + b * STAGE), nl = nh + N_BYTES, mh = nl + N_BYTES, ml = mh + M_BYTES;
#pragma unroll 1
      for (int kk = 0; kk < KC / 8; ++kk) {
        const uint32_t off = (uint32_t)kk * 256u;  // two core matrices along k per instruction
        const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
        mma_tf32(tmem, desc_noswizzle(nh + off, 128, SBO), desc_noswizzle(mh + off, 128, SBO), idesc, acc);
        mma_tf32(tmem, desc_noswizzle(nh + off, 128, SBO), desc_noswizzle(ml + off, 128, SBO), idesc, 1u);
        mma_tf32(tmem, desc_noswizzle(nl + off, 128, SBO), desc_noswizzle(mh + off, 128, SBO), idesc, 1u);
      }
      mma_commit(smem_u32(mbar + b));
    }
    if (c + 1 < nch) gload((c + 1) * KC);
  }
  if (ok) {  // the last commit completes after every MMA before it
    ok = mbar_wait(smem_u32(mbar + ((nch - 1) & 1)), (uint32_t)(((nch - 1) >> 1) & 1), TIMEOUT_NS);
    ok = !__syncthreads_or(!ok);
  }
  fence_after_sync();
  if (ok) {
    const int q = w & 3, hh = w >> 2;
    const int n = tn0 + 32 * q + lane;
    const uint32_t tl = (uint32_t)(32 * q) << 16;
#pragma unroll 1
    for (int cc = 0; cc < 8; ++cc) {
      float v[16];
      const int m0 = tm0 + 128 * hh + 16 * cc;
      tmem_ld16(tmem + tl + (uint32_t)(128 * hh + 16 * cc), v);
      if (n >= N) continue;
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int m = m0 + u;
        if (m >= M) break;
        if (phase <= 1) {
          X[(size_t)(m_off + m) * nT + n] -= v[u];
        } else if (phase == 3) {
          L[(size_t)(m_off + m) * nA + n_off + n] -= v[u];
        } else {
          const float d = cm ? Dm[(size_t)n * nT + m] : Dm[(size_t)m * nT + n];
          S[(size_t)m * nT + n] = d - v[u];
        }
      }
    }
  } else if (t == 0) {
    atomicOr(a.status, DEV_ERR_TIMEOUT);
    // the MMAs in flight finish (bounded) before their tensor memory is released
    mbar_wait(smem_u32(mbar), 0, TIMEOUT_NS);
    mbar_wait(smem_u32(mbar + 1), 0, TIMEOUT_NS);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (w == 0) tmem_dealloc(tmem, 256);
}

// 5. t = s - C x_r; unless solved with X: x_r = A^{-1} r (interchanges, forward, backward; FP64)
template <typename T>
__global__ void __launch_bounds__(BT) k_big_xr(const __grid_constant__ UnevenArgs a, const int* __restrict__ list,
                                               int nlist, int uni_nA, int uni_nT, int solved) {
  __shared__ double y[1024];
  __shared__ int pvs[1024];
  for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
    const Elem E = elem_of(a, list, li, uni_nA, uni_nT);
    const int nA = E.nA, nT = E.nT;
    const T* L = reinterpret_cast<const T*>(a.LU) + E.o[0];
    const T* Cm = reinterpret_cast<const T*>(a.C) + E.o[1];
    const int* piv = a.piv + E.o[3];
    const double* r = a.r + E.o[3];
    double* xr = a.xr + E.o[3];
    const double* sv = a.s + E.o[4];
    double* t = a.t + E.o[4];
    const bool cm = a.colmajor != 0;
    __syncthreads();
    if (solved) {  // x_r came with X (the right-hand side's column of the column-block solve)
      for (int i = threadIdx.x; i < nA; i += BT) y[i] = xr[i];
      __syncthreads();
    }
    if (!solved) {
      for (int i = threadIdx.x; i < nA; i += BT) {
        y[i] = r[i];
        pvs[i] = piv[i];
      }
      __syncthreads();
      if (threadIdx.x == 0)
        for (int j = 0; j < nA; ++j) {
          const int p = pvs[j];
          if (p >= 0 && p < nA && p != j) {
            const double u = y[j];
            y[j] = y[p];
            y[p] = u;
          }
        }
      __syncthreads();
      for (int j = 0; j < nA; ++j) {  // unit lower
        const double yj = y[j];
        for (int i = j + 1 + threadIdx.x; i < nA; i += BT) y[i] -= (double)L[(size_t)i * nA + j] * yj;
        __syncthreads();
      }
      for (int j = nA - 1; j >= 0; --j) {  // upper
        if (threadIdx.x == 0) y[j] /= (double)L[(size_t)j * nA + j];
        __syncthreads();
        const double yj = y[j];
        for (int i = threadIdx.x; i < j; i += BT) y[i] -= (double)L[(size_t)i * nA + j] * yj;
        __syncthreads();
      }
    }
    if (!solved)
      for (int i = threadIdx.x; i < nA; i += BT) xr[i] = y[i];
    for (int row = threadIdx.x; row < nT; row += BT) {
      double acc = 0.0;
      for (int c = 0; c < nA; ++c) acc += (double)(cm ? Cm[(size_t)c * nT + row] : Cm[(size_t)row * nA + c]) * y[c];
      t[row] = sv[row] - acc;
    }
  }
}

// the whole sequence over nlist elements (list: table positions, or null with a uniform shape);
// max_nA / max_nT: the largest shape (grid extents)
template <typename T>
cudaError_t condense_big(const UnevenArgs& a, const int* list, int nlist, int uni_nA, int uni_nT, int max_nA,
                         int max_nT, cudaStream_t st) {
  if (nlist <= 0) return cudaSuccess;
  if (max_nA > 1024 || max_nT > 16384) return cudaErrorInvalidValue;
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid1 = nlist < 4 * nsm ? nlist : 4 * nsm;
  cudaError_t e;
  const size_t psm = lu_panel_smem<T>(max_nA);
  if ((e = cudaFuncSetAttribute(k_big_lu_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm)) !=
      cudaSuccess)
    return e;
  int occ = 1;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_big_lu_panel<T>, BT, psm)) != cudaSuccess) return e;
  const int gridp = nlist < occ * nsm ? nlist : (occ > 0 ? occ : 1) * nsm;
  (hfr::count_launch(), k_big_lu_init<T><<<grid1, BT, 0, st>>>(a, list, nlist, uni_nA, uni_nT));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const bool tcg = sizeof(T) == 4 && HFR_BIG_GEMM_TC;  // FP32 GEMMs on the tensor cores
  if (tcg && (e = cudaFuncSetAttribute(k_big_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)btc::SMEM)) != cudaSuccess)
    return e;
  // one batched GEMM phase over elements [base, base + cnt): rows x cols of the largest shape.  The
  // tensor cores take S = D - C X_B (K = nA); the K = 32 updates of the LU and the triangular
  // solves, bound by the read-modify-write of their outputs, stay on the CUDA cores (two CTAs per
  // SM against one of the tensor-core kernel: measured faster on hexahedra)
  auto gemm = [&](int base, int cnt, int rows, int cols, int phase, int jb) {
    if (tcg && phase == 2) {
      const dim3 g((cols + btc::TN - 1) / btc::TN, (rows + btc::TM - 1) / btc::TM, cnt);
      (hfr::count_launch(), k_big_gemm_tc<<<g, btc::THREADS, btc::SMEM, st>>>(a, list, base, cnt, uni_nA, uni_nT,
                                                                                 phase, jb));
    } else {
      constexpr int TB = GemmCfg<T>::BM;
      const dim3 g((cols + TB - 1) / TB, (rows + TB - 1) / TB, cnt);
      (hfr::count_launch(), k_big_gemm<T><<<g, BT, 0, st>>>(a, list, base, cnt, uni_nA, uni_nT, phase, jb));
    }
  };
  const int npan = (max_nA + lu_panel<T>() - 1) / lu_panel<T>();
  for (int jb = 0; jb < npan; ++jb) {
    (hfr::count_launch(), k_big_lu_panel<T><<<gridp, BT, psm, st>>>(a, list, nlist, uni_nA, uni_nT, jb));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (jb + 1 == npan) break;
    const int rest = max_nA - (jb + 1) * lu_panel<T>();
    for (int base = 0; base < nlist; base += 65535) {
      const int cnt = nlist - base < 65535 ? nlist - base : 65535;
      gemm(base, cnt, rest, rest, 3, jb);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // X = A^{-1} P B: column blocks whole in shared memory when they fit, else the interchange copy
  // and the blocked triangular solves
  const size_t ssm = solve_smem<T>(max_nA);
  const bool fused = ssm <= 227 * 1024 &&
                     cudaFuncSetAttribute(k_big_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm) ==
                         cudaSuccess;
  cudaGetLastError();
  if (!fused) {
    (hfr::count_launch(), k_big_rhs<T><<<grid1, BT, 0, st>>>(a, list, nlist, uni_nA, uni_nT));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  const int nblk = (max_nA + NB - 1) / NB;
  constexpr int CH = 65535;  // grid y / z extent per launch
  for (int base = 0; base < nlist; base += CH) {
    const int cnt = nlist - base < CH ? nlist - base : CH;
    if (fused) {
      const dim3 gv((max_nT + 1 + SC - 1) / SC, cnt);  // and the column of r
      (hfr::count_launch(), k_big_solve<T><<<gv, BT, ssm, st>>>(a, list, base, cnt, uni_nA, uni_nT));
    } else {
      const dim3 gd((max_nT + 127) / 128, cnt);
      for (int jb = 0; jb < nblk; ++jb) {
        (hfr::count_launch(), k_big_trsm_diag<T><<<gd, 128, 0, st>>>(a, list, base, cnt, uni_nA, uni_nT, jb, 0));
        if (jb + 1 < nblk) gemm(base, cnt, max_nA - (jb + 1) * NB, max_nT, 0, jb);
      }
      for (int jb = nblk - 1; jb >= 0; --jb) {
        (hfr::count_launch(), k_big_trsm_diag<T><<<gd, 128, 0, st>>>(a, list, base, cnt, uni_nA, uni_nT, jb, 1));
        if (jb > 0) gemm(base, cnt, jb * NB, max_nT, 1, jb);
      }
    }
    gemm(base, cnt, max_nT, max_nT, 2, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  (hfr::count_launch(), k_big_xr<T><<<grid1, BT, 0, st>>>(a, list, nlist, uni_nA, uni_nT, fused ? 1 : 0));
  return cudaGetLastError();
}

}  // namespace big
}  // namespace hfr
