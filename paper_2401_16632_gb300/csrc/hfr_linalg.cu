// Trace-system operators (Pereira & Vermeire, arXiv 2401.16632, Sec. 3.2, eqs. assembly,
// assembly2, localproblems) and FP64 Krylov vector kernels.
//
// L is never assembled: y = L x = sum_k scatter(S_k gather_k(x)) is evaluated face by face.
// Trace face f has the two row blocks of the S_k of its neighbours; one warp per face gathers
// both neighbours' trace unknowns and reduces both row blocks, so every S_k row is read once
// per product and no atomics are needed (deterministic).
#include "hfr_internal.h"

namespace hfr {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// y = L x.  One warp per trace face, split into four groups of eight lanes; each group takes
// whole rows of the face's two row blocks (one per neighbour), the eight lanes of a group read
// consecutive columns, and a 3-step shuffle reduces the row.  Row i of the output is reduced by
// group i % 4 over both sides, so no cross-group accumulation is needed.  nT <= 96, bs <= 32.
constexpr int MV_CT = 12;  // columns per lane: nT / 8 <= 12
template <typename T>
__global__ void __launch_bounds__(256) k_trace_matvec(const __grid_constant__ TraceArgs a, const double* __restrict__ x,
                                                      double* __restrict__ y, const int* gate, int gj) {
  if (gate && *gate >= 0 && gj >= *gate) return;
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= a.ntrace) return;
  const int bs = a.n * a.nv, nT = a.nT;
  const int grp = lane >> 3, g8 = lane & 7;
  const T* S = reinterpret_cast<const T*>(a.S);
  int es[2], fs[2];
  T xv[2][MV_CT];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    es[side] = a.sides[t * 4 + side * 2];
    fs[side] = a.sides[t * 4 + side * 2 + 1];
#pragma unroll
    for (int c = 0; c < MV_CT; ++c) {
      const int l = g8 + 8 * c;
      T v = T(0);
      if (es[side] >= 0 && l < nT) {
        const int fp = l / bs;
        const int tf = a.tr_of_c[es[side] * 4 + fp];
        if (tf >= 0) v = T(x[(size_t)tf * bs + (l - fp * bs)]);
      }
      xv[side][c] = v;
    }
  }
  for (int i = grp; i < bs; i += 4) {
    T acc = T(0);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      if (es[side] < 0) continue;
      const T* row = S + ((size_t)es[side] * nT + (size_t)fs[side] * bs + i) * nT;
#pragma unroll
      for (int c = 0; c < MV_CT; ++c) {
        const int l = g8 + 8 * c;
        if (l < nT) acc += row[l] * xv[side][c];
      }
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (g8 == 0) y[(size_t)t * bs + i] = double(acc);
  }
}

// Same product with the shape fixed at compile time: every row of both row blocks is loaded up
// front (rows i = grp + 4u), so the loads of a face are all in flight before the reductions.
template <typename T, int NT, int BS>
__global__ void __launch_bounds__(256) k_trace_matvec_fixed(const __grid_constant__ TraceArgs a,
                                                            const double* __restrict__ x,
                                                            const float* __restrict__ x32, double* __restrict__ y,
                                                            const int* gate, int gj) {
  constexpr int CT = (NT + 7) / 8, RU = (BS + 3) / 4;
  if (gate && *gate >= 0 && gj >= *gate) return;
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= a.ntrace) return;
  const int grp = lane >> 3, g8 = lane & 7;
  const T* S = reinterpret_cast<const T*>(a.S);
  int es[2], fs[2];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    es[side] = a.sides[t * 4 + side * 2];
    fs[side] = a.sides[t * 4 + side * 2 + 1];
  }
  T sv[2][RU][CT];
#pragma unroll
  for (int side = 0; side < 2; ++side)
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int i = grp + 4 * u;
      const bool ok = es[side] >= 0 && i < BS;
      const T* row = S + ((size_t)(ok ? es[side] : 0) * NT + (size_t)(ok ? fs[side] : 0) * BS + (ok ? i : 0)) * NT;
#pragma unroll
      for (int c = 0; c < CT; ++c) {
        const int l = g8 + 8 * c;
        sv[side][u][c] = (ok && l < NT) ? row[l] : T(0);
      }
    }
  T xv[2][CT];
#pragma unroll
  for (int side = 0; side < 2; ++side)
#pragma unroll
    for (int c = 0; c < CT; ++c) {
      const int l = g8 + 8 * c;
      T v = T(0);
      if (es[side] >= 0 && l < NT) {
        const int fp = l / BS;
        const int tf = a.tr_of_c[es[side] * 4 + fp];
        if (tf >= 0) {
          const size_t ix = (size_t)tf * BS + (l - fp * BS);
          v = x32 ? T(x32[ix]) : T(x[ix]);
        }
      }
      xv[side][c] = v;
    }
#pragma unroll
  for (int u = 0; u < RU; ++u) {
    const int i = grp + 4 * u;
    T acc = T(0);
#pragma unroll
    for (int side = 0; side < 2; ++side)
#pragma unroll
      for (int c = 0; c < CT; ++c) acc += sv[side][u][c] * xv[side][c];
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (g8 == 0 && i < BS) y[(size_t)t * BS + i] = double(acc);
  }
}

// P_f = sum of both sides' diagonal face blocks of S_k, inverted in place by Gauss-Jordan with
// partial pivoting (pivot bookkeeping only, as in the condensation) in the block precision T.
// One warp per face, the bs x bs block in shared memory; Pinv_f = (P_f)^{-1} stored row-major.
constexpr int PB_WARPS = 4;
template <typename T>
__global__ void k_precond_build(const __grid_constant__ TraceArgs a, T* __restrict__ Pinv, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * PB_WARPS + wid;
  const int bs = a.n * a.nv, nT = a.nT;
  T* M = reinterpret_cast<T*>(smem_raw) + (size_t)wid * (bs * bs + 3 * 32);
  T* pr = M + bs * bs;
  int* ipiv = reinterpret_cast<int*>(pr + 32);  // physical row -> step
  int* pivs = ipiv + 32;                        // step -> physical row
  if (t >= a.ntrace) return;
  const T* S = reinterpret_cast<const T*>(a.S);
  for (int i = lane; i < bs * bs; i += 32) {
    const int r = i / bs, c = i % bs;
    T v = T(0);
    for (int side = 0; side < 2; ++side) {
      const int e = a.sides[t * 4 + side * 2], f = a.sides[t * 4 + side * 2 + 1];
      if (e >= 0) v += S[((size_t)e * nT + f * bs + r) * nT + f * bs + c];
    }
    M[i] = v;
  }
  __syncwarp();
  bool used = false, bad = false;  // lane r < bs: row r already a pivot
  for (int c = 0; c < bs; ++c) {
    T best = T(-1);
    int p = 0x7fffffff;
    if (lane < bs && !used) {
      const T v = M[lane * bs + c];
      best = v < T(0) ? -v : v;
      p = lane;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int op = __shfl_xor_sync(0xffffffffu, p, o);
      if (ob > best || (ob == best && op < p)) { best = ob; p = op; }
    }
    if (p >= bs) p = c;  // no candidate compared (NaN column): any row, flagged singular
    if (!(best > T(0))) bad = true;
    if (lane == p) used = true;
    if (lane == 0) {
      ipiv[p] = c;
      pivs[c] = p;
    }
    const T pv = M[p * bs + c];
    const T inv = pv != T(0) ? T(1) / pv : T(0);
    const T f = lane < bs ? M[lane * bs + c] : T(0);
    if (lane < bs) pr[lane] = lane == c ? inv : M[p * bs + lane] * inv;
    __syncwarp();
    for (int i = 0; i < bs; ++i) {
      const T fi = __shfl_sync(0xffffffffu, f, i);
      if (lane < bs) {
        const T pj = pr[lane];
        if (i == p)
          M[i * bs + lane] = pj;
        else
          M[i * bs + lane] = (lane == c ? T(0) : M[i * bs + lane]) - fi * pj;
      }
    }
    __syncwarp();
  }
  if (bad && lane == 0) atomicOr(status, DEV_ERR_SINGULAR);
  __syncwarp();
  // physical row r holds row ipiv[r] of (P P_f)^{-1}; (P_f)^{-1} = (P P_f)^{-1} P, i.e.
  // (P_f)^{-1}[ipiv[r]][pivs[c]] = M[r][c]
  for (int i = lane; i < bs * bs; i += 32) {
    const int r = i / bs, c = i % bs;
    Pinv[(size_t)t * bs * bs + (size_t)ipiv[r] * bs + pivs[c]] = M[i];
  }
  __syncwarp();
}

// The same inverse with the block in registers: one row per lane, W = 16 (bs <= 16, two faces per
// warp) or 32 lanes per face, cycling columns (every step shifts the rows left by one and appends
// the new column of the inverse, so the pivot column is always the first register and the bs
// steps unroll into one straight-line body), rows kept unnormalised (one division per row at the
// end).  Pivot: largest |a| among rows not yet used (ties: lowest row), by a butterfly over the
// lanes of the face; the pivot row reaches every lane by shuffles.
template <typename T, int BS>
__global__ void __launch_bounds__(128) k_precond_build_reg(const __grid_constant__ TraceArgs a, T* __restrict__ Pinv,
                                                           int* status) {
  constexpr int W = BS <= 16 ? 16 : 32;
  constexpr int FPW = 32 / W;
  const int lane = threadIdx.x & 31;
  const int sub = lane / W, r = lane % W;
  const int t = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * FPW + sub;
  const bool live = t < a.ntrace;
  const bool row_ok = live && r < BS;
  const int nT = a.nT;
  const T* S = reinterpret_cast<const T*>(a.S);
  T m[BS];
#pragma unroll
  for (int c = 0; c < BS; ++c) m[c] = T(0);
  if (row_ok) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int e = a.sides[t * 4 + side * 2], f = a.sides[t * 4 + side * 2 + 1];
      if (e >= 0) {
        const T* row = S + ((size_t)e * nT + (size_t)f * BS + r) * nT + (size_t)f * BS;
#pragma unroll
        for (int c = 0; c < BS; ++c) m[c] += __ldg(row + c);
      }
    }
  }
  bool used = !row_ok;
  int step = 0, pivs[BS];
  T dpiv = T(1);
  bool bad = false;
#pragma unroll
  for (int c = 0; c < BS; ++c) {
    // argmax of |m_0| over the unused rows of this face (largest magnitude, lowest row on ties)
    T best = used ? T(-1) : (m[0] < T(0) ? -m[0] : m[0]);
    int bi = used ? 0x7fffffff : r;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(0xffffffffu, best, o, W);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o, W);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    const int p = bi < BS ? bi : 0;
    pivs[c] = p;
    if (!(best > T(0))) bad = true;
    T prow[BS];
#pragma unroll
    for (int j = 0; j < BS; ++j) prow[j] = __shfl_sync(0xffffffffu, m[j], p, W);
    const bool isp = r == p;
    const T pinv = prow[0] != T(0) ? T(1) / prow[0] : T(0);
    const T fct = isp ? T(0) : m[0] * pinv;
    if (isp) {
      used = true;
      step = c;
      dpiv = m[0];
    }
#pragma unroll
    for (int j = 1; j < BS; ++j) m[j - 1] = m[j] - fct * prow[j];
    m[BS - 1] = (isp ? T(1) : T(0)) - fct;
  }
  if (bad && row_ok && r == 0) atomicOr(status, DEV_ERR_SINGULAR);
  if (!row_ok) return;
  // physical row r is row step of (P P_f)^{-1}; (P_f)^{-1}[step][pivs[c]] = m_c / pivot
  const T sc = dpiv != T(0) ? T(1) / dpiv : T(0);
  T* out = Pinv + (size_t)t * BS * BS + (size_t)step * BS;
#pragma unroll
  for (int c = 0; c < BS; ++c) out[pivs[c]] = m[c] * sc;
}

// y_f = Pinv_f x_f, one warp per face, lane = row.  With `hn` (GMRES), x is first normalised in
// place, x <- x / *hn (the new Krylov vector), before it is preconditioned.
template <typename T>
__global__ void k_precond_apply(const __grid_constant__ TraceArgs a, const T* __restrict__ Pinv,
                                double* __restrict__ x, double* __restrict__ y, const int* gate, int gj,
                                const double* inv_h, float* __restrict__ y32) {
  if (gate && *gate >= 0 && gj >= *gate) return;
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= a.ntrace) return;
  const int bs = a.n * a.nv;
  const T* P = Pinv + (size_t)t * bs * bs;
  double xd = lane < bs ? x[(size_t)t * bs + lane] : 0.0;
  if (inv_h) {
    xd *= *inv_h;
    if (lane < bs) x[(size_t)t * bs + lane] = xd;
  }
  const T xv = T(xd);
  T acc = T(0);
  for (int j = 0; j < bs; ++j) {
    const T xj = __shfl_sync(0xffffffffu, xv, j);
    if (lane < bs) acc += P[lane * bs + j] * xj;
  }
  if (lane < bs) {
    y[(size_t)t * bs + lane] = double(acc);
    if (y32) y32[(size_t)t * bs + lane] = float(acc);
  }
}

// global trace right-hand side t = sum_k scatter(t_k)
__global__ void k_assemble_t(const __grid_constant__ TraceArgs a, const double* __restrict__ te,
                             double* __restrict__ tg) {
  const int bs = a.n * a.nv;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.ntrace * bs) return;
  const int t = i / bs, kk = i % bs;
  double s = 0.0;
  for (int side = 0; side < 2; ++side) {
    const int e = a.sides[t * 4 + side * 2], f = a.sides[t * 4 + side * 2 + 1];
    if (e >= 0) s += te[(size_t)e * a.nT + f * bs + kk];
  }
  tg[i] = s;
}

// du_k = x_r - X_B du^_k: BE_EPB elements per CTA, one thread per row of X_B (the row read as
// VW-wide vectors, all of a thread's loads in flight together), du^_k gathered into shared
// memory once per element.
constexpr int BE_EPB = 4;
template <typename T, int VW>
__global__ void k_backsolve(const __grid_constant__ TraceArgs a, int Eim, int nA, const T* __restrict__ XB,
                            const double* __restrict__ xr, const double* __restrict__ duhat,
                            double* __restrict__ du) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int bs = a.n * a.nv, nT = a.nT;
  const int ld = (nT + 3) & ~3;
  T* xv_all = reinterpret_cast<T*>(smem_raw);
  const int per = blockDim.x / BE_EPB;  // threads per element (>= nA)
  const int g = threadIdx.x / per, i = threadIdx.x % per;
  const int k = blockIdx.x * BE_EPB + g;
  T* xv = xv_all + (size_t)g * ld;
  if (k < Eim) {
    for (int l = i; l < nT; l += per) {
      const int fp = l / bs;
      const int tf = a.tr_of_c[k * 4 + fp];
      xv[l] = tf >= 0 ? T(duhat[(size_t)tf * bs + (l - fp * bs)]) : T(0);
    }
  }
  __syncthreads();
  if (k >= Eim || i >= nA) return;
  const T* X = XB + ((size_t)k * nA + i) * nT;
  T p0 = T(0), p1 = T(0);
  if constexpr (VW == 4) {
#pragma unroll 8
    for (int l = 0; l < nT; l += 8) {
      const float4 x0 = __ldg(reinterpret_cast<const float4*>(X + l));
      const float4 v0 = *reinterpret_cast<const float4*>(xv + l);
      p0 += x0.x * v0.x + x0.y * v0.y + x0.z * v0.z + x0.w * v0.w;
      if (l + 4 < nT) {
        const float4 x1 = __ldg(reinterpret_cast<const float4*>(X + l + 4));
        const float4 v1 = *reinterpret_cast<const float4*>(xv + l + 4);
        p1 += x1.x * v1.x + x1.y * v1.y + x1.z * v1.z + x1.w * v1.w;
      }
    }
  } else {
    for (int l = 0; l < nT; l += 2) {
      p0 += X[l] * xv[l];
      if (l + 1 < nT) p1 += X[l + 1] * xv[l + 1];
    }
  }
  du[(size_t)k * nA + i] = xr[(size_t)k * nA + i] - double(p0 + p1);
}

// t_k = s_k - C_k x_r per element (the right-hand side of the condensed system for a new r with
// unchanged blocks): one CTA per element, x_r staged in shared memory, one warp per row of C_k
// with the lanes on consecutive columns.
template <typename T>
__global__ void k_rhs_condense(int Eim, int nA, int nT, const T* __restrict__ C, const double* __restrict__ xr,
                               const double* __restrict__ s, double* __restrict__ t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xv = reinterpret_cast<T*>(smem_raw);
  const int k = blockIdx.x;
  if (k >= Eim) return;
  for (int i = threadIdx.x; i < nA; i += blockDim.x) xv[i] = T(xr[(size_t)k * nA + i]);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const T* Ck = C + (size_t)k * nT * nA;
  for (int j = warp; j < nT; j += nw) {
    T p = T(0);
    for (int i = lane; i < nA; i += 32) p += Ck[(size_t)j * nA + i] * xv[i];
    p = warp_sum(p);
    if (lane == 0) t[(size_t)k * nT + j] = s[(size_t)k * nT + j] - double(p);
  }
}

cudaError_t launch_rhs_condense(int prec_bytes, int Eim, int nA, int nT, const void* C, const double* xr,
                                const double* s, double* t, cudaStream_t st) {
  if (Eim == 0) return cudaSuccess;
  if (prec_bytes == 8)
    (hfr::count_launch(), k_rhs_condense<double><<<Eim, 128, sizeof(double) * nA, st>>>(Eim, nA, nT, (const double*)C, xr, s, t));
  else
    (hfr::count_launch(), k_rhs_condense<float><<<Eim, 128, sizeof(float) * nA, st>>>(Eim, nA, nT, (const float*)C, xr, s, t));
  return cudaGetLastError();
}

cudaError_t launch_trace_matvec(int prec_bytes, const TraceArgs& a, const double* x, double* y, cudaStream_t st,
                                const int* gate, int gj, const float* x32) {
  if (a.ntrace == 0) return cudaSuccess;
  const int threads = 256;
  const int grid = (a.ntrace * 32 + threads - 1) / threads;
  const int bs = a.n * a.nv;
#define HFR_MV_FIXED(T_, NT_, BS_)                                                                       \
  if (a.nT == NT_ && bs == BS_) {                                                                        \
    (hfr::count_launch(), k_trace_matvec_fixed<T_, NT_, BS_><<<grid, threads, 0, st>>>(a, x, x32, y, gate, gj)); \
    return cudaGetLastError();                                                                           \
  }
  if (prec_bytes == 4) {
    HFR_MV_FIXED(float, 64, 16)
    HFR_MV_FIXED(float, 80, 20)
    HFR_MV_FIXED(float, 48, 12)
  } else {
    HFR_MV_FIXED(double, 64, 16)
    HFR_MV_FIXED(double, 80, 20)
    HFR_MV_FIXED(double, 48, 12)
  }
#undef HFR_MV_FIXED
  if (prec_bytes == 8)
    (hfr::count_launch(), k_trace_matvec<double><<<grid, threads, 0, st>>>(a, x, y, gate, gj));
  else
    (hfr::count_launch(), k_trace_matvec<float><<<grid, threads, 0, st>>>(a, x, y, gate, gj));
  return cudaGetLastError();
}

cudaError_t launch_precond_build(int prec_bytes, const TraceArgs& a, double* Pinv, int* status, cudaStream_t st) {
  if (a.ntrace == 0) return cudaSuccess;
  const int bs = a.n * a.nv;
  if (bs > 32) return cudaErrorInvalidValue;
#define HFR_PB(BS_)                                                                                         \
  if (bs == BS_) {                                                                                          \
    constexpr int FPW = BS_ <= 16 ? 2 : 1;                                                                  \
    const int grid = (a.ntrace + 4 * FPW - 1) / (4 * FPW);                                                  \
    if (prec_bytes == 8)                                                                                    \
      (hfr::count_launch(), k_precond_build_reg<double, BS_><<<grid, 128, 0, st>>>(a, Pinv, status));     \
    else                                                                                                    \
      (hfr::count_launch(), k_precond_build_reg<float, BS_><<<grid, 128, 0, st>>>(a, reinterpret_cast<float*>(Pinv), status)); \
    return cudaGetLastError();                                                                              \
  }
  HFR_PB(16)
  HFR_PB(12)
  HFR_PB(20)
#undef HFR_PB
  const int grid = (a.ntrace + PB_WARPS - 1) / PB_WARPS;
  if (prec_bytes == 8) {
    const size_t smem = sizeof(double) * (bs * bs + 3 * 32) * PB_WARPS;
    (hfr::count_launch(), k_precond_build<double><<<grid, 32 * PB_WARPS, smem, st>>>(a, Pinv, status));
  } else {
    const size_t smem = sizeof(float) * (bs * bs + 3 * 32) * PB_WARPS;
    (hfr::count_launch(), k_precond_build<float><<<grid, 32 * PB_WARPS, smem, st>>>(a, reinterpret_cast<float*>(Pinv), status));
  }
  return cudaGetLastError();
}

cudaError_t launch_precond_apply(int prec_bytes, const TraceArgs& a, const double* Pinv, double* x, double* y,
                                 cudaStream_t st, const int* gate, int gj, const double* inv_h, float* y32) {
  if (a.ntrace == 0) return cudaSuccess;
  const int threads = 256;
  const int grid = (a.ntrace * 32 + threads - 1) / threads;
  if (prec_bytes == 8)
    (hfr::count_launch(), k_precond_apply<double><<<grid, threads, 0, st>>>(a, Pinv, x, y, gate, gj, inv_h, y32));
  else
    (hfr::count_launch(), k_precond_apply<float><<<grid, threads, 0, st>>>(a, reinterpret_cast<const float*>(Pinv), x, y, gate, gj, inv_h, y32));
  return cudaGetLastError();
}

cudaError_t launch_assemble_t(const TraceArgs& a, const double* te, double* t, cudaStream_t st) {
  const int total = a.ntrace * a.n * a.nv;
  if (total == 0) return cudaSuccess;
  (hfr::count_launch(), k_assemble_t<<<(total + 255) / 256, 256, 0, st>>>(a, te, t));
  return cudaGetLastError();
}

cudaError_t launch_backsolve(int prec_bytes, const TraceArgs& a, int Eim, int nA, const void* XB, const double* xr,
                             const double* duhat, double* du, cudaStream_t st) {
  if (Eim == 0) return cudaSuccess;
  const int per = (nA + 31) & ~31;
  const int threads = per * BE_EPB;
  if (threads > 1024) return cudaErrorInvalidValue;
  const int grid = (Eim + BE_EPB - 1) / BE_EPB;
  const int ld = (a.nT + 3) & ~3;
  if (prec_bytes == 8)
    (hfr::count_launch(), k_backsolve<double, 1><<<grid, threads, sizeof(double) * ld * BE_EPB, st>>>(a, Eim, nA, (const double*)XB, xr, duhat, du));
  else if (a.nT % 8 == 0)
    (hfr::count_launch(), k_backsolve<float, 4><<<grid, threads, sizeof(float) * ld * BE_EPB, st>>>(a, Eim, nA, (const float*)XB, xr, duhat, du));
  else
    (hfr::count_launch(), k_backsolve<float, 1><<<grid, threads, sizeof(float) * ld * BE_EPB, st>>>(a, Eim, nA, (const float*)XB, xr, duhat, du));
  return cudaGetLastError();
}

}  // namespace hfr
