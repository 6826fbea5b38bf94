// Condensation of element blocks too large for one CTA's shared memory (FP64 p = 5 quadrilaterals,
// hexahedra: nA = 320, nT = 480), as a sequence of batched kernels over all such elements:
//   1. LU with partial pivoting of A in place (one CTA per element, rank-1 updates in L2-resident
//      global memory; largest |a|, lowest row on ties);
//   2. X = P [B] (the row interchanges applied to the right-hand sides);
//   3. forward substitution with the unit lower factor and back substitution with the upper factor,
//      both blocked by NB rows: a small triangular solve of the diagonal block (one thread per
//      right-hand side column), then the rest of the rows updated by a batched GEMM;
//   4. S = D - C X_B by the same batched GEMM;
//   5. x_r = A^{-1} r and t = s - C x_r in FP64 arithmetic (one CTA per element).
// The batched GEMM is a register-tiled CUDA-core kernel: 64 x 64 output tiles, 256 threads with
// 4 x 4 outputs each, K staged through shared memory 16 at a time; arithmetic in the block
// precision T.  Included by hfr_condense.cu (uses UnevenArgs and DEV_ERR_*).
#pragma once

namespace hfr {
namespace big {

constexpr int NB = 32;       // rows per diagonal block of the triangular solves
constexpr int GT = 64;       // GEMM output tile
constexpr int GK = 16;       // GEMM K chunk
constexpr int BT = 256;      // threads per CTA

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

// 1. LU factors in the LU slot (A copied in, transposed when stored column-major), pivots
template <typename T>
__global__ void __launch_bounds__(BT) k_big_lu(const __grid_constant__ UnevenArgs a, const int* __restrict__ list,
                                               int nlist, int uni_nA, int uni_nT) {
  __shared__ T prow[1024];
  __shared__ double pkey_v[BT / 32];
  __shared__ int pkey_i[BT / 32];
  __shared__ int s_piv, s_bad;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
    const Elem E = elem_of(a, list, li, uni_nA, uni_nT);
    const int nA = E.nA;
    const T* A = reinterpret_cast<const T*>(a.A) + E.o[0];
    T* L = reinterpret_cast<T*>(a.LU) + E.o[0];
    int* piv = a.piv + E.o[3];
    const bool cm = a.colmajor != 0;
    for (size_t i = tid; i < (size_t)nA * nA; i += BT) L[i] = cm ? A[(i % nA) * nA + i / nA] : A[i];
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int j = 0; j < nA; ++j) {
      double bv = -1.0;
      int bi = 0x7fffffff;
      for (int i = j + tid; i < nA; i += BT) {
        const double v = fabs((double)L[(size_t)i * nA + j]);
        if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (lane == 0) { pkey_v[wid] = bv; pkey_i[wid] = bi; }
      __syncthreads();
      if (tid == 0) {
        double v = pkey_v[0];
        int ii = pkey_i[0];
        for (int q = 1; q < BT / 32; ++q)
          if (pkey_v[q] > v || (pkey_v[q] == v && pkey_i[q] < ii)) { v = pkey_v[q]; ii = pkey_i[q]; }
        s_piv = ii;
        piv[j] = ii;
        if (!(v > 0.0)) s_bad = 1;
      }
      __syncthreads();
      if (s_bad) break;
      const int pr = s_piv;
      if (pr != j)
        for (int c = tid; c < nA; c += BT) {
          const T u = L[(size_t)j * nA + c];
          L[(size_t)j * nA + c] = L[(size_t)pr * nA + c];
          L[(size_t)pr * nA + c] = u;
        }
      __syncthreads();
      const T inv = T(1) / L[(size_t)j * nA + j];
      const int ncol = nA - j - 1;  // <= 1024 (nA <= 1025)
      for (int c = tid; c < ncol; c += BT) prow[c] = L[(size_t)j * nA + j + 1 + c];
      __syncthreads();
      for (int i = j + 1 + wid; i < nA; i += BT / 32) {
        T* Li = L + (size_t)i * nA;
        const T l = Li[j] * inv;
        for (int c = lane; c < ncol; c += 32) Li[j + 1 + c] -= l * prow[c];
        __syncwarp();
        if (lane == 0) Li[j] = l;
      }
      __syncthreads();
    }
    if (s_bad && tid == 0) {
      atomicOr(a.status, DEV_ERR_SINGULAR);
      atomicMin(a.status + 1, E.k);
    }
    __syncthreads();
  }
}

// 2. X = P B (rows in the order the interchanges leave them; B transposed when column-major)
template <typename T>
__global__ void __launch_bounds__(BT) k_big_rhs(const __grid_constant__ UnevenArgs a, const int* __restrict__ list,
                                                int nlist, int uni_nA, int uni_nT) {
  __shared__ int perm[1024];
  for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
    const Elem E = elem_of(a, list, li, uni_nA, uni_nT);
    const int nA = E.nA, nT = E.nT;
    const T* B = reinterpret_cast<const T*>(a.B) + E.o[1];
    T* X = reinterpret_cast<T*>(a.XB) + E.o[1];
    const int* piv = a.piv + E.o[3];
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 0; i < nA; ++i) perm[i] = i;
      for (int j = 0; j < nA; ++j) {
        const int p = piv[j];
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

// 3b / 4. batched GEMM Out -= A B on 64 x 64 tiles:
//   phase 0: rows [r1, nA) of X -= L[r1:, r0:r1] X[r0:r1, :]     (forward, block jb)
//   phase 1: rows [0, r0) of X  -= L[:r0, r0:r1] X[r0:r1, :]     (backward, block jb)
//   phase 2: S = D - C X_B (C, D column-major when the blocks are)
template <typename T>
__global__ void __launch_bounds__(BT) k_big_gemm(const __grid_constant__ UnevenArgs a, const int* __restrict__ list,
                                                 int base, int nlist, int uni_nA, int uni_nT, int phase, int jb) {
  __shared__ T As[GK][GT + 4];  // [k][m]
  __shared__ T Bs[GK][GT];      // [k][n]
  if ((int)blockIdx.z >= nlist) return;
  const int li = base + blockIdx.z;
  const Elem E = elem_of(a, list, li, uni_nA, uni_nT);
  const int nA = E.nA, nT = E.nT;
  const bool cm = a.colmajor != 0;
  int M, N, K, m_off = 0, k_off = 0;
  const T* L = reinterpret_cast<const T*>(a.LU) + E.o[0];
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
    m_off = 0;
    k_off = r0;
  } else {
    M = nT;
    N = nT;
    K = nA;
  }
  const int tm0 = blockIdx.y * GT, tn0 = blockIdx.x * GT;
  if (M <= 0 || K <= 0 || tm0 >= M || tn0 >= N) return;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) acc[i][jj] = T(0);
  for (int k0 = 0; k0 < K; k0 += GK) {
    // A tile (64 rows m x 16 k) and B tile (16 k x 64 n)
    for (int idx = tid; idx < GT * GK; idx += BT) {
      const int mm = idx % GT, kk = idx / GT;
      const int m = tm0 + mm, k = k0 + kk;
      T v = T(0);
      if (m < M && k < K) {
        if (phase <= 1)
          v = L[(size_t)(m_off + m) * nA + k_off + k];
        else
          v = cm ? Cm[(size_t)k * nT + m] : Cm[(size_t)m * nA + k];
      }
      As[kk][mm] = v;
    }
    for (int idx = tid; idx < GT * GK; idx += BT) {
      const int nn = idx % GT, kk = idx / GT;
      const int n = tn0 + nn, k = k0 + kk;
      T v = T(0);
      if (n < N && k < K) v = X[(size_t)(k_off + k) * nT + n];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) bv[jj] = Bs[kk][tx + 16 * jj];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] += av[i] * bv[jj];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = tm0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int n = tn0 + tx + 16 * jj;
      if (n >= N) continue;
      if (phase <= 1) {
        X[(size_t)(m_off + m) * nT + n] -= acc[i][jj];
      } else {
        const T d = cm ? Dm[(size_t)n * nT + m] : Dm[(size_t)m * nT + n];
        S[(size_t)m * nT + n] = d - acc[i][jj];
      }
    }
  }
}

// 5. x_r = A^{-1} r (interchanges, forward, backward; FP64) and t = s - C x_r
template <typename T>
__global__ void __launch_bounds__(BT) k_big_xr(const __grid_constant__ UnevenArgs a, const int* __restrict__ list,
                                               int nlist, int uni_nA, int uni_nT) {
  __shared__ double y[1024];
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
    for (int i = threadIdx.x; i < nA; i += BT) y[i] = r[i];
    __syncthreads();
    if (threadIdx.x == 0)
      for (int j = 0; j < nA; ++j) {
        const int p = piv[j];
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
  (hfr::count_launch(), k_big_lu<T><<<grid1, BT, 0, st>>>(a, list, nlist, uni_nA, uni_nT));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  (hfr::count_launch(), k_big_rhs<T><<<grid1, BT, 0, st>>>(a, list, nlist, uni_nA, uni_nT));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int nblk = (max_nA + NB - 1) / NB;
  constexpr int CH = 65535;  // grid y / z extent per launch
  for (int base = 0; base < nlist; base += CH) {
    const int cnt = nlist - base < CH ? nlist - base : CH;
    const dim3 gd((max_nT + 127) / 128, cnt);
    const dim3 gg((max_nT + GT - 1) / GT, (max_nA + GT - 1) / GT, cnt);
    for (int jb = 0; jb < nblk; ++jb) {
      (hfr::count_launch(), k_big_trsm_diag<T><<<gd, 128, 0, st>>>(a, list, base, cnt, uni_nA, uni_nT, jb, 0));
      if (jb + 1 < nblk)
        (hfr::count_launch(), k_big_gemm<T><<<gg, BT, 0, st>>>(a, list, base, cnt, uni_nA, uni_nT, 0, jb));
    }
    for (int jb = nblk - 1; jb >= 0; --jb) {
      (hfr::count_launch(), k_big_trsm_diag<T><<<gd, 128, 0, st>>>(a, list, base, cnt, uni_nA, uni_nT, jb, 1));
      if (jb > 0) (hfr::count_launch(), k_big_gemm<T><<<gg, BT, 0, st>>>(a, list, base, cnt, uni_nA, uni_nT, 1, jb));
    }
    const dim3 gs((max_nT + GT - 1) / GT, (max_nT + GT - 1) / GT, cnt);
    (hfr::count_launch(), k_big_gemm<T><<<gs, BT, 0, st>>>(a, list, base, cnt, uni_nA, uni_nT, 2, 0));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  (hfr::count_launch(), k_big_xr<T><<<grid1, BT, 0, st>>>(a, list, nlist, uni_nA, uni_nT));
  return cudaGetLastError();
}

}  // namespace big
}  // namespace hfr
