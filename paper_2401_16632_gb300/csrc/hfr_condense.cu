// Static condensation of the hybridized Newton system (Pereira & Vermeire, arXiv 2401.16632,
// Sec. 3.2): per implicit element k,
//     X = A_k^{-1} [B_k | r_k]          (LU with partial pivoting, largest |a|, lowest row on ties)
//     S_k = D_k - C_k X_B,  t_k = s_k - C_k x_r          (elemental L^k and t^k)
// One CTA per element; A and [B | r] are eliminated together in shared memory, the LU factors
// and pivots are kept for later solves.  T = double (plain) or float (mixed precision).
#include "hfr_internal.h"

namespace hfr {

constexpr int COND_THREADS = 256;

template <typename T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

template <typename T>
__global__ void __launch_bounds__(COND_THREADS) k_condense(const __grid_constant__ CondArgs a) {
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
  for (int i = tid; i < nA * nA; i += COND_THREADS) sA[i] = gA[i];
  for (int i = tid; i < nA * ldx; i += COND_THREADS) {
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
      for (int j = tid; j < nA; j += COND_THREADS) {
        T t0 = sA[c * nA + j];
        sA[c * nA + j] = sA[p * nA + j];
        sA[p * nA + j] = t0;
      }
      for (int j = tid; j < ldx; j += COND_THREADS) {
        T t0 = sX[c * ldx + j];
        sX[c * ldx + j] = sX[p * ldx + j];
        sX[p * ldx + j] = t0;
      }
    }
    __syncthreads();
    const T pv = sA[c * nA + c];
    const T inv = pv != T(0) ? T(1) / pv : T(0);
    for (int i = c + 1 + tid; i < nA; i += COND_THREADS) sA[i * nA + c] *= inv;
    __syncthreads();
    const int nr = nA - c - 1;
    const int ncA = nA - c - 1;
    const int ncols = ncA + ldx;
    for (int it = tid; it < nr * ncols; it += COND_THREADS) {
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
    for (int j = tid; j < ldx; j += COND_THREADS) sX[c * ldx + j] *= inv;
    __syncthreads();
    for (int it = tid; it < c * ldx; it += COND_THREADS) {
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
  for (int i = tid; i < nA * nA; i += COND_THREADS) gLU[i] = sA[i];
  for (int i = tid; i < nA * ldx; i += COND_THREADS) {
    const int r = i / ldx, c = i % ldx;
    if (c < nT)
      gXB[(size_t)r * nT + c] = sX[i];
    else
      a.xr[(size_t)k * nA + r] = double(sX[i]);
  }
  __syncthreads();
  // C into the freed A region, then S = D - C X_B and t = s - C x_r
  for (int i = tid; i < nT * nA; i += COND_THREADS) sA[i] = gC[i];
  __syncthreads();
  T* gS = reinterpret_cast<T*>(a.S) + (size_t)k * nT * nT;
  for (int it = tid; it < nT * ldx; it += COND_THREADS) {
    const int i = it / ldx, j = it % ldx;
    T acc = T(0);
    for (int l = 0; l < nA; ++l) acc += sA[i * nA + l] * sX[l * ldx + j];
    if (j < nT)
      gS[(size_t)i * nT + j] = gD[(size_t)i * nT + j] - acc;
    else
      a.t[(size_t)k * nT + i] = a.s[(size_t)k * nT + i] - double(acc);
  }
}

// x = A^{-1} b with the stored LU factors (row interchanges recorded in piv), in place on b.
template <typename T>
__global__ void k_lu_solve(int Eim, int nA, const T* __restrict__ LU, const int* __restrict__ piv,
                           double* __restrict__ b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* x = reinterpret_cast<double*>(smem_raw);
  const int k = blockIdx.x;
  if (k >= Eim) return;
  const T* L = LU + (size_t)k * nA * nA;
  const int* pv = piv + (size_t)k * nA;
  double* bk = b + (size_t)k * nA;
  for (int i = threadIdx.x; i < nA; i += blockDim.x) x[i] = bk[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < nA; ++c) {
      const int p = pv[c];
      if (p != c) {
        double t0 = x[c];
        x[c] = x[p];
        x[p] = t0;
      }
    }
  }
  __syncthreads();
  // forward (unit lower), one warp cooperating per column
  for (int c = 0; c < nA; ++c) {
    const double xc = x[c];
    for (int i = c + 1 + threadIdx.x; i < nA; i += blockDim.x) x[i] -= double(L[(size_t)i * nA + c]) * xc;
    __syncthreads();
  }
  for (int c = nA - 1; c >= 0; --c) {
    if (threadIdx.x == 0) x[c] /= double(L[(size_t)c * nA + c]);
    __syncthreads();
    const double xc = x[c];
    for (int i = threadIdx.x; i < c; i += blockDim.x) x[i] -= double(L[(size_t)i * nA + c]) * xc;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < nA; i += blockDim.x) bk[i] = x[i];
}

template <typename T>
static cudaError_t cond_impl(const CondArgs& a, cudaStream_t st) {
  const int rows2 = a.nA > a.nT ? a.nA : a.nT;
  size_t smem = sizeof(T) * ((size_t)rows2 * a.nA + (size_t)a.nA * (a.nT + 1));
  cudaError_t err = cudaFuncSetAttribute(k_condense<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (a.Eim == 0) return cudaSuccess;
  (hfr::count_launch(), k_condense<T><<<a.Eim, COND_THREADS, smem, st>>>(a));
  return cudaGetLastError();
}

cudaError_t launch_condense(int prec_bytes, const CondArgs& a, cudaStream_t st) {
  return prec_bytes == 8 ? cond_impl<double>(a, st) : cond_impl<float>(a, st);
}

cudaError_t launch_lu_solve(int prec_bytes, int Eim, int nA, const void* LU, const int* piv, double* b,
                            cudaStream_t st) {
  if (Eim == 0) return cudaSuccess;
  size_t smem = sizeof(double) * nA;
  if (prec_bytes == 8)
    (hfr::count_launch(), k_lu_solve<double><<<Eim, 64, smem, st>>>(Eim, nA, (const double*)LU, piv, b));
  else
    (hfr::count_launch(), k_lu_solve<float><<<Eim, 64, smem, st>>>(Eim, nA, (const float*)LU, piv, b));
  return cudaGetLastError();
}

}  // namespace hfr
