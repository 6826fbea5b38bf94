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

// y = L x.  One warp per trace face; nT <= 96, bs = n nv <= 32.
template <typename T>
__global__ void k_trace_matvec(const __grid_constant__ TraceArgs a, const double* __restrict__ x,
                               double* __restrict__ y, const int* gate, int gj) {
  if (gate && *gate >= 0 && gj >= *gate) return;
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= a.ntrace) return;
  const int bs = a.n * a.nv, nT = a.nT;
  const T* S = reinterpret_cast<const T*>(a.S);
  T acc = T(0);
  for (int side = 0; side < 2; ++side) {
    const int e = a.sides[t * 4 + side * 2], f = a.sides[t * 4 + side * 2 + 1];
    if (e < 0) continue;
    T xv[3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      const int l = lane + 32 * kk;
      T v = T(0);
      if (l < nT) {
        const int fp = l / bs;
        const int tf = a.tr_of_c[e * 4 + fp];
        if (tf >= 0) v = T(x[(size_t)tf * bs + (l - fp * bs)]);
      }
      xv[kk] = v;
    }
    const T* Sr = S + ((size_t)e * nT + (size_t)f * bs) * nT;
    for (int i = 0; i < bs; ++i) {
      T p = T(0);
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) {
        const int l = lane + 32 * kk;
        if (l < nT) p += Sr[(size_t)i * nT + l] * xv[kk];
      }
      p = warp_sum(p);
      if (lane == i) acc += p;
    }
  }
  if (lane < bs) y[(size_t)t * bs + lane] = double(acc);
}

// P_f = sum of both sides' diagonal face blocks of S_k, inverted by Gauss-Jordan with partial
// pivoting in FP64.  One block of 64 threads per face.
template <typename T>
__global__ void k_precond_build(const __grid_constant__ TraceArgs a, double* __restrict__ Pinv, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t = blockIdx.x;
  const int bs = a.n * a.nv, nT = a.nT;
  const int ld = 2 * bs;
  double* M = reinterpret_cast<double*>(smem_raw);  // bs x 2bs  [P | I]
  __shared__ int s_piv;
  __shared__ double fac[32];
  const T* S = reinterpret_cast<const T*>(a.S);
  for (int i = threadIdx.x; i < bs * ld; i += blockDim.x) {
    const int r = i / ld, c = i % ld;
    double v = 0.0;
    if (c < bs) {
      for (int side = 0; side < 2; ++side) {
        const int e = a.sides[t * 4 + side * 2], f = a.sides[t * 4 + side * 2 + 1];
        if (e >= 0) v += double(S[((size_t)e * nT + f * bs + r) * nT + f * bs + c]);
      }
    } else {
      v = (c - bs == r) ? 1.0 : 0.0;
    }
    M[i] = v;
  }
  __syncthreads();
  for (int c = 0; c < bs; ++c) {
    if (threadIdx.x == 0) {
      int p = c;
      double best = fabs(M[c * ld + c]);
      for (int i = c + 1; i < bs; ++i) {
        double v = fabs(M[i * ld + c]);
        if (v > best) { best = v; p = i; }
      }
      s_piv = p;
      if (!(best > 0.0)) {
        atomicOr(status, DEV_ERR_SINGULAR);
      }
    }
    __syncthreads();
    const int p = s_piv;
    if (p != c)
      for (int j = threadIdx.x; j < ld; j += blockDim.x) {
        double t0 = M[c * ld + j];
        M[c * ld + j] = M[p * ld + j];
        M[p * ld + j] = t0;
      }
    __syncthreads();
    const double pv = M[c * ld + c];
    const double inv = pv != 0.0 ? 1.0 / pv : 0.0;
    __syncthreads();
    for (int j = threadIdx.x; j < ld; j += blockDim.x) M[c * ld + j] *= inv;
    for (int i = threadIdx.x; i < bs; i += blockDim.x) fac[i] = M[i * ld + c];
    __syncthreads();
    for (int it = threadIdx.x; it < bs * ld; it += blockDim.x) {
      const int i = it / ld, j = it % ld;
      if (i != c) M[i * ld + j] -= fac[i] * M[c * ld + j];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < bs * bs; i += blockDim.x) {
    const int r = i / bs, c = i % bs;
    Pinv[(size_t)t * bs * bs + i] = M[r * ld + bs + c];
  }
}

// y_f = Pinv_f x_f, one warp per face, lane = row
__global__ void k_precond_apply(const __grid_constant__ TraceArgs a, const double* __restrict__ Pinv,
                                const double* __restrict__ x, double* __restrict__ y, const int* gate, int gj) {
  if (gate && *gate >= 0 && gj >= *gate) return;
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= a.ntrace) return;
  const int bs = a.n * a.nv;
  const double* P = Pinv + (size_t)t * bs * bs;
  const double xv = lane < bs ? x[(size_t)t * bs + lane] : 0.0;
  double acc = 0.0;
  for (int j = 0; j < bs; ++j) {
    const double xj = __shfl_sync(0xffffffffu, xv, j);
    if (lane < bs) acc += P[lane * bs + j] * xj;
  }
  if (lane < bs) y[(size_t)t * bs + lane] = acc;
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

// du_k = x_r - X_B du^_k ; one warp per row, 4 warps per element
template <typename T>
__global__ void k_backsolve(const __grid_constant__ TraceArgs a, int Eim, int nA, const T* __restrict__ XB,
                            const double* __restrict__ xr, const double* __restrict__ duhat,
                            double* __restrict__ du) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xv = reinterpret_cast<T*>(smem_raw);
  const int k = blockIdx.x;
  if (k >= Eim) return;
  const int bs = a.n * a.nv, nT = a.nT;
  for (int l = threadIdx.x; l < nT; l += blockDim.x) {
    const int fp = l / bs;
    const int tf = a.tr_of_c[k * 4 + fp];
    xv[l] = tf >= 0 ? T(duhat[(size_t)tf * bs + (l - fp * bs)]) : T(0);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  const T* X = XB + (size_t)k * nA * nT;
  for (int i = warp; i < nA; i += nw) {
    T p = T(0);
    for (int l = lane; l < nT; l += 32) p += X[(size_t)i * nT + l] * xv[l];
    p = warp_sum(p);
    if (lane == 0) du[(size_t)k * nA + i] = xr[(size_t)k * nA + i] - double(p);
  }
}

cudaError_t launch_trace_matvec(int prec_bytes, const TraceArgs& a, const double* x, double* y, cudaStream_t st,
                                const int* gate, int gj) {
  if (a.ntrace == 0) return cudaSuccess;
  const int threads = 256;
  const int grid = (a.ntrace * 32 + threads - 1) / threads;
  if (prec_bytes == 8)
    (hfr::count_launch(), k_trace_matvec<double><<<grid, threads, 0, st>>>(a, x, y, gate, gj));
  else
    (hfr::count_launch(), k_trace_matvec<float><<<grid, threads, 0, st>>>(a, x, y, gate, gj));
  return cudaGetLastError();
}

cudaError_t launch_precond_build(int prec_bytes, const TraceArgs& a, double* Pinv, int* status, cudaStream_t st) {
  if (a.ntrace == 0) return cudaSuccess;
  const int bs = a.n * a.nv;
  size_t smem = sizeof(double) * bs * 2 * bs;
  if (prec_bytes == 8)
    (hfr::count_launch(), k_precond_build<double><<<a.ntrace, 64, smem, st>>>(a, Pinv, status));
  else
    (hfr::count_launch(), k_precond_build<float><<<a.ntrace, 64, smem, st>>>(a, Pinv, status));
  return cudaGetLastError();
}

cudaError_t launch_precond_apply(const TraceArgs& a, const double* Pinv, const double* x, double* y,
                                 cudaStream_t st, const int* gate, int gj) {
  if (a.ntrace == 0) return cudaSuccess;
  const int threads = 256;
  (hfr::count_launch(), k_precond_apply<<<(a.ntrace * 32 + threads - 1) / threads, threads, 0, st>>>(a, Pinv, x, y, gate, gj));
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
  if (prec_bytes == 8)
    (hfr::count_launch(), k_backsolve<double><<<Eim, 128, sizeof(double) * a.nT, st>>>(a, Eim, nA, (const double*)XB, xr, duhat, du));
  else
    (hfr::count_launch(), k_backsolve<float><<<Eim, 128, sizeof(float) * a.nT, st>>>(a, Eim, nA, (const float*)XB, xr, duhat, du));
  return cudaGetLastError();
}

}  // namespace hfr
