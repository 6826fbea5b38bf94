// Pipe peaks of the running GPU, measured with CUDA events (no counterpart in the paper): the
// denominators of the roofline fractions of kernels bound by the FP64 or FP32 FMA pipes or by the
// TF32 tensor-core pipe.
//
//   FP64 / FP32: every thread runs 8 independent FMA chains (x <- x m + c), 16 unrolled steps per
//                loop trip, 8 CTAs of 256 threads per SM; 2 flops per FMA.
//   TF32:        one elected thread per CTA issues tcgen05.mma.kind::tf32 of shape M = 128,
//                N = 256, K = 8 back to back on fixed shared-memory operands into a tensor-memory
//                accumulator (2 M N K flops each), two CTAs per SM; completion through an mbarrier
//                whose wait is bounded.
// Nothing is allocated: the kernels write only a file-scope device sink.
#include <math.h>

#include "../../include/hfr.h"
#include "hfr_internal.h"
#include "hfr_tc.cuh"

namespace {

__device__ double g_peak_sink[4];
__device__ unsigned g_peak_status;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_loop(int iters, T m, T c) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = fma(x[i], m, c);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == T(-1.2345e30)) g_peak_sink[sizeof(T) == 8 ? 0 : 1] = (double)s;  // keeps the chains alive
}

constexpr int MMA_M = 128, MMA_N = 256, MMA_K = 8;  // K in TF32 elements: one 32-byte K extent
constexpr uint32_t MMA_SBO = 256;                   // (K / 4) * 128 bytes between 8-row groups

__global__ void __launch_bounds__(128) k_tf32_mma_loop(int reps) {
  using namespace hfr::tc;
  __shared__ __align__(1024) unsigned char opA[MMA_M * MMA_K * 4];
  __shared__ __align__(1024) unsigned char opB[MMA_N * MMA_K * 4];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int t = threadIdx.x, w = t >> 5;
  for (int i = t; i < MMA_M * MMA_K; i += 128)
    reinterpret_cast<float*>(opA)[i] = __uint_as_float(0x3c000000u + (unsigned)(i & 7) * 0x2000u);
  for (int i = t; i < MMA_N * MMA_K; i += 128)
    reinterpret_cast<float*>(opB)[i] = __uint_as_float(0x3c000000u + (unsigned)(i & 3) * 0x2000u);
  if (t == 0) mbar_init(smem_u32(&mbar), 1);
  if (w == 0) tmem_alloc(smem_u32(&tslot), MMA_N);
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tslot;
  bool ok = true;
  if (t == 0) {
    const uint64_t da = desc_noswizzle(smem_u32(opA), 128, MMA_SBO);
    const uint64_t db = desc_noswizzle(smem_u32(opB), 128, MMA_SBO);
    constexpr uint32_t idesc = idesc_tf32(MMA_M, MMA_N);
#pragma unroll 1
    for (int r = 0; r < reps; ++r) mma_tf32(tmem, da, db, idesc, r > 0 ? 1u : 0u);
    mma_commit(smem_u32(&mbar));
  }
  ok = mbar_wait(smem_u32(&mbar), 0, TIMEOUT_NS);
  if (!ok) atomicOr(&g_peak_status, 1u);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (w == 0) tmem_dealloc(tmem, MMA_N);
}

}  // namespace

extern "C" int fr_measure_peak(int which, void* stream, double* tflops) {
  if (!tflops || which < 0 || which > 2) return FR_ERR_INVALID_ARG;
  *tflops = 0.0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FR_ERR_CUDA;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return FR_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return FR_ERR_CUDA;
  }
  const unsigned zero = 0;
  int rc = FR_OK;
  double flops = 0.0;
  // warm-up launch, then the timed one (a few tens of milliseconds each)
  for (int pass = 0; pass < 2 && rc == FR_OK; ++pass) {
    if (pass == 1 && cudaEventRecord(e0, st) != cudaSuccess) rc = FR_ERR_CUDA;
    const int grid = which == 2 ? 2 * nsm : 8 * nsm;
    if (which == 0) {
      const int iters = 1200;
      (hfr::count_launch(), k_fma_loop<double><<<grid, 256, 0, st>>>(iters, 0.999999, 1e-7));
      flops = 2.0 * 8 * 16 * (double)iters * grid * 256;
    } else if (which == 1) {
      const int iters = 40000;
      (hfr::count_launch(), k_fma_loop<float><<<grid, 256, 0, st>>>(iters, 0.999999f, 1e-7f));
      flops = 2.0 * 8 * 16 * (double)iters * grid * 256;
    } else {
      if (pass == 0 && cudaMemcpyToSymbolAsync(g_peak_status, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = FR_ERR_CUDA;
      // 96 KB of (unused) dynamic shared memory holds residency at two CTAs per SM, so that the
      // two 256-column tensor-memory allocations of an SM never wait for each other
      const int reps = 40000;
      const int dyn = 96 * 1024;
      if (pass == 0 && cudaFuncSetAttribute(k_tf32_mma_loop, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess)
        rc = FR_ERR_CUDA;
      (hfr::count_launch(), k_tf32_mma_loop<<<grid, 128, dyn, st>>>(reps));
      flops = 2.0 * MMA_M * MMA_N * MMA_K * (double)reps * grid;
    }
    if (cudaGetLastError() != cudaSuccess) rc = FR_ERR_CUDA;
    if (pass == 1 && cudaEventRecord(e1, st) != cudaSuccess) rc = FR_ERR_CUDA;
  }
  float ms = 0.f;
  if (rc == FR_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    rc = FR_ERR_CUDA;
  if (rc == FR_OK && which == 2) {
    unsigned status = 0;
    if (cudaMemcpyFromSymbol(&status, g_peak_status, sizeof(status)) != cudaSuccess) rc = FR_ERR_CUDA;
    else if (status) rc = FR_ERR_TIMEOUT;
  }
  if (rc == FR_OK && ms > 0.f) *tflops = flops / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}
