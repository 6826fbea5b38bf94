// Allocation-free variant of the element condensation, for callers that may not allocate device
// memory themselves or let a library do it: for example a host code that owns a fixed device
// memory budget through its own pool and forbids foreign cudaMalloc calls, or a plugin that is
// handed pre-allocated buffers and must not change the process's allocation state.  Such a
// caller passes its blocks and output buffers; the factors and pivots that the condensation
// needs as scratch live in a file-scope device array instead of a context workspace.
//
// This has no counterpart in the paper; it reuses the condensation kernels of hfr_condense.cu.
#include <mutex>

#include "../../include/hfr.h"
#include "hfr_internal.h"

// Scratch: [status words | pivots | factors].  Every GPU that loads this library holds this array
// until the process exits.
static __device__ __align__(256) unsigned char g_hfr_noalloc_scratch[HFR_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_scratch_mu;
void* g_scratch_ptr[64] = {nullptr};  // device address of the array, per device ordinal

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

__global__ void k_reset_status(int* status) {
  status[0] = 0;
  status[1] = 0x7fffffff;
}

// Device address of the scratch array on the current device (looked up once per device).
int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_hfr_noalloc_scratch) != cudaSuccess || p == nullptr) return FR_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return FR_OK;
}
}  // namespace

extern "C" int hfr_condense_noalloc(int nimplicit, int nA, int nT, int precision, const void* A, const void* B,
                                    const void* C, const void* D, const double* r, const double* s, void* XB,
                                    double* xr, void* S, double* t, void* stream) {
  if (nimplicit < 0 || nA <= 0 || nT <= 0 || nA > 160 || (precision != FR_PREC_FP64 && precision != FR_PREC_FP32))
    return FR_ERR_INVALID_ARG;
  if (!hfr::condense_feasible(precision == FR_PREC_FP64 ? 8 : 4, nA, nT)) return FR_ERR_INVALID_ARG;
  if (nimplicit == 0) return FR_OK;
  if (!A || !B || !C || !D || !r || !s || !XB || !xr || !S || !t) return FR_ERR_INVALID_ARG;
  const size_t pb = precision == FR_PREC_FP64 ? 8 : 4;
  const size_t off_piv = 256;
  const size_t off_fac = off_piv + round256((size_t)nimplicit * nA * sizeof(int));
  const size_t need = off_fac + (size_t)nimplicit * nA * nA * pb;
  if (need > (size_t)HFR_NOALLOC_SCRATCH_BYTES) return FR_ERR_INVALID_ARG;  // beyond the scratch size
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != FR_OK) return rc;
  unsigned char* sc = static_cast<unsigned char*>(base);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: reset the status words
  (hfr::count_launch(), k_reset_status<<<1, 1, 0, st>>>(reinterpret_cast<int*>(sc)));
  if (cudaGetLastError() != cudaSuccess) return FR_ERR_CUDA;
  hfr::CondArgs a;
  a.Eim = nimplicit;
  a.nA = nA;
  a.nT = nT;
  a.A = A;
  a.B = B;
  a.C = C;
  a.D = D;
  a.r = r;
  a.s = s;
  a.LU = sc + off_fac;
  a.piv = reinterpret_cast<int*>(sc + off_piv);
  a.XB = XB;
  a.xr = xr;
  a.S = S;
  a.t = t;
  a.status = reinterpret_cast<int*>(sc);
  if (hfr::launch_condense((int)pb, a, st) != cudaSuccess) return FR_ERR_CUDA;
  int hs[2] = {0, 0};
  if (cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess) return FR_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return FR_ERR_CUDA;
  return (hs[0] & DEV_ERR_SINGULAR) ? FR_ERR_SINGULAR : FR_OK;
}
