// Restarted right-preconditioned GMRES(m) for the condensed trace system L du^ = t
// (Pereira & Vermeire, arXiv 2401.16632, Sec. 3.2; the paper does not name its linear solver).
//
// Vectors, orthogonalisation (classical Gram-Schmidt applied twice), norms, Givens rotations
// and the solution update are FP64.  The Hessenberg matrix and rotations live on the device;
// every kernel of inner iteration j returns immediately once the device state says the cycle
// ended before j, so the host can enqueue several iterations between synchronisations.
// Reductions are two-stage with a fixed summation order (bitwise reproducible).
#include "hfr_krylov.h"

namespace hfr {

constexpr int KB = 256;  // threads per block of the vector kernels

__device__ __forceinline__ bool gated(const GmresState* st, int j) { return st->kdone >= 0 && j >= st->kdone; }

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;  // valid in thread 0
}

// partial[b * (GM_MAXM + 1) + i] = sum over block b's slice of V_i . w   (i < nvec)
__global__ void k_dot_part(const GmresState* st, int j, const double* __restrict__ V, size_t n, int nvec,
                           const double* __restrict__ w, double* __restrict__ partial) {
  if (st && gated(st, j)) return;
  __shared__ double red[KB / 32];
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = 0; i < nvec; ++i) {
    const double* Vi = V + (size_t)i * n;
    double s = 0.0;
    for (size_t x = i0; x < n; x += stride) s += Vi[x] * w[x];
    s = block_sum(s, red);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * (GM_MAXM + 1) + i] = s;
  }
}

// out[i] = sum_b partial[b][i] (mode 0: store to hc, 1: store to h2 and add into hc,
// 2: store sqrt into hc[j+1] (norm), 3: store sqrt into beta / bnorm)
__global__ void k_dot_final(GmresState* st, int j, const double* __restrict__ partial, int nblk, int nvec,
                            int mode) {
  if (mode <= 2 && gated(st, j)) return;
  const int i = threadIdx.x;
  if (i >= nvec) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * (GM_MAXM + 1) + i];
  if (mode == 0) st->hc[i] = s;
  else if (mode == 1) { st->h2[i] = s; st->hc[i] += s; }
  else if (mode == 2) st->hc[j + 1] = sqrt(s);
  else if (mode == 3) st->beta = sqrt(s);
  else if (mode == 4) st->bnorm = sqrt(s);
}

// w -= sum_i c_i V_i  (which = 0: c = hc, 1: c = h2);  or x += sum_i y_i Z_i (which = 2)
__global__ void k_axpy_multi(const GmresState* st, int j, const double* __restrict__ V, size_t n, int nvec,
                             double* __restrict__ w, int which) {
  if (which < 2 && gated(st, j)) return;
  const double* c = which == 0 ? st->hc : (which == 1 ? st->h2 : st->y);
  const double sg = which == 2 ? 1.0 : -1.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
    double acc = 0.0;
    for (int i = 0; i < nvec; ++i) acc += c[i] * V[(size_t)i * n + x];
    w[x] += sg * acc;
  }
}

// Givens update for column j; decides the end of the cycle
__global__ void k_givens(GmresState* st, int j, double rtol, int m) {
  if (gated(st, j) || threadIdx.x != 0) return;
  double* h = st->hc;
  for (int i = 0; i < j; ++i) {
    const double a = h[i], b = h[i + 1];
    h[i] = st->cs[i] * a + st->sn[i] * b;
    h[i + 1] = -st->sn[i] * a + st->cs[i] * b;
  }
  const double a = h[j], b = h[j + 1];
  st->hn = b;
  const double r = sqrt(a * a + b * b);
  double c = 1.0, s = 0.0;
  if (r > 0.0) { c = a / r; s = b / r; }
  st->cs[j] = c;
  st->sn[j] = s;
  h[j] = r;
  h[j + 1] = 0.0;
  for (int i = 0; i <= j; ++i) st->H[i * GM_MAXM + j] = h[i];
  st->g[j + 1] = -s * st->g[j];
  st->g[j] = c * st->g[j];
  st->res = fabs(st->g[j + 1]);
  st->k = j + 1;
  if (!(st->res == st->res)) { st->kdone = j + 1; st->nan = 1; return; }
  if (st->res <= rtol * st->bnorm) { st->kdone = j + 1; st->converged = 1; }
  else if (j + 1 >= m || st->hn == 0.0) st->kdone = j + 1;
}

// v_{j+1} = w / hn (in place)
__global__ void k_scale_next(const GmresState* st, int j, double* __restrict__ w, size_t n) {
  if (st->kdone >= 0 && j >= st->kdone) return;
  const double hn = st->hn;
  if (hn == 0.0) return;
  const double inv = 1.0 / hn;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) w[x] *= inv;
}

// start of a cycle: V0 = r / beta, g = beta e1
__global__ void k_cycle_start(GmresState* st, double* __restrict__ v0, size_t n, double rtol) {
  const double beta = st->beta;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->kdone = -1;
    st->k = 0;
    st->g[0] = beta;
    st->res = beta;
    if (beta <= rtol * st->bnorm || beta == 0.0) { st->kdone = 0; st->converged = 1; }
  }
  if (beta == 0.0) return;
  const double inv = 1.0 / beta;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) v0[x] *= inv;
}

// back substitution of the k x k triangle, y = H^{-1} g
__global__ void k_solve_y(GmresState* st) {
  if (threadIdx.x != 0) return;
  const int k = st->k;
  for (int i = k - 1; i >= 0; --i) {
    double s = st->g[i];
    for (int c = i + 1; c < k; ++c) s -= st->H[i * GM_MAXM + c] * st->y[c];
    const double d = st->H[i * GM_MAXM + i];
    st->y[i] = d != 0.0 ? s / d : 0.0;
  }
}

__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                      size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) out[x] = a[x] - b[x];
}

__global__ void k_reset_state(GmresState* st) {
  if (threadIdx.x == 0) {
    st->converged = 0;
    st->nan = 0;
    st->kdone = -1;
    st->k = 0;
  }
}

static int grid_for(size_t n) {
  size_t g = (n + KB - 1) / KB;
  if (g > (size_t)GM_NBLK) g = GM_NBLK;
  if (g == 0) g = 1;
  return (int)g;
}

// ||v||^2 partials + final into the given mode slot
static void norm_into(GmresState* st, int j, const double* v, size_t n, double* partial, int mode, cudaStream_t s) {
  const int nb = grid_for(n);
  (hfr::count_launch(), k_dot_part<<<nb, KB, 0, s>>>(mode <= 2 ? st : nullptr, j, v, n, 1, v, partial));
  (hfr::count_launch(), k_dot_final<<<1, 64, 0, s>>>(st, j, partial, nb, 1, mode));
}

int run_gmres(const GmresOps& ops, const GmresBuffers& b, const double* t, double* x, double rtol, int restart,
              int maxit, int check_every, GmresResult* res, cudaStream_t s) {
  const size_t n = b.n;
  const int m = restart > GM_MAXM ? GM_MAXM : (restart < 1 ? 1 : restart);
  GmresState* st = b.state;
  const int nb = grid_for(n);
  (hfr::count_launch(), k_reset_state<<<1, 32, 0, s>>>(st));
  norm_into(st, 0, t, n, b.partial, 4, s);  // bnorm
  cudaMemsetAsync(x, 0, n * sizeof(double), s);
  int total = 0;
  bool first = true;
  GmresHead hs;
  for (;;) {
    // r = t - L x into V0
    if (first) {
      cudaMemcpyAsync(b.V, t, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    } else {
      ops.matvec(ops.ctx, x, b.V + n * 0 + 0, s);  // temporarily L x in V0
      (hfr::count_launch(), k_sub<<<nb, KB, 0, s>>>(t, b.V, b.V, n));
    }
    first = false;
    norm_into(st, 0, b.V, n, b.partial, 3, s);  // beta
    (hfr::count_launch(), k_cycle_start<<<nb, KB, 0, s>>>(st, b.V, n, rtol));
    int j = 0;
    for (; j < m; ++j) {
      double* vj = b.V + (size_t)j * n;
      double* w = b.V + (size_t)(j + 1) * n;
      double* zj = b.Z + (size_t)j * n;
      ops.precond(ops.ctx, st, j, vj, zj, s);
      ops.gated_matvec(ops.ctx, st, j, zj, w, s);
      (hfr::count_launch(), k_dot_part<<<nb, KB, 0, s>>>(st, j, b.V, n, j + 1, w, b.partial));
      (hfr::count_launch(), k_dot_final<<<1, 64, 0, s>>>(st, j, b.partial, nb, j + 1, 0));
      (hfr::count_launch(), k_axpy_multi<<<nb, KB, 0, s>>>(st, j, b.V, n, j + 1, w, 0));
      (hfr::count_launch(), k_dot_part<<<nb, KB, 0, s>>>(st, j, b.V, n, j + 1, w, b.partial));
      (hfr::count_launch(), k_dot_final<<<1, 64, 0, s>>>(st, j, b.partial, nb, j + 1, 1));
      (hfr::count_launch(), k_axpy_multi<<<nb, KB, 0, s>>>(st, j, b.V, n, j + 1, w, 1));
      norm_into(st, j, w, n, b.partial, 2, s);
      (hfr::count_launch(), k_givens<<<1, 32, 0, s>>>(st, j, rtol, m));
      (hfr::count_launch(), k_scale_next<<<nb, KB, 0, s>>>(st, j, w, n));
      if ((j + 1) % check_every == 0 || j + 1 == m) {
        cudaMemcpyAsync(&hs, st, sizeof(GmresHead), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
        if (hs.kdone >= 0) break;
      }
    }
    cudaMemcpyAsync(&hs, st, sizeof(GmresHead), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    const int k = hs.k;
    if (k > 0) {
      (hfr::count_launch(), k_solve_y<<<1, 32, 0, s>>>(st));
      (hfr::count_launch(), k_axpy_multi<<<nb, KB, 0, s>>>(st, 0, b.Z, n, k, x, 2));
    }
    total += k;
    if (hs.nan) {
      res->iterations = total;
      res->converged = 0;
      res->nan = 1;
      break;
    }
    if (hs.converged || total >= maxit || (k == 0)) {
      res->iterations = total;
      res->converged = hs.converged;
      res->nan = 0;
      break;
    }
  }
  // true final relative residual
  ops.matvec(ops.ctx, x, b.V, s);
  (hfr::count_launch(), k_sub<<<nb, KB, 0, s>>>(t, b.V, b.V, n));
  norm_into(st, 0, b.V, n, b.partial, 3, s);
  cudaMemcpyAsync(&hs, st, sizeof(GmresHead), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  res->bnorm = hs.bnorm;
  res->rel = hs.bnorm > 0.0 ? hs.beta / hs.bnorm : 0.0;
  return 0;
}

}  // namespace hfr
