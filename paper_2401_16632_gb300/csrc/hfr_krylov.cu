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

// One fused pass of classical Gram-Schmidt (twice) over the Krylov basis:
//   pre 0: (nothing)   1: w -= sum_i hc_i V_i   2: w -= sum_i h2_i V_i      (i < na)
// then the dots out_i = D_i . w (i < nd; D = V, or D = w itself for a norm) accumulated eight
// at a time in registers, one partial per block, and the last block to finish (ticket) reduces
// the partials in a fixed order (deterministic) and applies `mode`:
//   0: hc[i] = s   1: h2[i] = s, hc[i] += s   2: hc[j+1] = sqrt(s) + Givens update of column j
//   3: beta = sqrt(s)   4: bnorm = sqrt(s)
// Each thread re-reads only its own w entries after updating them, so no grid-wide barrier is
// needed between the update and the dots.
__device__ void givens_update(GmresState* st, int j, double rtol, int m);

__global__ void __launch_bounds__(KB) k_cgs(GmresState* st, int j, const double* __restrict__ V, size_t n, int na,
                                            int pre, const double* D, int nd, double* w,
                                            double* __restrict__ partial, unsigned int* ticket, int mode, double rtol,
                                            int m, int only_if_reorth) {
  if ((mode <= 2 || mode >= 5) && gated(st, j)) return;
  if (only_if_reorth && !st->reorth) return;
  __shared__ double red[GM_MAXM + 1][KB / 32];
  __shared__ bool last;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (pre) {
    const double* c = pre == 1 ? st->hc : st->h2;
    for (size_t x = i0; x < n; x += stride) {
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      int i = 0;
      for (; i + 3 < na; i += 4) {
        a0 += c[i] * V[(size_t)i * n + x];
        a1 += c[i + 1] * V[(size_t)(i + 1) * n + x];
        a2 += c[i + 2] * V[(size_t)(i + 2) * n + x];
        a3 += c[i + 3] * V[(size_t)(i + 3) * n + x];
      }
      for (; i < na; ++i) a0 += c[i] * V[(size_t)i * n + x];
      w[x] -= (a0 + a1) + (a2 + a3);
    }
  }
  // sixteen dots at a time: per-thread partial sums, then a warp reduce-scatter (each butterfly
  // level halves the values a lane carries: 16 shuffles for 16 sums instead of 80), so lane l
  // ends with the warp sum of value l >> 1
  for (int c0 = 0; c0 < nd; c0 += 16) {
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (size_t x = i0; x < n; x += stride) {
      const double wx = w[x];
#pragma unroll
      for (int q = 0; q < 16; ++q)
        if (c0 + q < nd) acc[q] += D[(size_t)(c0 + q) * n + x] * wx;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const bool up = lane & 16;
      const double send = up ? acc[q] : acc[q + 8];
      const double keep = up ? acc[q + 8] : acc[q];
      acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool up = lane & 8;
      const double send = up ? acc[q] : acc[q + 4];
      const double keep = up ? acc[q + 4] : acc[q];
      acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const bool up = lane & 4;
      const double send = up ? acc[q] : acc[q + 2];
      const double keep = up ? acc[q + 2] : acc[q];
      acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
      const bool up = lane & 2;
      const double send = up ? acc[0] : acc[1];
      const double keep = up ? acc[1] : acc[0];
      acc[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
    const int vi = c0 + (lane >> 1);
    if ((lane & 1) == 0 && vi < nd) red[vi][wid] = acc[0];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nd; i += KB) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < KB / 32; ++k) t += red[i][k];
    partial[(size_t)blockIdx.x * (GM_MAXM + 1) + i] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int i = wid; i < nd; i += KB / 32) {
    double t = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(&partial[(size_t)b * (GM_MAXM + 1) + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) {
      if (mode == 0) st->hc[i] = t;
      else if (mode == 1) { st->h2[i] = t; st->hc[i] += t; }
      else if (mode == 2 || mode == 6) st->hc[j + 1] = sqrt(t);
      else if (mode == 3) st->beta = sqrt(t);
      else if (mode == 4) st->bnorm = sqrt(t);
      else if (mode == 5) { if (i < nd - 1) st->hc[i] = t; else st->wnorm_old = sqrt(t); }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *ticket = 0u;
    if (mode == 2) {
      st->reorth = 0;
      givens_update(st, j, rtol, m);
    } else if (mode == 6) {
      // DGKS: a second Gram-Schmidt pass only when the projection removed most of w
      if (st->hc[j + 1] < 0.70710678118654752 * st->wnorm_old) st->reorth = 1;
      else givens_update(st, j, rtol, m);
    }
  }
}

// w -= sum_i c_i V_i  (which = 0: c = hc, 1: c = h2);  or x += sum_i y_i Z_i (which = 2)
__global__ void k_axpy_multi(const GmresState* st, int j, const double* __restrict__ V, size_t n, int nvec,
                             double* __restrict__ w, int which) {
  if (which < 2 && gated(st, j)) return;
  const double* c = which == 0 ? st->hc : (which == 1 ? st->h2 : st->y);
  const double sg = which == 2 ? 1.0 : -1.0;
  if (nvec < 0) nvec = st->k;  // the cycle's length, from the device state
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
    double acc = 0.0;
    for (int i = 0; i < nvec; ++i) acc += c[i] * V[(size_t)i * n + x];
    w[x] += sg * acc;
  }
}

// Givens update for column j; decides the end of the cycle
__device__ void givens_update(GmresState* st, int j, double rtol, int m) {
  double* h = st->hc;
  for (int i = 0; i < j; ++i) {
    const double a = h[i], b = h[i + 1];
    h[i] = st->cs[i] * a + st->sn[i] * b;
    h[i + 1] = -st->sn[i] * a + st->cs[i] * b;
  }
  const double a = h[j], b = h[j + 1];
  st->hn = b;
  st->inv_hn = b != 0.0 ? 1.0 / b : 0.0;
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
    st->reorth = 0;
    st->inv_hn = 0.0;
  }
}

static int grid_for(size_t n) {
  size_t g = (n + KB - 1) / KB;
  if (g > (size_t)GM_NBLK) g = GM_NBLK;
  if (g == 0) g = 1;
  return (int)g;
}

// ||v||^2 into the given mode slot (mode 2 also performs the Givens update)
static void norm_into(const GmresBuffers& b, int j, double* v, size_t n, int mode, double rtol, int m,
                      cudaStream_t s) {
  const int nb = grid_for(n);
  (hfr::count_launch(), k_cgs<<<nb, KB, 0, s>>>(b.state, j, nullptr, n, 0, 0, v, 1, v, b.partial, b.ticket, mode,
                                                 rtol, m, 0));
}

int run_gmres(const GmresOps& ops, const GmresBuffers& b, const double* t, double* x, double rtol, int restart,
              int maxit, int check_every, GmresResult* res, cudaStream_t s) {
  const size_t n = b.n;
  const int m = restart > GM_MAXM ? GM_MAXM : (restart < 1 ? 1 : restart);
  GmresState* st = b.state;
  const int nb = grid_for(n);
  (hfr::count_launch(), k_reset_state<<<1, 32, 0, s>>>(st));
  // (reorth flag and inv_hn are reset by k_reset_state)
  norm_into(b, 0, const_cast<double*>(t), n, 4, rtol, m, s);  // bnorm (t is only read)
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
    // this cycle's length: the restart length, capped by the iterations left
    const int mc = m < maxit - total ? m : maxit - total;
    norm_into(b, 0, b.V, n, 3, rtol, mc, s);  // beta
    (hfr::count_launch(), k_cycle_start<<<nb, KB, 0, s>>>(st, b.V, n, rtol));
    int j = 0;
    for (; j < mc; ++j) {
      double* vj = b.V + (size_t)j * n;
      double* w = b.V + (size_t)(j + 1) * n;
      double* zj = b.Z + (size_t)j * n;
      // v_j = w_j / h_{j,j-1} is normalised in place by the preconditioner kernel (j > 0)
      ops.precond(ops.ctx, st, j, vj, zj, b.z32, s);
      ops.gated_matvec(ops.ctx, st, j, zj, b.z32, w, s);
      // classical Gram-Schmidt with a conditional second pass (DGKS): pass 1 also yields ||w||,
      // since w = V_{j+1} follows V_j in memory
      (hfr::count_launch(), k_cgs<<<nb, KB, 0, s>>>(st, j, b.V, n, j + 1, 0, b.V, j + 2, w, b.partial, b.ticket, 5,
                                                     rtol, mc, 0));
      (hfr::count_launch(), k_cgs<<<nb, KB, 0, s>>>(st, j, b.V, n, j + 1, 1, w, 1, w, b.partial, b.ticket, 6, rtol,
                                                     mc, 0));
      (hfr::count_launch(), k_cgs<<<nb, KB, 0, s>>>(st, j, b.V, n, j + 1, 0, b.V, j + 1, w, b.partial, b.ticket, 1,
                                                     rtol, mc, 1));
      (hfr::count_launch(), k_cgs<<<nb, KB, 0, s>>>(st, j, b.V, n, j + 1, 2, w, 1, w, b.partial, b.ticket, 2, rtol,
                                                     mc, 1));
      if ((j + 1) % check_every == 0 || j + 1 == mc) {
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
  norm_into(b, 0, b.V, n, 3, rtol, m, s);
  cudaMemcpyAsync(&hs, st, sizeof(GmresHead), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  res->bnorm = hs.bnorm;
  res->rel = hs.bnorm > 0.0 ? hs.beta / hs.bnorm : 0.0;
  return 0;
}

// ------------------------------------------------------------ GMRES inside a captured graph
__global__ void k_gg_begin(GmresGraphDev* d, cudaGraphConditionalHandle hw) {
  d->first = 1;
  d->total = 0;
  d->cycles = 0;
  d->nan = 0;
  d->converged = 0;
  cudaGraphSetConditional(hw, 1u);
}
// the residual mat-vec runs on every cycle but the first (x = 0 there)
__global__ void k_gg_ifres(const GmresGraphDev* d, cudaGraphConditionalHandle hi) {
  cudaGraphSetConditional(hi, d->first ? 0u : 1u);
}
// V0 = t on the first cycle (later ones hold t - L x already)
__global__ void k_gg_start(const GmresGraphDev* d, const double* __restrict__ t, double* __restrict__ v0, size_t n) {
  if (!d->first) return;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) v0[x] = t[x];
}
// the restart decision of the host driver, on the device
__global__ void k_gg_after(GmresGraphDev* d, const GmresState* st, int maxit, cudaGraphConditionalHandle hw) {
  const int k = st->k;
  d->total += k;
  d->cycles += 1;
  d->first = 0;
  if (st->nan) d->nan = 1;
  d->converged = st->converged;
  const int cont = (st->nan || st->converged || d->total >= maxit || k == 0) ? 0 : 1;
  cudaGraphSetConditional(hw, (unsigned)cont);
}

cudaError_t capture_gmres(const GmresOps& ops, const GmresBuffers& b, const double* t, double* x, double rtol,
                          int restart, int maxit, GmresGraphDev* dev, cudaStream_t s, const cudaStream_t sc[2],
                          GmresGraphLaunches* counts) {
  const size_t n = b.n;
  const int m = restart > GM_MAXM ? GM_MAXM : (restart < 1 ? 1 : restart);
  GmresState* st = b.state;
  const int nb = grid_for(n);
  cudaError_t e;
  const unsigned long long l0 = hfr::launch_count();
  cudaGraphConditionalHandle hw, hi;
  if ((e = graph_conditional_handle(s, 0u, 0u, &hw)) != cudaSuccess) return e;
  (hfr::count_launch(), k_reset_state<<<1, 32, 0, s>>>(st));
  norm_into(b, 0, const_cast<double*>(t), n, 4, rtol, m, s);  // bnorm
  if ((e = cudaMemsetAsync(x, 0, n * sizeof(double), s)) != cudaSuccess) return e;
  (hfr::count_launch(), k_gg_begin<<<1, 1, 0, s>>>(dev, hw));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cudaGraph_t body = nullptr, ifb = nullptr;
  if ((e = graph_add_conditional(s, hw, cudaGraphCondTypeWhile, &body)) != cudaSuccess) return e;
  const unsigned long long l1 = hfr::launch_count();
  // ---- one restart cycle
  if ((e = cudaStreamBeginCaptureToGraph(sc[0], body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
      cudaSuccess)
    return e;
  auto abort0 = [&](cudaError_t ee) {
    cudaGraph_t tmp = nullptr;
    cudaStreamEndCapture(sc[0], &tmp);
    return ee;
  };
  if ((e = graph_conditional_handle(sc[0], 0u, 0u, &hi)) != cudaSuccess) return abort0(e);
  (hfr::count_launch(), k_gg_ifres<<<1, 1, 0, sc[0]>>>(dev, hi));
  if ((e = graph_add_conditional(sc[0], hi, cudaGraphCondTypeIf, &ifb)) != cudaSuccess) return abort0(e);
  const unsigned long long l2 = hfr::launch_count();
  if ((e = cudaStreamBeginCaptureToGraph(sc[1], ifb, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
      cudaSuccess)
    return abort0(e);
  ops.matvec(ops.ctx, x, b.V, sc[1]);  // L x into V0
  (hfr::count_launch(), k_sub<<<nb, KB, 0, sc[1]>>>(t, b.V, b.V, n));
  e = cudaGetLastError();
  {
    cudaGraph_t tmp = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(sc[1], &tmp);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return abort0(e);
  const unsigned long long l3 = hfr::launch_count();
  (hfr::count_launch(), k_gg_start<<<nb, KB, 0, sc[0]>>>(dev, t, b.V, n));
  norm_into(b, 0, b.V, n, 3, rtol, m, sc[0]);  // beta
  (hfr::count_launch(), k_cycle_start<<<nb, KB, 0, sc[0]>>>(st, b.V, n, rtol));
  for (int j = 0; j < m; ++j) {  // every iteration enqueued; those after the cycle's end return at once
    double* vj = b.V + (size_t)j * n;
    double* w = b.V + (size_t)(j + 1) * n;
    double* zj = b.Z + (size_t)j * n;
    ops.precond(ops.ctx, st, j, vj, zj, b.z32, sc[0]);
    ops.gated_matvec(ops.ctx, st, j, zj, b.z32, w, sc[0]);
    (hfr::count_launch(), k_cgs<<<nb, KB, 0, sc[0]>>>(st, j, b.V, n, j + 1, 0, b.V, j + 2, w, b.partial, b.ticket, 5,
                                                       rtol, m, 0));
    (hfr::count_launch(), k_cgs<<<nb, KB, 0, sc[0]>>>(st, j, b.V, n, j + 1, 1, w, 1, w, b.partial, b.ticket, 6, rtol,
                                                       m, 0));
    (hfr::count_launch(), k_cgs<<<nb, KB, 0, sc[0]>>>(st, j, b.V, n, j + 1, 0, b.V, j + 1, w, b.partial, b.ticket, 1,
                                                       rtol, m, 1));
    (hfr::count_launch(), k_cgs<<<nb, KB, 0, sc[0]>>>(st, j, b.V, n, j + 1, 2, w, 1, w, b.partial, b.ticket, 2, rtol,
                                                       m, 1));
  }
  (hfr::count_launch(), k_solve_y<<<1, 32, 0, sc[0]>>>(st));
  (hfr::count_launch(), k_axpy_multi<<<nb, KB, 0, sc[0]>>>(st, 0, b.Z, n, -1, x, 2));
  (hfr::count_launch(), k_gg_after<<<1, 1, 0, sc[0]>>>(dev, st, maxit, hw));
  e = cudaGetLastError();
  {
    cudaGraph_t tmp = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(sc[0], &tmp);
    if (e == cudaSuccess) e = e2;
  }
  const unsigned long long l4 = hfr::launch_count();
  if (counts) {
    counts->fixed = (int)(l1 - l0);
    counts->cycle = (int)((l4 - l3) + (l2 - l1));
    counts->residual = (int)(l3 - l2);
  }
  return e;
}

}  // namespace hfr
