// One restart cycle of right-preconditioned GMRES(m) for the condensed trace system
// L du^ = t (Pereira & Vermeire, arXiv 2401.16632, Sec. 3.2: L = sum_k scatter(S_k) gather_k,
// face-block-Jacobi preconditioner) in a single cooperative launch.
//
// The multi-kernel cycle of hfr_krylov.cu spends most of an iteration launching and draining
// short kernels.  Here one CTA per SM runs the whole cycle: each CTA owns a contiguous range of
// trace faces (and so of every Krylov vector), and the CTAs meet at a grid barrier only where an
// iteration needs data from other faces or a global sum:
//   (A) after z = P^{-1} v_j        (the mat-vec gathers z on neighbouring faces)
//   (B) after w = L z and its dots  (classical Gram-Schmidt coefficients and ||w||)
//   (C) after w -= V h and its dots (second-pass coefficients and ||w||, for the DGKS test)
//   (D) only when the second pass runs: after it, for the new norm
// Every CTA reduces the per-CTA partial sums in the same fixed order, so all CTAs hold bitwise
// identical Hessenberg columns, rotations and convergence decisions and take the same path.
// The barrier waits are bounded: a wait that outlasts PG_TIMEOUT_NS raises an abort flag that the
// host reads, and every CTA leaves at its next barrier.
#include "hfr_krylov.h"

namespace hfr {

namespace {

constexpr int PG_THREADS = 512;
constexpr int PG_WARPS = PG_THREADS / 32;
constexpr int PG_ND = GM_MAXM + 2;  // dots per reduction: j + 2 <= m + 1
constexpr unsigned long long PG_TIMEOUT_NS = 2000000000ull;
constexpr unsigned PG_MAX_SPINS = 1u << 26;

struct PGShared {
  double red[PG_ND][PG_WARPS];
  double dot[PG_ND];
  double H[(GM_MAXM + 1) * GM_MAXM];
  double hc[GM_MAXM + 2];
  double g[GM_MAXM + 1];
  double cs[GM_MAXM], sn[GM_MAXM], y[GM_MAXM];
  double beta, bnorm, inv, res, hn, ww;
  int done, k, conv, nan, ok;
};

__device__ __forceinline__ unsigned long long pg_clock() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned pg_load_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier of a cooperative launch (all CTAs resident).  bar[0] counts arrivals over the
// whole launch (zeroed before it), bar[1] is the abort flag.  Returns false on abort.
__device__ bool pg_sync(PGShared& sh, unsigned* bar, unsigned& epoch) {
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = epoch * gridDim.x;
    __threadfence();
    atomicAdd(bar, 1u);
    const unsigned long long t0 = pg_clock();
    for (unsigned it = 0; pg_load_acquire(bar) < target; ++it) {
      if (pg_load_acquire(bar + 1) != 0u) {
        ok = 0;
        break;
      }
      if (it >= PG_MAX_SPINS || ((it & 63u) == 63u && pg_clock() - t0 > PG_TIMEOUT_NS)) {
        atomicExch(bar + 1, 1u);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    sh.ok = ok;
  }
  __syncthreads();
  return sh.ok != 0;
}

// Warp reduce-scatter of 16 per-lane values: afterwards lane l holds the warp sum of value l >> 1.
__device__ __forceinline__ double pg_scatter16(double (&acc)[16], int lane) {
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
  return acc[0] + __shfl_xor_sync(0xffffffffu, acc[0], 1);
}

// CTA partial of D_i . w over this CTA's entries [x0, x1), i < nd, D_i = V + i n, written to
// partial[i * gridDim.x + blockIdx.x].  Each thread visits the entries x0 + tid + PG_THREADS u,
// the same ones the vector updates of this file give it, so it only re-reads its own writes.
__device__ void pg_block_dots(PGShared& sh, const double* V, size_t n, int nd, const double* w, size_t x0,
                              size_t x1, double* partial) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c0 = 0; c0 < nd; c0 += 16) {
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (size_t x = x0 + threadIdx.x; x < x1; x += PG_THREADS) {
      const double wx = __ldcg(w + x);
#pragma unroll
      for (int q = 0; q < 16; ++q)
        if (c0 + q < nd) acc[q] += __ldcg(V + (size_t)(c0 + q) * n + x) * wx;
    }
    const double s = pg_scatter16(acc, lane);
    const int vi = c0 + (lane >> 1);
    if ((lane & 1) == 0 && vi < nd) sh.red[vi][wid] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nd; i += PG_THREADS) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < PG_WARPS; ++k) t += sh.red[i][k];
    partial[(size_t)i * gridDim.x + blockIdx.x] = t;
  }
}

// CTA partials of ||u||^2 (slot 0) and, if v, ||v||^2 (slot 1)
__device__ void pg_block_sq(PGShared& sh, const double* u, const double* v, size_t x0, size_t x1, double* partial) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double su = 0.0, sv = 0.0;
  for (size_t x = x0 + threadIdx.x; x < x1; x += PG_THREADS) {
    const double a = __ldcg(u + x);
    su += a * a;
    if (v) {
      const double b = __ldcg(v + x);
      sv += b * b;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    su += __shfl_xor_sync(0xffffffffu, su, o);
    sv += __shfl_xor_sync(0xffffffffu, sv, o);
  }
  if (lane == 0) {
    sh.red[0][wid] = su;
    sh.red[1][wid] = sv;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < PG_WARPS; ++k) t += sh.red[threadIdx.x][k];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
}

// After the barrier: sh.dot[i] = sum over CTAs of partial slot i, in the same order everywhere.
__device__ void pg_reduce(PGShared& sh, int nd, const double* partial) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < nd; i += PG_WARPS) {
    double t = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(partial + (size_t)i * gridDim.x + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sh.dot[i] = t;
  }
  __syncthreads();
}

// Rows grp + 4u of (L s)_f for trace face f, in every lane of 8-lane group grp: both neighbours'
// row blocks of S_k against the neighbours' gathered trace values (src in the block precision T,
// or FP64 when SRC_D).  Lanes of a group read consecutive columns of a row.
template <typename T, int NT, int BS, bool SRC_D>
__device__ __forceinline__ void pg_face_rows(const FusedArgs& a, int f, const void* src, T (&acc)[(BS + 3) / 4]) {
  constexpr int CT = (NT + 7) / 8, RU = (BS + 3) / 4;
  // both sides' rows in flight at once when they fit in registers
  constexpr bool BOTH = 2 * RU * CT * (int)sizeof(T) <= 256;
  const int lane = threadIdx.x & 31;
  const int grp = lane >> 3, g8 = lane & 7;
  const T* S = reinterpret_cast<const T*>(a.S);
#pragma unroll
  for (int u = 0; u < RU; ++u) acc[u] = T(0);
#pragma unroll(BOTH ? 2 : 1)
  for (int side = 0; side < 2; ++side) {
    const int e = __ldg(a.sides + f * 4 + side * 2);
    if (e < 0) continue;
    const int fs = __ldg(a.sides + f * 4 + side * 2 + 1);
    T sv[RU][CT];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int i = grp + 4 * u;
      const bool ok = i < BS;
      const T* row = S + ((size_t)e * NT + (size_t)fs * BS + (ok ? i : 0)) * NT;
#pragma unroll
      for (int c = 0; c < CT; ++c) {
        const int l = g8 + 8 * c;
        sv[u][c] = (ok && l < NT) ? __ldg(row + l) : T(0);
      }
    }
    T xv[CT];
#pragma unroll
    for (int c = 0; c < CT; ++c) {
      const int l = g8 + 8 * c;
      T v = T(0);
      if (l < NT) {
        const int fp = l / BS;
        const int tf = __ldg(a.tr_of_c + e * 4 + fp);
        if (tf >= 0) {
          const size_t ix = (size_t)tf * BS + (l - fp * BS);
          v = SRC_D ? T(__ldcg(reinterpret_cast<const double*>(src) + ix))
                    : __ldcg(reinterpret_cast<const T*>(src) + ix);
        }
      }
      xv[c] = v;
    }
#pragma unroll
    for (int u = 0; u < RU; ++u)
#pragma unroll
      for (int c = 0; c < CT; ++c) acc[u] += sv[u][c] * xv[c];
  }
#pragma unroll
  for (int u = 0; u < RU; ++u) {
    acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], 4);
    acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], 2);
    acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], 1);
  }
}

// out_f = t_f - (L src)_f when RES, else (L src)_f, for this CTA's faces (one warp per face)
template <typename T, int NT, int BS, bool SRC_D, bool RES>
__device__ void pg_matvec(const FusedArgs& a, const void* src, double* out, int fb0, int fb1) {
  constexpr int RU = (BS + 3) / 4;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int grp = lane >> 3, g8 = lane & 7;
  for (int f = fb0 + wid; f < fb1; f += PG_WARPS) {
    T acc[RU];
    pg_face_rows<T, NT, BS, SRC_D>(a, f, src, acc);
    if (g8 == 0) {
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const int i = grp + 4 * u;
        if (i < BS) {
          const size_t ix = (size_t)f * BS + i;
          out[ix] = RES ? __ldcg(a.t + ix) - double(acc[u]) : double(acc[u]);
        }
      }
    }
  }
}

// Row r of the face block P_f^{-1} (block precision) into registers, lanes r < BS
template <typename T, int BS>
__device__ __forceinline__ void pg_prow(const T* P, int f, int r, T (&row)[BS]) {
  const T* src = P + ((size_t)f * BS + r) * BS;
  if constexpr (sizeof(T) == 4 && BS % 4 == 0) {
#pragma unroll
    for (int c = 0; c < BS / 4; ++c) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(src) + c);
      row[4 * c] = q.x;
      row[4 * c + 1] = q.y;
      row[4 * c + 2] = q.z;
      row[4 * c + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int c = 0; c < BS; ++c) row[c] = __ldg(src + c);
  }
}

// v_j <- v_j * inv (in place, when scale) and z = P^{-1} v_j in the block precision, one warp per
// face of this CTA, lane r < BS owns row r
template <typename T, int BS>
__device__ void pg_precond(const FusedArgs& a, double* vj, double inv, bool scale, int fb0, int fb1) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const T* P = reinterpret_cast<const T*>(a.Pinv);
  T* z = reinterpret_cast<T*>(a.z);
  const int r = lane < BS ? lane : 0;
  for (int f = fb0 + wid; f < fb1; f += PG_WARPS) {
    const size_t ix = (size_t)f * BS + r;
    double v = 0.0;
    if (lane < BS) {
      v = __ldcg(vj + ix);
      if (scale) {
        v *= inv;
        vj[ix] = v;
      }
    }
    T row[BS];
    pg_prow<T, BS>(P, f, r, row);
    const T vt = T(v);
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < BS; ++c) acc += row[c] * __shfl_sync(0xffffffffu, vt, c);
    if (lane < BS) z[ix] = acc;
  }
}

// x_f += P_f^{-1} (sum_{i<k} y_i V_i)_f in FP64 arithmetic, one warp per face
template <typename T, int BS>
__device__ void pg_update_x(const FusedArgs& a, const PGShared& sh, int k, int fb0, int fb1) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const T* P = reinterpret_cast<const T*>(a.Pinv);
  const int r = lane < BS ? lane : 0;
  for (int f = fb0 + wid; f < fb1; f += PG_WARPS) {
    const size_t ix = (size_t)f * BS + r;
    double u0 = 0.0, u1 = 0.0;
    int i = 0;
    for (; i + 1 < k; i += 2) {
      u0 += sh.y[i] * __ldcg(a.V + (size_t)i * a.n + ix);
      u1 += sh.y[i + 1] * __ldcg(a.V + (size_t)(i + 1) * a.n + ix);
    }
    if (i < k) u0 += sh.y[i] * __ldcg(a.V + (size_t)i * a.n + ix);
    const double u = lane < BS ? u0 + u1 : 0.0;
    T row[BS];
    pg_prow<T, BS>(P, f, r, row);
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < BS; ++c) acc += double(row[c]) * __shfl_sync(0xffffffffu, u, c);
    if (lane < BS) a.x[ix] += acc;
  }
}

// Givens update of Hessenberg column j (sh.hc[0..j+1]); decides the end of the cycle
__device__ void pg_givens(PGShared& sh, int j, double rtol, int m) {
  double* h = sh.hc;
  for (int i = 0; i < j; ++i) {
    const double a = h[i], b = h[i + 1];
    h[i] = sh.cs[i] * a + sh.sn[i] * b;
    h[i + 1] = -sh.sn[i] * a + sh.cs[i] * b;
  }
  const double a = h[j], b = h[j + 1];
  sh.hn = b;
  sh.inv = b != 0.0 ? 1.0 / b : 0.0;
  const double r = sqrt(a * a + b * b);
  double c = 1.0, s = 0.0;
  if (r > 0.0) {
    c = a / r;
    s = b / r;
  }
  sh.cs[j] = c;
  sh.sn[j] = s;
  h[j] = r;
  for (int i = 0; i <= j; ++i) sh.H[i * GM_MAXM + j] = h[i];
  sh.g[j + 1] = -s * sh.g[j];
  sh.g[j] = c * sh.g[j];
  sh.res = fabs(sh.g[j + 1]);
  sh.k = j + 1;
  if (!(sh.res == sh.res)) {
    sh.nan = 1;
    sh.done = 1;
  } else if (sh.res <= rtol * sh.bnorm) {
    sh.conv = 1;
    sh.done = 1;
  } else if (j + 1 >= m || b == 0.0) {
    sh.done = 1;
  }
}

template <typename T, int NT, int BS>
__global__ void __launch_bounds__(PG_THREADS, 1) k_gmres_cycle(const __grid_constant__ FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PGShared& sh = *reinterpret_cast<PGShared*>(smem_raw);
  const int F = a.ntrace;
  const int fb0 = (int)((long long)blockIdx.x * F / gridDim.x);
  const int fb1 = (int)((long long)(blockIdx.x + 1) * F / gridDim.x);
  const size_t n = a.n, x0 = (size_t)fb0 * BS, x1 = (size_t)fb1 * BS;
  const int tid = threadIdx.x;
  unsigned epoch = 0;
  int par = 0;
  const size_t pstride = (size_t)PG_ND * gridDim.x;
  double* V = a.V;

  // r0 = t - L x into V_0 (x = 0: r0 = t); beta = ||r0||, bnorm = ||t||
  if (a.x_zero) {
    for (size_t x = x0 + tid; x < x1; x += PG_THREADS) V[x] = __ldcg(a.t + x);
  } else {
    pg_matvec<T, NT, BS, true, true>(a, a.x, V, fb0, fb1);
  }
  __syncthreads();
  pg_block_sq(sh, V, a.t, x0, x1, a.partial + par * pstride);
  if (!pg_sync(sh, a.bar, epoch)) return;
  pg_reduce(sh, 2, a.partial + par * pstride);
  par ^= 1;
  if (tid == 0) {
    const double beta = sqrt(sh.dot[0]);
    sh.beta = beta;
    sh.bnorm = sqrt(sh.dot[1]);
    sh.g[0] = beta;
    sh.res = beta;
    sh.k = 0;
    sh.conv = 0;
    sh.nan = 0;
    sh.done = 0;
    sh.inv = beta > 0.0 ? 1.0 / beta : 0.0;
    if (!(beta == beta)) {
      sh.nan = 1;
      sh.done = 1;
    } else if (beta <= a.rtol * sh.bnorm || beta == 0.0) {
      sh.conv = 1;
      sh.done = 1;
    }
  }
  __syncthreads();

  for (int j = 0; j < a.m && !sh.done; ++j) {
    double* vj = V + (size_t)j * n;
    double* w = V + (size_t)(j + 1) * n;
    // (A) v_j = w_j / h_{j,j-1} (in place), z = P^{-1} v_j
    pg_precond<T, BS>(a, vj, sh.inv, true, fb0, fb1);
    if (!pg_sync(sh, a.bar, epoch)) return;
    // (B) w = L z and its dots with V_0 .. V_j and itself
    pg_matvec<T, NT, BS, false, false>(a, a.z, w, fb0, fb1);
    __syncthreads();
    double* part = a.partial + par * pstride;
    pg_block_dots(sh, V, n, j + 2, w, x0, x1, part);
    if (!pg_sync(sh, a.bar, epoch)) return;
    pg_reduce(sh, j + 2, part);
    par ^= 1;
    for (int i = tid; i <= j + 1; i += PG_THREADS) {
      if (i <= j)
        sh.hc[i] = sh.dot[i];
      else
        sh.ww = sh.dot[i];
    }
    __syncthreads();
    // (C) first Gram-Schmidt pass, then the dots of its result (second-pass coefficients, norm)
    for (size_t x = x0 + tid; x < x1; x += PG_THREADS) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int i = 0;
      for (; i + 3 <= j; i += 4) {
        s0 += sh.hc[i] * __ldcg(V + (size_t)i * n + x);
        s1 += sh.hc[i + 1] * __ldcg(V + (size_t)(i + 1) * n + x);
        s2 += sh.hc[i + 2] * __ldcg(V + (size_t)(i + 2) * n + x);
        s3 += sh.hc[i + 3] * __ldcg(V + (size_t)(i + 3) * n + x);
      }
      for (; i <= j; ++i) s0 += sh.hc[i] * __ldcg(V + (size_t)i * n + x);
      w[x] = __ldcg(w + x) - ((s0 + s1) + (s2 + s3));
    }
    part = a.partial + par * pstride;
    pg_block_dots(sh, V, n, j + 2, w, x0, x1, part);
    if (!pg_sync(sh, a.bar, epoch)) return;
    pg_reduce(sh, j + 2, part);
    par ^= 1;
    // DGKS: a second pass only when the first removed most of w (same decision in every CTA)
    if (sh.dot[j + 1] < 0.5 * sh.ww) {
      // (D) w -= V d, h += d, new norm
      for (size_t x = x0 + tid; x < x1; x += PG_THREADS) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int i = 0;
        for (; i + 3 <= j; i += 4) {
          s0 += sh.dot[i] * __ldcg(V + (size_t)i * n + x);
          s1 += sh.dot[i + 1] * __ldcg(V + (size_t)(i + 1) * n + x);
          s2 += sh.dot[i + 2] * __ldcg(V + (size_t)(i + 2) * n + x);
          s3 += sh.dot[i + 3] * __ldcg(V + (size_t)(i + 3) * n + x);
        }
        for (; i <= j; ++i) s0 += sh.dot[i] * __ldcg(V + (size_t)i * n + x);
        w[x] = __ldcg(w + x) - ((s0 + s1) + (s2 + s3));
      }
      for (int i = tid; i <= j; i += PG_THREADS) sh.hc[i] += sh.dot[i];
      part = a.partial + par * pstride;
      pg_block_sq(sh, w, nullptr, x0, x1, part);
      if (!pg_sync(sh, a.bar, epoch)) return;
      pg_reduce(sh, 1, part);
      par ^= 1;
      if (tid == 0) sh.hc[j + 1] = sqrt(sh.dot[0]);
    } else if (tid == 0) {
      sh.hc[j + 1] = sqrt(sh.dot[j + 1]);
    }
    __syncthreads();
    if (tid == 0) pg_givens(sh, j, a.rtol, a.m);
    __syncthreads();
  }

  // y = H^{-1} g, x += P^{-1} V y
  const int k = sh.k;
  if (tid == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double s = sh.g[i];
      for (int c = i + 1; c < k; ++c) s -= sh.H[i * GM_MAXM + c] * sh.y[c];
      const double d = sh.H[i * GM_MAXM + i];
      sh.y[i] = d != 0.0 ? s / d : 0.0;
    }
  }
  __syncthreads();
  if (k > 0) pg_update_x<T, BS>(a, sh, k, fb0, fb1);
  if (!pg_sync(sh, a.bar, epoch)) return;
  // true residual ||t - L x|| (V_0 as scratch)
  pg_matvec<T, NT, BS, true, true>(a, a.x, V, fb0, fb1);
  __syncthreads();
  pg_block_sq(sh, V, nullptr, x0, x1, a.partial + par * pstride);
  if (!pg_sync(sh, a.bar, epoch)) return;
  pg_reduce(sh, 1, a.partial + par * pstride);
  if (blockIdx.x == 0 && tid == 0) {
    GmresState* st = a.st;
    st->beta = sqrt(sh.dot[0]);
    st->bnorm = sh.bnorm;
    st->res = sh.res;
    st->hn = sh.hn;
    st->k = k;
    st->kdone = k;
    st->converged = sh.conv;
    st->nan = sh.nan;
  }
}

template <typename T, int NT, int BS>
cudaError_t launch_cycle(const FusedArgs& a, int grid, cudaStream_t s) {
  const size_t smem = sizeof(PGShared);
  cudaError_t e = cudaFuncSetAttribute(k_gmres_cycle<T, NT, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<FusedArgs*>(&a)};
  (hfr::count_launch(),
   e = cudaLaunchCooperativeKernel((const void*)k_gmres_cycle<T, NT, BS>, dim3(grid), dim3(PG_THREADS), args, smem, s));
  return e;
}

template <typename T, int NT, int BS>
int occupancy_of() {
  int nb = 0;
  const size_t smem = sizeof(PGShared);
  if (cudaFuncSetAttribute(k_gmres_cycle<T, NT, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gmres_cycle<T, NT, BS>, PG_THREADS, smem) != cudaSuccess)
    return 0;
  return nb;
}

typedef cudaError_t (*CycleFn)(const FusedArgs&, int, cudaStream_t);

CycleFn pick(int prec_bytes, int nT, int bs, int* occ) {
#define HFR_PG(T_, NT_, BS_)                  \
  if (nT == NT_ && bs == BS_) {               \
    *occ = occupancy_of<T_, NT_, BS_>();      \
    return launch_cycle<T_, NT_, BS_>;        \
  }
  if (prec_bytes == 4) {
    HFR_PG(float, 64, 16)
    HFR_PG(float, 80, 20)
    HFR_PG(float, 48, 12)
  } else {
    HFR_PG(double, 64, 16)
    HFR_PG(double, 80, 20)
    HFR_PG(double, 48, 12)
  }
#undef HFR_PG
  *occ = 0;
  return nullptr;
}

}  // namespace

size_t fused_partial_doubles(int max_blocks) { return (size_t)2 * PG_ND * (size_t)max_blocks; }

int fused_gmres_grid(int prec_bytes, int nT, int bs) {
  int dev = 0, coop = 0, nsm = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (!pick(prec_bytes, nT, bs, &occ) || occ < 1) return 0;
  return nsm;  // one CTA per SM
}

int run_gmres_fused(const FusedArgs& base, int prec_bytes, int grid, double rtol, int restart, int maxit,
                    GmresResult* res, int* timed_out, cudaStream_t s) {
  int occ = 0;
  const int bs = (int)(base.n / (size_t)base.ntrace);
  CycleFn fn = pick(prec_bytes, base.nT, bs, &occ);
  *timed_out = 0;
  if (!fn || grid < 1) return -1;
  const int m = restart > GM_MAXM ? GM_MAXM : (restart < 1 ? 1 : restart);
  FusedArgs a = base;
  a.rtol = rtol;
  if (cudaMemsetAsync(a.x, 0, a.n * sizeof(double), s) != cudaSuccess) return -1;
  int total = 0;
  bool first = true;
  for (;;) {
    a.m = m < maxit - total ? m : maxit - total;
    a.x_zero = first ? 1 : 0;
    first = false;
    if (cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), s) != cudaSuccess) return -1;
    if (fn(a, grid, s) != cudaSuccess) return -1;
    GmresHead hs;
    unsigned flags[2] = {0u, 0u};
    if (cudaMemcpyAsync(&hs, a.st, sizeof(GmresHead), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    if (cudaMemcpyAsync(flags, a.bar, sizeof(flags), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    if (flags[1] != 0u) {
      *timed_out = 1;
      res->iterations = total;
      res->converged = 0;
      res->nan = 0;
      return 0;
    }
    total += hs.k;
    res->bnorm = hs.bnorm;
    res->rel = hs.bnorm > 0.0 ? hs.beta / hs.bnorm : 0.0;
    res->iterations = total;
    res->nan = hs.nan;
    res->converged = hs.converged;
    if (hs.nan || hs.converged || total >= maxit || hs.k == 0) return 0;
  }
}

}  // namespace hfr
