// One restart cycle of right-preconditioned GMRES(m) for the condensed trace system
// L du^ = t (Pereira & Vermeire, arXiv 2401.16632, Sec. 3.2: L = sum_k scatter(S_k) gather_k,
// face-block-Jacobi preconditioner) in a single cooperative launch.
//
// The multi-kernel cycle of hfr_krylov.cu spends most of an iteration launching and draining
// short kernels.  Here one CTA per SM runs the whole cycle: each CTA owns a contiguous range of
// trace faces (and so of every Krylov vector), and the CTAs meet at a grid barrier only where an
// iteration needs data from other faces or a global sum:
//   (A) after z = P^{-1} v_j        (the mat-vec gathers z on neighbouring faces)
//   (B) after w = L z and its dots  (classical Gram-Schmidt coefficients h = V^T w)
//   (C) after w' = w - V h and its dots (second-pass coefficients d = V^T w' and ||w'||)
// Classical Gram-Schmidt is applied twice (CGS2).  The second pass w'' = w' - V d is not a pass
// of its own: its norm follows from ||w''||^2 = ||w'||^2 - ||d||^2 (V orthonormal), and the
// subtraction is folded into the pass that normalises v_{j+1} = w'' / ||w''|| before the next
// preconditioner application.  Only when the second pass removes more than a quarter of
// ||w'||^2 (severe cancellation) is w'' formed and its norm summed explicitly, at one more
// barrier.
// Every CTA reduces the per-CTA partial sums in the same fixed order, so all CTAs hold bitwise
// identical Hessenberg columns, rotations and convergence decisions and take the same path.
// The barrier waits are bounded: a wait that outlasts PG_TIMEOUT_NS raises an abort flag that the
// host reads, and every CTA leaves at its next barrier.
//
// Precision: the Krylov basis, its dots and updates use the block precision T (FP32 in the mixed
// path, where FP64 lanes are 1/64 of the FP32 lanes on this GPU and the GMRES tolerance is loose;
// FP64 in the FP64 path).  The Hessenberg matrix, the Givens rotations, y, the solution du^ and
// the right-hand side stay FP64.  The Givens update of column j-1 (one thread per CTA) runs while
// the other warps finish and precondition v_j, which needs only ||w_j||.
//
// Each CTA reads and writes only its own range of the Krylov vectors, so those accesses go
// through L1; values other CTAs read (z, du^, partial sums) use L2-only loads.  The S blocks,
// re-read by every mat-vec of a cycle, are loaded with an L2 evict-last policy and returned to
// the normal policy when the cycle ends.
#include "hfr_krylov.h"

namespace hfr {

namespace {

constexpr int PG_THREADS = 512;
constexpr int PG_WARPS = PG_THREADS / 32;
constexpr int PG_ND = GM_MAXM + 2;  // dots per reduction: j + 2 <= m + 1
constexpr unsigned long long PG_TIMEOUT_NS = 2000000000ull;
constexpr unsigned PG_MAX_SPINS = 1u << 26;

template <typename T>
struct PGShared {
  T red[PG_ND][PG_WARPS];
  T cf[PG_ND];   // Gram-Schmidt coefficients in the vector precision
  T yT[GM_MAXM];
  T invT;        // 1 / ||w_j||: normalises v_j
  double dot[PG_ND];
  double H[(GM_MAXM + 1) * GM_MAXM];
  double hc[GM_MAXM + 2];
  double g[GM_MAXM + 1];
  double cs[GM_MAXM], sn[GM_MAXM], y[GM_MAXM];
  double rdi[GM_MAXM];  // 1 / H[j][j]
  double beta, bnorm, res, hn;
  int done, k, conv, nan, ok, corr;
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
// whole launch (zeroed before it), bar[1] is the abort flag.  A wait longer than timeout_ns (or
// PG_MAX_SPINS polls) raises the abort flag; a CTA that sees the flag leaves.  Returns false on
// abort.  ok: a shared-memory word of the CTA.
__device__ bool pg_grid_sync(int& ok_shared, unsigned* bar, unsigned& epoch, unsigned long long timeout_ns) {
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = epoch * gridDim.x;
    // release: the CTA's writes (ordered before by the CTA barrier) are visible before the arrival
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    const unsigned long long t0 = pg_clock();
    for (unsigned it = 0; pg_load_acquire(bar) < target; ++it) {
      if ((it & 63u) == 63u) {
        if (pg_load_acquire(bar + 1) != 0u) {
          ok = 0;
          break;
        }
        if (it >= PG_MAX_SPINS || pg_clock() - t0 > timeout_ns) {
          atomicExch(bar + 1, 1u);
          ok = 0;
          break;
        }
      }
      __nanosleep(20);
    }
    ok_shared = ok;
  }
  __syncthreads();
  return ok_shared != 0;
}

template <typename T>
__device__ __forceinline__ bool pg_sync(PGShared<T>& sh, unsigned* bar, unsigned& epoch) {
  return pg_grid_sync(sh.ok, bar, epoch, PG_TIMEOUT_NS);
}

// Self-test of the barrier: `rounds` grid barriers; CTA `absent` (if in range) leaves at once and
// never arrives, so the others' first wait runs out.  passed[0] += barriers each CTA got through.
__global__ void __launch_bounds__(128) k_barrier_probe(unsigned* bar, int absent, int rounds,
                                                       unsigned long long timeout_ns, int* passed) {
  __shared__ int ok;
  if ((int)blockIdx.x == absent) return;
  unsigned epoch = 0;
  int r = 0;
  while (r < rounds && pg_grid_sync(ok, bar, epoch, timeout_ns)) ++r;
  if (threadIdx.x == 0) atomicAdd(passed, r);
}

// Warp reduce-scatter of 16 per-lane values: afterwards lane l holds the warp sum of value l >> 1.
template <typename T>
__device__ __forceinline__ T pg_scatter16(T (&acc)[16], int lane) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const bool up = lane & 16;
    const T send = up ? acc[q] : acc[q + 8];
    const T keep = up ? acc[q + 8] : acc[q];
    acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const bool up = lane & 8;
    const T send = up ? acc[q] : acc[q + 4];
    const T keep = up ? acc[q + 4] : acc[q];
    acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const bool up = lane & 4;
    const T send = up ? acc[q] : acc[q + 2];
    const T keep = up ? acc[q + 2] : acc[q];
    acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const bool up = lane & 2;
    const T send = up ? acc[0] : acc[1];
    const T keep = up ? acc[1] : acc[0];
    acc[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  return acc[0] + __shfl_xor_sync(0xffffffffu, acc[0], 1);
}

// Warp reduce-scatter of 8 per-lane values: afterwards lane l holds the warp sum of value l >> 2.
template <typename T>
__device__ __forceinline__ T pg_scatter8(T (&acc)[8], int lane) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const bool up = lane & 16;
    const T send = up ? acc[q] : acc[q + 4];
    const T keep = up ? acc[q + 4] : acc[q];
    acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const bool up = lane & 8;
    const T send = up ? acc[q] : acc[q + 2];
    const T keep = up ? acc[q + 2] : acc[q];
    acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    const bool up = lane & 4;
    const T send = up ? acc[0] : acc[1];
    const T keep = up ? acc[1] : acc[0];
    acc[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 2);
  return acc[0] + __shfl_xor_sync(0xffffffffu, acc[0], 1);
}

// 16-byte vector of W values of the basis (W = 16 / sizeof(T)), default (L1-allocating) loads
template <typename T, int W>
struct PGV {
  T v[W];
};
template <typename T, int W>
__device__ __forceinline__ PGV<T, W> pg_ldv(const T* p) {
  PGV<T, W> r;
  if constexpr (sizeof(T) == 4 && W == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    r.v[0] = q.x;
    r.v[1] = q.y;
    r.v[2] = q.z;
    r.v[3] = q.w;
  } else if constexpr (sizeof(T) == 8 && W == 2) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    r.v[0] = q.x;
    r.v[1] = q.y;
  } else {
#pragma unroll
    for (int e = 0; e < W; ++e) r.v[e] = p[e];
  }
  return r;
}
// basis vectors per step of the vector dot pass (two W-vectors of each in flight per thread)
constexpr int PG_VC = 4;
// vector width of the dot pass: 16 bytes when face blocks (hence every CTA's range and the vector
// length) are whole vectors, else scalar
template <typename T, int BS>
__host__ __device__ constexpr int pg_basis_width() {
  return BS % (16 / (int)sizeof(T)) == 0 ? 16 / (int)sizeof(T) : 1;
}

// CTA partial of V_i . w over this CTA's entries [x0, x1), i < nd, written to
// partial[i * gridDim.x + blockIdx.x].  Each thread visits the entries x0 + tid + PG_THREADS u,
// the same ones the vector updates of this file give it, so it only re-reads its own writes.
// With W > 1 the thread visits the W-vectors x0 / W + tid + PG_THREADS u instead (two W-vectors of
// w and of PG_VC basis vectors per step, 2 PG_VC + 2 loads of 16 bytes in flight); w's entries are
// then not the thread's own writes, so the caller puts a block barrier between the update of w and
// this pass.
template <typename T, int W = 1>
__device__ void pg_block_dots(PGShared<T>& sh, const T* V, size_t n, int nd, const T* w, size_t x0, size_t x1,
                              T* partial) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if constexpr (W > 1) {
    const size_t g0 = x0 / W, g1 = x1 / W, nW = n / W;
    for (int c0 = 0; c0 < nd; c0 += PG_VC) {
      T acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = T(0);
      for (size_t ga = g0 + threadIdx.x; ga < g1; ga += 2 * PG_THREADS) {
        const size_t gb = ga + PG_THREADS;
        const bool okb = gb < g1;
        const size_t gbs = okb ? gb : ga;
        const PGV<T, W> wa = pg_ldv<T, W>(w + ga * W);
        PGV<T, W> wb = pg_ldv<T, W>(w + gbs * W);
        if (!okb) {
#pragma unroll
          for (int e = 0; e < W; ++e) wb.v[e] = T(0);
        }
        PGV<T, W> va[PG_VC], vb[PG_VC];
#pragma unroll
        for (int q = 0; q < PG_VC; ++q)
          if (c0 + q < nd) {
            va[q] = pg_ldv<T, W>(V + ((size_t)(c0 + q) * nW + ga) * W);
            vb[q] = pg_ldv<T, W>(V + ((size_t)(c0 + q) * nW + gbs) * W);
          }
#pragma unroll
        for (int q = 0; q < PG_VC; ++q)
          if (c0 + q < nd) {
#pragma unroll
            for (int e = 0; e < W; ++e) acc[q] += va[q].v[e] * wa.v[e] + vb[q].v[e] * wb.v[e];
          }
      }
      const T s = pg_scatter8(acc, lane);
      const int vi = c0 + (lane >> 2);
      if ((lane & 3) == 0 && vi < nd) sh.red[vi][wid] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nd; i += PG_THREADS) {
      T t = T(0);
#pragma unroll
      for (int k = 0; k < PG_WARPS; ++k) t += sh.red[i][k];
      partial[(size_t)i * gridDim.x + blockIdx.x] = t;
    }
  } else {
    for (int c0 = 0; c0 < nd; c0 += 16) {
      T acc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = T(0);
      // two entries per iteration: 34 independent loads in flight per thread
      for (size_t xa = x0 + threadIdx.x; xa < x1; xa += 2 * PG_THREADS) {
        const size_t xb = xa + PG_THREADS;
        const bool okb = xb < x1;
        const T wa = w[xa];
        const T wb = okb ? w[xb] : T(0);
        const size_t xbs = okb ? xb : xa;
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (c0 + q < nd) {
            const T va = V[(size_t)(c0 + q) * n + xa];
            const T vb = V[(size_t)(c0 + q) * n + xbs];
            acc[q] += va * wa + vb * wb;
          }
      }
      const T s = pg_scatter16(acc, lane);
      const int vi = c0 + (lane >> 1);
      if ((lane & 1) == 0 && vi < nd) sh.red[vi][wid] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nd; i += PG_THREADS) {
      T t = T(0);
#pragma unroll
      for (int k = 0; k < PG_WARPS; ++k) t += sh.red[i][k];
      partial[(size_t)i * gridDim.x + blockIdx.x] = t;
    }
  }
}

// CTA partials of ||u||^2 (slot 0) and, if v, ||v||^2 (slot 1), in the vector precision
template <typename T, typename U2>
__device__ void pg_block_sq(PGShared<T>& sh, const T* u, const U2* v, size_t x0, size_t x1, T* partial) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T su = T(0), sv = T(0);
  for (size_t x = x0 + threadIdx.x; x < x1; x += PG_THREADS) {
    const T a = u[x];
    su += a * a;
    if (v) {
      const T b = T(__ldcg(v + x));
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
    T t = T(0);
#pragma unroll
    for (int k = 0; k < PG_WARPS; ++k) t += sh.red[threadIdx.x][k];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
}

// After the barrier: sh.dot[i] = sum over CTAs of partial slot i, in the same order everywhere.
template <typename T>
__device__ void pg_reduce(PGShared<T>& sh, int nd, const T* partial) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nb = (int)gridDim.x;
  for (int i = wid; i < nd; i += PG_WARPS) {
    const T* pi = partial + (size_t)i * nb;
    T t = T(0);
    for (int b0 = 0; b0 < nb; b0 += 32 * 8) {
      T v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int b = b0 + lane + 32 * q;
        v[q] = b < nb ? __ldcg(pi + b) : T(0);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) t += v[q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sh.dot[i] = double(t);
  }
  __syncthreads();
}

// Vector loads of VW consecutive values.  The S blocks are read with an L2 evict-last policy so
// that they stay resident in L2 across the iterations of a cycle (they are the largest operand and
// are re-read by every mat-vec); everything else uses the default policy.
template <typename T, int VW>
struct PGVec {
  T v[VW];
};

__device__ __forceinline__ unsigned long long pg_policy_keep() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

template <typename T, int VW>
__device__ __forceinline__ PGVec<T, VW> pg_ld_keep(const T* ptr, unsigned long long pol) {
  PGVec<T, VW> r;
  if constexpr (sizeof(T) == 4 && VW == 4) {
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3])
        : "l"(ptr), "l"(pol));
  } else if constexpr (sizeof(T) == 4 && VW == 2) {
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(r.v[0]), "=f"(r.v[1]) : "l"(ptr), "l"(pol));
  } else if constexpr (sizeof(T) == 8 && VW == 2) {
    asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(r.v[0]), "=d"(r.v[1]) : "l"(ptr), "l"(pol));
  } else {
#pragma unroll
    for (int q = 0; q < VW; ++q) r.v[q] = __ldg(ptr + q);
  }
  return r;
}

// VW consecutive BF16 values (the trace operator stored in BF16) widened to FP32, with the same
// evict-last policy; BF16 is the upper half of an FP32 word, so widening is a 16-bit shift
template <int VW>
__device__ __forceinline__ PGVec<float, VW> pg_ld_keep_bf16(const unsigned short* ptr, unsigned long long pol) {
  PGVec<float, VW> r;
  if constexpr (VW == 4) {
    unsigned a, b;
    asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(a), "=r"(b) : "l"(ptr), "l"(pol));
    r.v[0] = __uint_as_float(a << 16);
    r.v[1] = __uint_as_float(a & 0xffff0000u);
    r.v[2] = __uint_as_float(b << 16);
    r.v[3] = __uint_as_float(b & 0xffff0000u);
  } else if constexpr (VW == 2) {
    unsigned a;
    asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(a) : "l"(ptr), "l"(pol));
    r.v[0] = __uint_as_float(a << 16);
    r.v[1] = __uint_as_float(a & 0xffff0000u);
  } else {
#pragma unroll
    for (int q = 0; q < VW; ++q) r.v[q] = __uint_as_float((unsigned)__ldg(ptr + q) << 16);
  }
  return r;
}

template <typename T, int VW>
__device__ __forceinline__ PGVec<T, VW> pg_ld_cg(const T* ptr) {
  PGVec<T, VW> r;
  if constexpr (sizeof(T) == 4 && VW == 4) {
    const float4 q = __ldcg(reinterpret_cast<const float4*>(ptr));
    r.v[0] = q.x;
    r.v[1] = q.y;
    r.v[2] = q.z;
    r.v[3] = q.w;
  } else if constexpr (sizeof(T) == 4 && VW == 2) {
    const float2 q = __ldcg(reinterpret_cast<const float2*>(ptr));
    r.v[0] = q.x;
    r.v[1] = q.y;
  } else if constexpr (sizeof(T) == 8 && VW == 2) {
    const double2 q = __ldcg(reinterpret_cast<const double2*>(ptr));
    r.v[0] = q.x;
    r.v[1] = q.y;
  } else {
#pragma unroll
    for (int q = 0; q < VW; ++q) r.v[q] = __ldcg(ptr + q);
  }
  return r;
}

// widest vector (16 bytes at most) that divides both the per-lane column count and the face block
template <typename T, int NT, int BS>
struct PGShape {
  static constexpr int CT = NT / 8;  // columns per lane
  static constexpr int VMAX = 16 / (int)sizeof(T);
  static constexpr int VW = (CT % 4 == 0 && BS % 4 == 0 && VMAX >= 4) ? 4 : ((CT % 2 == 0 && BS % 2 == 0) ? 2 : 1);
  static constexpr int CV = CT / VW;  // vectors per lane and row
  static constexpr int RU = (BS + 3) / 4;
  static_assert(NT % 8 == 0, "nT must be a multiple of 8");
};

// Rows grp + 4u of (L s)_f for trace face f, in every lane of 8-lane group grp: both neighbours'
// row blocks of S_k against the neighbours' gathered trace values (src in the block precision T,
// or FP64 when SRC_D).  Lane g8 of a group holds the columns VW (g8 + 8 c) + q of each row, so
// every load is a VW-wide vector and no vector crosses a face block.
template <typename T, int NT, int BS, bool SRC_D, bool SB>
__device__ __forceinline__ void pg_face_rows(const FusedArgs& a, int f, const void* src, unsigned long long pol,
                                             T (&acc)[(BS + 3) / 4]) {
  using Sh = PGShape<T, NT, BS>;
  constexpr int VW = Sh::VW, CV = Sh::CV, RU = Sh::RU;
  // both sides' rows in flight at once when they fit in registers
  constexpr bool BOTH = 2 * RU * CV * VW * (int)sizeof(T) <= 256;
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
    PGVec<T, VW> sv[RU][CV];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int i = grp + 4 * u;
      const int ii = i < BS ? i : 0;
      const size_t ro = ((size_t)e * NT + (size_t)fs * BS + ii) * NT;
      if constexpr (SB) {
        const unsigned short* row = reinterpret_cast<const unsigned short*>(a.S) + ro;
#pragma unroll
        for (int c = 0; c < CV; ++c) {
          const PGVec<float, VW> x = pg_ld_keep_bf16<VW>(row + VW * (g8 + 8 * c), pol);
#pragma unroll
          for (int q = 0; q < VW; ++q) sv[u][c].v[q] = T(x.v[q]);
        }
      } else {
        const T* row = S + ro;
#pragma unroll
        for (int c = 0; c < CV; ++c) sv[u][c] = pg_ld_keep<T, VW>(row + VW * (g8 + 8 * c), pol);
      }
    }
    PGVec<T, VW> xv[CV];
#pragma unroll
    for (int c = 0; c < CV; ++c) {
      const int l = VW * (g8 + 8 * c);
      const int fp = l / BS;
      const int tf = __ldg(a.tr_of_c + e * 4 + fp);
      const size_t ix = (size_t)(tf >= 0 ? tf : 0) * BS + (l - fp * BS);
      if (SRC_D) {
        const PGVec<double, VW> d = pg_ld_cg<double, VW>(reinterpret_cast<const double*>(src) + ix);
#pragma unroll
        for (int q = 0; q < VW; ++q) xv[c].v[q] = tf >= 0 ? T(d.v[q]) : T(0);
      } else {
        xv[c] = pg_ld_cg<T, VW>(reinterpret_cast<const T*>(src) + ix);
        if (tf < 0) {
#pragma unroll
          for (int q = 0; q < VW; ++q) xv[c].v[q] = T(0);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      if (grp + 4 * u < BS) {
#pragma unroll
        for (int c = 0; c < CV; ++c)
#pragma unroll
          for (int q = 0; q < VW; ++q) acc[u] += sv[u][c].v[q] * xv[c].v[q];
      }
    }
  }
#pragma unroll
  for (int u = 0; u < RU; ++u) {
    acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], 4);
    acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], 2);
    acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], 1);
  }
}

// out_f = t_f - (L src)_f when RES, else (L src)_f, for this CTA's faces (one warp per face),
// stored in the vector precision T
template <typename T, int NT, int BS, bool SRC_D, bool RES, bool SB>
__device__ void pg_matvec(const FusedArgs& a, const void* src, T* out, int fb0, int fb1) {
  constexpr int RU = (BS + 3) / 4;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int grp = lane >> 3, g8 = lane & 7;
  const unsigned long long pol = pg_policy_keep();
  for (int f = fb0 + wid; f < fb1; f += PG_WARPS) {
    T acc[RU];
    pg_face_rows<T, NT, BS, SRC_D, SB>(a, f, src, pol, acc);
    if (g8 == 0) {
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const int i = grp + 4 * u;
        if (i < BS) {
          const size_t ix = (size_t)f * BS + i;
          out[ix] = RES ? T(__ldcg(a.t + ix) - double(acc[u])) : acc[u];
        }
      }
    }
  }
}

// Row r of the face block P_f^{-1} (block precision) into registers
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

// z = P^{-1} v_j, one warp per face of this CTA (two faces per step), lane r < BS owns row r.
// Warp 0 takes no face: its lane 0 updates the Givens rotations meanwhile.
template <typename T, int BS>
__device__ void pg_precond(const FusedArgs& a, const T* vj, int fb0, int fb1) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid == 0) return;
  const T* P = reinterpret_cast<const T*>(a.Pinv);
  T* z = reinterpret_cast<T*>(a.z);
  const int r = lane < BS ? lane : 0;
  constexpr int NW = PG_WARPS - 1;
  for (int f = fb0 + wid - 1; f < fb1; f += 2 * NW) {
    // two faces per step: both blocks' loads in flight together
    const int f2 = f + NW;
    const bool two = f2 < fb1;
    const size_t ix = (size_t)f * BS + r, ix2 = (size_t)(two ? f2 : f) * BS + r;
    const T v = lane < BS ? vj[ix] : T(0);
    const T v2 = lane < BS ? vj[ix2] : T(0);
    T row[BS], row2[BS];
    pg_prow<T, BS>(P, f, r, row);
    pg_prow<T, BS>(P, two ? f2 : f, r, row2);
    T acc = T(0), acc2 = T(0);
#pragma unroll
    for (int c = 0; c < BS; ++c) {
      acc += row[c] * __shfl_sync(0xffffffffu, v, c);
      acc2 += row2[c] * __shfl_sync(0xffffffffu, v2, c);
    }
    if (lane < BS) {
      z[ix] = acc;
      if (two) z[ix2] = acc2;
    }
  }
}

// dst[x] = (dst[x] - sum_{i<cnt} c_i V_i[x]) * scale over the entries x0 + tid0 + m nthreads of this
// thread; four entries per iteration and two basis vectors per inner step keep eight independent
// loads in flight per thread (the basis of a large system streams from HBM)
template <typename T>
__device__ __forceinline__ void pg_axpy_multi(const T* V, size_t n, const T* c, int cnt, T* dst, T scale,
                                              size_t x0, size_t x1, int tid0, int nthreads) {
  const size_t st = (size_t)nthreads;
  for (size_t xb = x0 + tid0; xb < x1; xb += 4 * st) {
    size_t xs[4];
    bool ok[4];
    T sacc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      xs[u] = xb + u * st;
      ok[u] = xs[u] < x1;
      if (!ok[u]) xs[u] = xb;
      sacc[u] = T(0);
    }
    int i = 0;
    for (; i + 2 <= cnt; i += 2) {
      const T ca = c[i], cb = c[i + 1];
      const T* Va = V + (size_t)i * n;
      const T* Vb = Va + n;
#pragma unroll
      for (int u = 0; u < 4; ++u) sacc[u] += ca * Va[xs[u]] + cb * Vb[xs[u]];
    }
    if (i < cnt) {
      const T ca = c[i];
      const T* Va = V + (size_t)i * n;
#pragma unroll
      for (int u = 0; u < 4; ++u) sacc[u] += ca * Va[xs[u]];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (ok[u]) dst[xs[u]] = (dst[xs[u]] - sacc[u]) * scale;
  }
}

// v_j <- (v_j - sum_{i<jc} c_i V_i) * inv over this CTA's entries, by warps 1.. only (jc = 0: scale)
template <typename T>
__device__ void pg_finish(const T* V, size_t n, const T* c, int jc, T inv, T* vj, size_t x0, size_t x1) {
  if (threadIdx.x < 32) return;
  pg_axpy_multi(V, n, c, jc, vj, inv, x0, x1, (int)threadIdx.x - 32, PG_THREADS - 32);
}

// named barrier of warps 1 .. PG_WARPS-1 (warp 0 is busy with the Givens update)
__device__ __forceinline__ void pg_sync_workers() {
  asm volatile("bar.sync 1, %0;" ::"n"(PG_THREADS - 32) : "memory");
}

// x_f += P_f^{-1} (sum_{i<k} y_i V_i)_f: first u = V y over this CTA's entries into the z buffer
// (free at the end of the cycle; a streaming pass with many loads in flight), then P_f^{-1} u_f in
// the vector precision added to the FP64 solution, one warp per face
template <typename T, int BS>
__device__ void pg_update_x(const FusedArgs& a, const PGShared<T>& sh, const T* V, int k, int fb0, int fb1) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const T* P = reinterpret_cast<const T*>(a.Pinv);
  T* u = reinterpret_cast<T*>(a.z);
  const size_t x0 = (size_t)fb0 * BS, x1 = (size_t)fb1 * BS;
  for (size_t x = x0 + threadIdx.x; x < x1; x += PG_THREADS) u[x] = T(0);
  __syncthreads();
  pg_axpy_multi(V, a.n, sh.yT, k, u, T(-1), x0, x1, (int)threadIdx.x, PG_THREADS);
  __syncthreads();
  const int r = lane < BS ? lane : 0;
  for (int f = fb0 + wid; f < fb1; f += PG_WARPS) {
    const size_t ix = (size_t)f * BS + r;
    const T uv = lane < BS ? u[ix] : T(0);
    T row[BS];
    pg_prow<T, BS>(P, f, r, row);
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < BS; ++c) acc += row[c] * __shfl_sync(0xffffffffu, uv, c);
    if (lane < BS) a.x[ix] += double(acc);
  }
}

template <typename T>
__device__ __forceinline__ void pg_subtract(const T* V, size_t n, const T* c, int j, T* w, size_t x0, size_t x1) {
  pg_axpy_multi(V, n, c, j + 1, w, T(1), x0, x1, (int)threadIdx.x, PG_THREADS);
}

// Givens update of Hessenberg column j (sh.hc[0..j+1]), FP64; decides the end of the cycle
template <typename T>
__device__ void pg_givens(PGShared<T>& sh, int j, double rtol, int m) {
  double* h = sh.hc;
  for (int i = 0; i < j; ++i) {
    const double a = h[i], b = h[i + 1];
    h[i] = sh.cs[i] * a + sh.sn[i] * b;
    h[i + 1] = -sh.sn[i] * a + sh.cs[i] * b;
  }
  const double a = h[j], b = h[j + 1];
  sh.hn = b;
  const double r = sqrt(a * a + b * b);
  const double ri = r > 0.0 ? 1.0 / r : 0.0;
  double c = 1.0, s = 0.0;
  if (r > 0.0) {
    c = a * ri;
    s = b * ri;
  }
  sh.cs[j] = c;
  sh.sn[j] = s;
  sh.rdi[j] = ri;
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

template <typename T, int NT, int BS, bool SB>
__global__ void __launch_bounds__(PG_THREADS, 1) k_gmres_cycle(const __grid_constant__ FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PGShared<T>& sh = *reinterpret_cast<PGShared<T>*>(smem_raw);
  const int F = a.ntrace;
  const int fb0 = (int)((long long)blockIdx.x * F / gridDim.x);
  const int fb1 = (int)((long long)(blockIdx.x + 1) * F / gridDim.x);
  const size_t n = a.n, x0 = (size_t)fb0 * BS, x1 = (size_t)fb1 * BS;
  constexpr int VWB = pg_basis_width<T, BS>();
  const int tid = threadIdx.x;
  unsigned epoch = 0;
  int par = 0;
  const size_t pstride = (size_t)PG_ND * gridDim.x;
  T* V = reinterpret_cast<T*>(a.V);
  T* const partial = reinterpret_cast<T*>(a.partial);

  const int xz = a.dyn ? a.dyn[0] : a.x_zero;
  const int mm = a.dyn ? a.dyn[1] : a.m;
  // r0 = t - L x into V_0 (x = 0: r0 = t); beta = ||r0||, bnorm = ||t||
  if (xz) {
    for (size_t x = x0 + tid; x < x1; x += PG_THREADS) V[x] = T(__ldcg(a.t + x));
  } else {
    pg_matvec<T, NT, BS, true, true, SB>(a, a.x, V, fb0, fb1);
  }
  __syncthreads();
  pg_block_sq(sh, V, a.t, x0, x1, partial + par * pstride);
  if (!pg_sync(sh, a.bar, epoch)) return;
  pg_reduce(sh, 2, partial + par * pstride);
  par ^= 1;
  if (tid == 0) {
    const double beta = sqrt(sh.dot[0]);
    sh.beta = beta;
    sh.bnorm = sqrt(sh.dot[1]);
    sh.g[0] = beta;
    sh.res = beta;
    sh.hn = beta;
    sh.k = 0;
    sh.conv = 0;
    sh.nan = 0;
    sh.done = 0;
    sh.corr = 0;
    sh.invT = T(beta > 0.0 ? 1.0 / beta : 0.0);
    if (!(beta == beta)) {
      sh.nan = 1;
      sh.done = 1;
    } else if (beta <= a.rtol * sh.bnorm || beta == 0.0) {
      sh.conv = 1;
      sh.done = 1;
    }
  }
  __syncthreads();

  if (!sh.done) {
    for (int j = 0;; ++j) {
      T* vj = V + (size_t)j * n;
      T* w = V + (size_t)(j + 1) * n;
      // (A) lane 0 of warp 0: Givens rotation of column j-1.  Warps 1..: finish v_j (deferred
      // second Gram-Schmidt pass, normalisation) and form z = P^{-1} v_j.
      if (j > 0 && tid == 0) pg_givens(sh, j - 1, a.rtol, mm);
      if (tid >= 32) {
        pg_finish(V, n, sh.cf, sh.corr ? j : 0, sh.invT, vj, x0, x1);
        pg_sync_workers();
        pg_precond<T, BS>(a, vj, fb0, fb1);
      }
      if (!pg_sync(sh, a.bar, epoch)) return;
      if (sh.done) break;
      // (B) w = L z and h = V^T w
      pg_matvec<T, NT, BS, false, false, SB>(a, a.z, w, fb0, fb1);
      __syncthreads();
      T* part = partial + par * pstride;
      pg_block_dots<T, VWB>(sh, V, n, j + 1, w, x0, x1, part);
      if (!pg_sync(sh, a.bar, epoch)) return;
      pg_reduce(sh, j + 1, part);
      par ^= 1;
      for (int i = tid; i <= j; i += PG_THREADS) {
        sh.hc[i] = sh.dot[i];
        sh.cf[i] = T(sh.dot[i]);
      }
      __syncthreads();
      // (C) w' = w - V h, then d = V^T w' and ||w'||^2 (dot j+1: V_{j+1} is w' itself)
      pg_subtract(V, n, sh.cf, j, w, x0, x1);
      if (VWB > 1) __syncthreads();  // the dot pass visits w in its own (vector) order
      part = partial + par * pstride;
      pg_block_dots<T, VWB>(sh, V, n, j + 2, w, x0, x1, part);
      if (!pg_sync(sh, a.bar, epoch)) return;
      pg_reduce(sh, j + 2, part);
      par ^= 1;
      if (tid < 32) {
        // ||d||^2 (fixed order), h += d, coefficients of the deferred pass
        double dd = 0.0;
        for (int i = tid; i <= j; i += 32) {
          const double d = sh.dot[i];
          dd += d * d;
          sh.hc[i] += d;
          sh.cf[i] = T(d);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
        if (tid == 0) {
          const double n1 = sh.dot[j + 1];
          sh.corr = dd <= 0.25 * n1 ? 1 : 0;
          if (sh.corr) sh.hc[j + 1] = sqrt(n1 - dd);
        }
      }
      __syncthreads();
      if (!sh.corr) {
        // severe cancellation: form w'' = w' - V d now and sum its norm
        pg_subtract(V, n, sh.cf, j, w, x0, x1);
        part = partial + par * pstride;
        pg_block_sq(sh, w, (const T*)nullptr, x0, x1, part);
        if (!pg_sync(sh, a.bar, epoch)) return;
        pg_reduce(sh, 1, part);
        par ^= 1;
        if (tid == 0) sh.hc[j + 1] = sqrt(sh.dot[0]);
      }
      if (tid == 0) sh.invT = T(sh.hc[j + 1] != 0.0 ? 1.0 / sh.hc[j + 1] : 0.0);
      __syncthreads();
    }
  }

  // y = H^{-1} g, x += P^{-1} V y
  const int k = sh.k;
  if (tid == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double s = sh.g[i];
      for (int c = i + 1; c < k; ++c) s -= sh.H[i * GM_MAXM + c] * sh.y[c];
      sh.y[i] = s * sh.rdi[i];
      sh.yT[i] = T(sh.y[i]);
    }
  }
  __syncthreads();
  if (k > 0) pg_update_x<T, BS>(a, sh, V, k, fb0, fb1);
  if (a.true_res) {
    // true residual ||t - L x|| (V_0 as scratch)
    if (!pg_sync(sh, a.bar, epoch)) return;
    pg_matvec<T, NT, BS, true, true, SB>(a, a.x, V, fb0, fb1);
    __syncthreads();
    pg_block_sq(sh, V, (const T*)nullptr, x0, x1, partial + par * pstride);
    if (!pg_sync(sh, a.bar, epoch)) return;
    pg_reduce(sh, 1, partial + par * pstride);
  }
  // the S blocks go back to the normal L2 eviction policy (the next condensation rewrites them)
  for (size_t off = ((size_t)blockIdx.x * PG_THREADS + tid) * 128; off < a.S_bytes;
       off += (size_t)gridDim.x * PG_THREADS * 128)
    asm volatile("applypriority.global.L2::evict_normal [%0], 128;" ::"l"(reinterpret_cast<const char*>(a.S) + off)
                 : "memory");
  if (blockIdx.x == 0 && tid == 0) {
    GmresState* st = a.st;
    st->beta = a.true_res ? sqrt(sh.dot[0]) : sh.res;
    st->bnorm = sh.bnorm;
    st->res = sh.res;
    st->hn = sh.hn;
    st->k = k;
    st->kdone = k;
    st->converged = sh.conv;
    st->nan = sh.nan;
  }
}

template <typename T, int NT, int BS, bool SB>
cudaError_t launch_cycle(const FusedArgs& a, int grid, cudaStream_t s) {
  const size_t smem = sizeof(PGShared<T>);
  cudaError_t e = cudaFuncSetAttribute(k_gmres_cycle<T, NT, BS, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<FusedArgs*>(&a)};
  (hfr::count_launch(),
   e = cudaLaunchCooperativeKernel((const void*)k_gmres_cycle<T, NT, BS, SB>, dim3(grid), dim3(PG_THREADS), args, smem, s));
  return e;
}

template <typename T, int NT, int BS, bool SB>
int occupancy_of() {
  int nb = 0;
  const size_t smem = sizeof(PGShared<T>);
  if (cudaFuncSetAttribute(k_gmres_cycle<T, NT, BS, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gmres_cycle<T, NT, BS, SB>, PG_THREADS, smem) != cudaSuccess)
    return 0;
  return nb;
}

typedef cudaError_t (*CycleFn)(const FusedArgs&, int, cudaStream_t);

// s_bf16: the trace operator S is stored in BF16 (FP32 blocks, basis and arithmetic otherwise)
CycleFn pick(int prec_bytes, int nT, int bs, int* occ, bool s_bf16 = false) {
#define HFR_PG(T_, NT_, BS_, SB_)                  \
  if (nT == NT_ && bs == BS_) {                    \
    *occ = occupancy_of<T_, NT_, BS_, SB_>();      \
    return launch_cycle<T_, NT_, BS_, SB_>;        \
  }
  if (prec_bytes == 4 && s_bf16) {
    HFR_PG(float, 64, 16, true)
    HFR_PG(float, 80, 20, true)
    HFR_PG(float, 48, 12, true)
  } else if (prec_bytes == 4) {
    HFR_PG(float, 64, 16, false)
    HFR_PG(float, 80, 20, false)
    HFR_PG(float, 48, 12, false)
  } else {
    HFR_PG(double, 64, 16, false)
    HFR_PG(double, 80, 20, false)
    HFR_PG(double, 48, 12, false)
  }
#undef HFR_PG
  *occ = 0;
  return nullptr;
}

}  // namespace

size_t fused_partial_doubles(int max_blocks) { return (size_t)2 * PG_ND * (size_t)max_blocks; }  // >= T slots

int fused_gmres_grid(int prec_bytes, int nT, int bs) {
  int dev = 0, coop = 0, nsm = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (!pick(prec_bytes, nT, bs, &occ) || occ < 1) return 0;
  return nsm;  // one CTA per SM
}

int run_gmres_fused(const FusedArgs& base, int prec_bytes, int grid, double rtol, int restart, int maxit,
                    GmresResult* res, int* timed_out, cudaStream_t s, const int* dev_status, int* host_status) {
  int occ = 0;
  const int bs = (int)(base.n / (size_t)base.ntrace);
  CycleFn fn = pick(prec_bytes, base.nT, bs, &occ, base.s_bf16 != 0);
  *timed_out = 0;
  if (!fn || grid < 1) return -1;
  const int m = restart > GM_MAXM ? GM_MAXM : (restart < 1 ? 1 : restart);
  FusedArgs a = base;
  a.rtol = rtol;
  if (cudaMemsetAsync(a.x, 0, a.n * sizeof(double), s) != cudaSuccess) return -1;
  int total = 0;
  bool first = true, first_cycle = true;
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
    if (dev_status && first_cycle &&
        cudaMemcpyAsync(host_status, dev_status, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return -1;
    first_cycle = false;
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

cudaError_t launch_gmres_cycle(const FusedArgs& a, int prec_bytes, int grid, cudaStream_t s) {
  int occ = 0;
  const int bs = (int)(a.n / (size_t)(a.ntrace > 0 ? a.ntrace : 1));
  CycleFn fn = pick(prec_bytes, a.nT, bs, &occ, a.s_bf16 != 0);
  if (!fn || grid < 1) return cudaErrorInvalidValue;
  return fn(a, grid, s);
}

// Host side of the barrier self-test (declared in hfr_krylov.h).
int barrier_selftest(int nblocks, int absent, int rounds, double timeout_s, int* passed, int* timed_out,
                     cudaStream_t s) {
  *passed = 0;
  *timed_out = 0;
  int dev = 0, nsm = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_barrier_probe, 128, 0) != cudaSuccess) return -1;
  if (!coop || nblocks < 1 || nblocks > nsm * per_sm || rounds < 0) return -2;
  unsigned* bar = nullptr;
  int* dpass = nullptr;
  if (cudaMalloc((void**)&bar, 2 * sizeof(unsigned) + sizeof(int)) != cudaSuccess) return -1;
  dpass = reinterpret_cast<int*>(bar + 2);
  int rc = 0;
  unsigned flags[2] = {0u, 0u};
  unsigned long long tns = (unsigned long long)(timeout_s * 1e9);
  void* args[] = {&bar, &absent, &rounds, &tns, &dpass};
  if (cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned) + sizeof(int), s) != cudaSuccess ||
      cudaLaunchCooperativeKernel((const void*)k_barrier_probe, dim3(nblocks), dim3(128), args, 0, s) != cudaSuccess ||
      cudaMemcpyAsync(flags, bar, sizeof(flags), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(passed, dpass, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    rc = -1;
  cudaStreamSynchronize(s);
  cudaFree(bar);
  *timed_out = flags[1] != 0u;
  return rc;
}

}  // namespace hfr
