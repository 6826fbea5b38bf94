// GMRES driver interface (internal).
#pragma once

#include "hfr_internal.h"

namespace hfr {

constexpr int GM_MAXM = 64;
constexpr int GM_NBLK = 608;  // four blocks per SM for the vector passes

// scalars first: the host reads only the head (sizeof(GmresHead)) between iterations
struct GmresHead {
  double beta, bnorm, res, hn;
  int k, kdone, converged, nan;
};
struct GmresState {
  double beta, bnorm, res, hn;
  int k, kdone, converged, nan;
  double inv_hn;     // 1 / hn, used to normalise the next Krylov vector
  double wnorm_old;  // ||w|| before orthogonalisation (re-orthogonalisation test)
  int reorth;        // 1 when the current column needs a second Gram-Schmidt pass
  double H[(GM_MAXM + 1) * GM_MAXM];
  double g[GM_MAXM + 1];
  double cs[GM_MAXM], sn[GM_MAXM];
  double hc[GM_MAXM + 1];
  double h2[GM_MAXM + 1];
  double y[GM_MAXM];
};

// operator callbacks (enqueue only)
struct GmresOps {
  void* ctx;
  void (*matvec)(void* ctx, const double* x, double* y, cudaStream_t s);
  void (*gated_matvec)(void* ctx, const GmresState* st, int j, const double* x, const float* x32, double* y,
                       cudaStream_t s);
  // z = P^{-1} v_j (and its FP32 copy when z32 != null); for j > 0 it first normalises v_j in
  // place by st->inv_hn = 1 / h_{j,j-1}
  void (*precond)(void* ctx, const GmresState* st, int j, double* v, double* z, float* z32, cudaStream_t s);
};

struct GmresBuffers {
  size_t n;
  double* V;        // (GM_MAXM + 1) x n
  double* Z;        // GM_MAXM x n
  float* z32;       // n: FP32 copy of the current preconditioned vector (FP32 mat-vec), or null
  double* partial;  // GM_NBLK x (GM_MAXM + 1)
  unsigned int* ticket;  // zero-initialised completion counter of the reduction kernels
  GmresState* state;
};

struct GmresResult {
  int iterations;
  int converged;
  int nan;
  double rel;
  double bnorm;
};

// One restart cycle per cooperative launch (hfr_gmres_fused.cu): fixed shapes (nT, bs) in
// {(64,16), (80,20), (48,12)} of either block precision.
struct FusedArgs {
  int ntrace, nT;
  const int* sides;    // ntrace x 4 (e0, f0, e1, f1), compact implicit element ids
  const int* tr_of_c;  // Eim x 4 trace face of each element face
  const void* S;       // Eim x nT x nT, block precision (BF16 when s_bf16)
  size_t S_bytes;      // size of S
  int s_bf16 = 0;      // 1: S holds BF16 values (FP32 path only)
  const void* Pinv;    // ntrace x bs x bs face-block inverses, block precision
  const double* t;     // right-hand side
  double* x;           // solution (zeroed by run_gmres_fused)
  double* V;           // (GM_MAXM + 1) x n Krylov basis
  void* z;             // n values of the block precision: the current preconditioned vector
  double* partial;     // fused_partial_doubles(grid)
  unsigned* bar;       // 2 words: barrier arrivals, abort flag
  GmresState* st;
  size_t n;
  int m;
  double rtol;
  int x_zero;
  int true_res;  // 1: compute ||t - L x|| after the cycle (else the estimate is reported)
  // nullable: device words {x_zero, m} read by the cycle instead of the two fields above (a cycle
  // captured once in a graph whose restarts a device kernel decides)
  const int* dyn = nullptr;
};
size_t fused_partial_doubles(int max_blocks);
// CTAs of the cooperative launch (one per SM), 0 when the shape or the device does not allow it
int fused_gmres_grid(int prec_bytes, int nT, int bs);
// returns 0 (result in res; *timed_out = 1 if a grid barrier wait ran out) or -1 on a CUDA error.
// dev_status (nullable): two device status words copied to host_status with the first cycle's result
int run_gmres_fused(const FusedArgs& a, int prec_bytes, int grid, double rtol, int restart, int maxit,
                    GmresResult* res, int* timed_out, cudaStream_t s, const int* dev_status = nullptr,
                    int* host_status = nullptr);
// one restart cycle (enqueue only; a.bar must be zeroed before it): cudaErrorInvalidValue when
// the shape has no single-launch cycle
cudaError_t launch_gmres_cycle(const FusedArgs& a, int prec_bytes, int grid, cudaStream_t s);
// Self-test of the bounded grid barrier used by the single-launch cycle (cooperative launch of
// nblocks CTAs, `rounds` barriers; CTA `absent` never arrives when 0 <= absent < nblocks).
// Returns 0 (timed_out set when the abort flag was raised), -1 on a CUDA error, -2 on arguments
// the device cannot run as one cooperative launch.
int barrier_selftest(int nblocks, int absent, int rounds, double timeout_s, int* passed, int* timed_out,
                     cudaStream_t s);

int run_gmres(const GmresOps& ops, const GmresBuffers& b, const double* t, double* x, double rtol, int restart,
              int maxit, int check_every, GmresResult* res, cudaStream_t s);

// The same GMRES(m) enqueued on a capturing stream s for a whole-stage graph: the restart cycles
// are a WHILE node (body captured on sc[0]) whose restart decision is taken on the device, the
// residual mat-vec of every cycle but the first an IF node (body on sc[1]), and the m iterations
// of a cycle enqueued unrolled, each returning at once after the cycle's end (device state).
// The iteration limit is checked per cycle.  dev: the solve's counters (device memory).
struct GmresGraphDev {
  int first, total, cycles, nan, converged;
};
struct GmresGraphLaunches {
  int fixed = 0;     // once per solve
  int cycle = 0;     // per cycle
  int residual = 0;  // per cycle but the first
};
cudaError_t capture_gmres(const GmresOps& ops, const GmresBuffers& b, const double* t, double* x, double rtol,
                          int restart, int maxit, GmresGraphDev* dev, cudaStream_t s, const cudaStream_t sc[2],
                          GmresGraphLaunches* counts);

}  // namespace hfr
