// C-ABI entry points of the hybridized IMEX FR stage library (declared in include/hfr.h).
//
// Host side: reference operators (Gauss-Legendre nodes by Newton iteration, barycentric
// Lagrange derivatives, DG-recovering correction lift l_i(+-1)/w_i), bilinear metrics, face
// classification and trace numbering, workspace management, and the Newton / IMEX stage
// driver (Pereira & Vermeire, arXiv 2401.16632, Sec. 3.1 and Algorithm 1).  Every step of the
// numerical path runs in the CUDA kernels of this library.
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <utility>
#include <vector>

#include "../../include/hfr.h"
#include "hfr_internal.h"
#include "hfr_krylov.h"
#include "hfr_general.h"

using namespace hfr;

static std::atomic<unsigned long long> g_launches(0);
void hfr::count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long hfr::launch_count() { return g_launches.load(std::memory_order_relaxed); }
namespace {
using ChkCollect = int (*)(unsigned long long*, unsigned long long*);
std::vector<ChkCollect>& checked_units() {
  static std::vector<ChkCollect> v;
  return v;
}
}  // namespace
void hfr::checked_register(int (*collect)(unsigned long long* first, unsigned long long* count)) {
  checked_units().push_back(collect);
}
void hfr::launch_count_add(long long delta) {
  g_launches.fetch_add((unsigned long long)delta, std::memory_order_relaxed);
}

// Device-side state of a stage run as one CUDA graph (imex_stage_set_graph): Newton norms and
// counters, and the arguments of the next GMRES restart cycle.
struct StageDev {
  double norm0, norm;
  int it, gtot, conv, err;  // err bits: 1 non-finite residual, 2 non-finite GMRES, 4 barrier timeout
  int gm_total, cycles;
  int dyn[2];  // x_zero, m of the next restart cycle
};

struct StageGraphKey {
  int stage, nmax, gmax, refine;
  double dt, ntol, grtol;
  const double *u_n, *u_stage, *uhat, *R_hist;
  bool operator==(const StageGraphKey& o) const {
    return stage == o.stage && nmax == o.nmax && gmax == o.gmax && refine == o.refine && dt == o.dt &&
           ntol == o.ntol && grtol == o.grtol && u_n == o.u_n && u_stage == o.u_stage && uhat == o.uhat &&
           R_hist == o.R_hist;
  }
};

struct fr_ctx {
  hfr::gen::GenCtx* gen = nullptr;  // general meshes (per-element degree, boundary faces)
  int E = 0, p = 0, n = 0, ns = 0, nv = 0, nA = 0, nT = 0, ntrace = 0, Eim = 0;
  int prec_bytes = 8;
  int tableau = 0;
  int restart = 30;
  bool need_nbr = false;
  bool has_explicit = false;
  cudaStream_t stream = 0;
  RefOps ref;
  PhysParams pp;
  size_t bytes = 0;
  std::vector<void*> allocs;
  std::vector<double> xy_host;  // solution point coordinates
  // geometry / connectivity (device)
  double *geo_sol = nullptr, *geo_face = nullptr;
  int *nbr = nullptr, *nbr_face = nullptr, *kind = nullptr, *tr_of = nullptr;
  unsigned char* implicit = nullptr;
  int *sides_e = nullptr, *sides_c = nullptr, *imp_idx = nullptr, *tr_of_c = nullptr;
  // residual workspace
  double *Uf_all = nullptr, *qf_all = nullptr, *Rw = nullptr, *gview = nullptr, *gw = nullptr;
  double *dUw = nullptr, *dRw = nullptr, *dgview = nullptr;
  // Newton system
  double *r = nullptr, *s = nullptr, *xr = nullptr, *te = nullptr, *tg = nullptr, *Pinv = nullptr;
  void *A = nullptr, *B = nullptr, *C = nullptr, *D = nullptr, *LU = nullptr, *XB = nullptr, *S = nullptr;
  unsigned short* S16 = nullptr;  // FR_PREC_BF16: the trace operator in BF16 for the GMRES mat-vec
  int* piv = nullptr;
  int* status = nullptr;  // [0] bits, [1] first element
  // Krylov
  GmresBuffers gm;
  int gm_mode = 0;          // 0: multi-kernel cycle, 1: one cooperative launch per cycle
  int jac_policy = 0;       // fr_jacobian_policy
  // condensation held for FR_JAC_KEEP: valid, for which a_ii dt, refresh asked by the caller
  int keep_valid = 0;
  double keep_adt = 0.0;
  int keep_refresh = 0;
  long long jac_refreshes = 0;  // element-block linearisations made by imex_stage
  int cond_mode = 0;        // fr_condense_mode of the FP32 condensation
  int inv_ctas = 0;         // CTAs per SM of the tensor-core inverse (0: default)
  double* filt = nullptr;   // ns x ns modal filter operator (fr_modal_filter)
  // whole-stage CUDA graph
  int use_graph = 0;
  StageDev* sdev = nullptr;
  cudaStream_t cap[4] = {nullptr, nullptr, nullptr, nullptr};
  bool gvalid = false;
  StageGraphKey gkey{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int gl_top = 0, gl_newton = 0, gl_solve = 0, gl_cycle = 0;  // kernel launches per part of the graph
  unsigned long long gl_replayed = 0;                            // kernel executions in graph replays
  int gm_fused_grid = 0;    // CTAs of the cooperative launch (0: not available)
  unsigned* gm_bar = nullptr;
  double *duhat = nullptr, *du = nullptr, *res_tmp = nullptr, *Ustar = nullptr, *red = nullptr;
  // linearisation point used by the FP64 refinement (context-owned copies for the ABI call,
  // the stage's own buffers inside imex_stage)
  double *lin_Ubuf = nullptr, *lin_uhbuf = nullptr;
  const double* lin_U = nullptr;
  const double* lin_uhat = nullptr;
  double lin_adt = 0.0;
  fr_error_info err;
  // per-phase event timing
  bool prof = false;
  std::vector<cudaEvent_t> evpool;
  size_t evused = 0;
  std::vector<std::pair<int, std::pair<int, int>>> pend;
  double pms[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  long long pcnt[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
};

enum { PH_RES = 0, PH_JAC = 1, PH_COND = 2, PH_PREC = 3, PH_GMRES = 4, PH_BACK = 5, PH_NEWTON = 6, PH_REFX = 7, PH_MATVEC = 8, PH_CPROD = 9 };

static int prof_begin(fr_ctx* ctx, int phase) {
  if (!ctx->prof || ctx->evused + 2 > ctx->evpool.size()) return -1;
  const int a = (int)ctx->evused++;
  cudaEventRecord(ctx->evpool[a], ctx->stream);
  ctx->pend.push_back({phase, {a, -1}});
  return (int)ctx->pend.size() - 1;
}
static void prof_end(fr_ctx* ctx, int h) {
  if (h < 0) return;
  const int b = (int)ctx->evused++;
  cudaEventRecord(ctx->evpool[b], ctx->stream);
  ctx->pend[h].second.second = b;
}
// after the stream has been synchronised
static void prof_collect(fr_ctx* ctx) {
  for (auto& p : ctx->pend) {
    if (p.second.second < 0) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->evpool[p.second.first], ctx->evpool[p.second.second]) == cudaSuccess) {
      ctx->pms[p.first] += ms;
      ctx->pcnt[p.first] += 1;
    }
  }
  ctx->pend.clear();
  ctx->evused = 0;
}

// ------------------------------------------------------------------------------ errors
static int set_err(fr_ctx* c, int code, const char* msg, int elem = -1, int it = -1, double val = 0.0) {
  if (c) {
    c->err.code = code;
    c->err.element = elem;
    c->err.iteration = it;
    c->err.value = val;
    snprintf(c->err.message, sizeof(c->err.message), "%s", msg);
  }
  return code;
}
// hooks of the general path into this context
static int hook_prof_begin(void* c, int ph) { return prof_begin((fr_ctx*)c, ph); }
static void hook_prof_end(void* c, int h) { prof_end((fr_ctx*)c, h); }
static int hook_set_err(void* c, int code, const char* msg, int elem, int it, double val) {
  return set_err((fr_ctx*)c, code, msg, elem, it, val);
}
// entry points that the general path does not build
#define NOT_GENERAL(ctx, name)                                                                       \
  do {                                                                                               \
    if ((ctx) && (ctx)->gen) return set_err((ctx), FR_ERR_UNSUPPORTED, name ": not built for general meshes"); \
  } while (0)

#define CK(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e_));        \
  } while (0)

// --------------------------------------------------------------------- reference element
void hfr::gauss_legendre_nodes(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    // classic initial guess, then Newton on P_n
    double z = cos(M_PI * (4.0 * (n - i) - 1.0) / (4.0 * n + 2.0));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      double pn = n == 0 ? 1.0 : p1, pm = p0;
      if (n == 1) { pn = z; pm = 1.0; }
      double dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) {
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        break;
      }
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
}

void hfr::build_ref_ops(int p, RefOps& R) {
  memset(&R, 0, sizeof(R));
  const int n = p + 1;
  double x[HFR_MAXN], w[HFR_MAXN], bw[HFR_MAXN];
  hfr::gauss_legendre_nodes(n, x, w);
  for (int j = 0; j < n; ++j) {  // barycentric weights
    double prod = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) prod *= (x[j] - x[k]);
    bw[j] = 1.0 / prod;
  }
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (i == j) continue;
      R.D[i][j] = (bw[j] / bw[i]) / (x[i] - x[j]);
      diag -= R.D[i][j];
    }
    R.D[i][i] = diag;
  }
  for (int side = 0; side < 2; ++side) {  // l_j(-1), l_j(+1), barycentric formula
    const double z = side ? 1.0 : -1.0;
    double den = 0.0;
    for (int j = 0; j < n; ++j) den += bw[j] / (z - x[j]);
    for (int j = 0; j < n; ++j) (side ? R.lp : R.lm)[j] = (bw[j] / (z - x[j])) / den;
  }
  for (int i = 0; i < n; ++i) {
    R.w[i] = w[i];
    R.dgL[i] = -R.lm[i] / w[i];
    R.dgR[i] = R.lp[i] / w[i];
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) R.M[i][j] = R.D[i][j] - R.dgL[i] * R.lm[j] - R.dgR[i] * R.lp[j];
}

// bilinear map derivatives at reference point (xi, eta)
static void bilinear(const double* V, double xi, double eta, double* J, double S[2][2], double* xy) {
  const double sa[4] = {-1, 1, -1, 1}, sb[4] = {-1, -1, 1, 1};
  double xx = 0, xe = 0, yx = 0, ye = 0, px = 0, py = 0;
  for (int k = 0; k < 4; ++k) {
    const double dNx = 0.25 * sa[k] * (1 + sb[k] * eta), dNe = 0.25 * sb[k] * (1 + sa[k] * xi);
    const double Nk = 0.25 * (1 + sa[k] * xi) * (1 + sb[k] * eta);
    xx += dNx * V[2 * k];
    yx += dNx * V[2 * k + 1];
    xe += dNe * V[2 * k];
    ye += dNe * V[2 * k + 1];
    px += Nk * V[2 * k];
    py += Nk * V[2 * k + 1];
  }
  *J = xx * ye - xe * yx;
  S[0][0] = ye;
  S[0][1] = -xe;
  S[1][0] = -yx;
  S[1][1] = xx;
  if (xy) { xy[0] = px; xy[1] = py; }
}

template <typename T>
static T* dalloc(fr_ctx* c, size_t count, int* rc) {
  if (count == 0) count = 1;
  void* p = nullptr;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    *rc = FR_ERR_OOM;
    return nullptr;
  }
  c->allocs.push_back(p);
  c->bytes += count * sizeof(T);
  return (T*)p;
}

// ------------------------------------------------------------------------ small kernels
__global__ void k_form_rhs(int Eim, int nA, int nT, const int* __restrict__ imp_idx, const double* __restrict__ U,
                           const double* __restrict__ Ustar, const double* __restrict__ R,
                           const double* __restrict__ gview, double adt, double* __restrict__ r,
                           double* __restrict__ s) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nr = (size_t)Eim * nA, ns = (size_t)Eim * nT;
  if (i < nr) {
    const int k = (int)(i / nA), q = (int)(i % nA);
    const size_t ix = (size_t)imp_idx[k] * nA + q;
    const double us = Ustar ? Ustar[ix] : U[ix];
    r[i] = -(U[ix] - us - adt * R[ix]);
  } else if (i < nr + ns) {
    const size_t j = i - nr;
    const int k = (int)(j / nT), q = (int)(j % nT);
    s[j] = -gview[(size_t)imp_idx[k] * nT + q];
  }
}

// deterministic sum of squares of two vectors: partials then final
__global__ void k_sumsq_part(const double* __restrict__ a, size_t na, const double* __restrict__ b, size_t nb,
                             double* __restrict__ partial) {
  __shared__ double red[8];
  double s = 0.0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < na + nb; x += stride) {
    const double v = x < na ? a[x] : b[x - na];
    s += v * v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    partial[blockIdx.x] = t;
  }
}
// one warp: lane l sums partials l, l + 32, ... in order, then a fixed butterfly (deterministic)
__global__ void k_sumsq_final(const double* __restrict__ partial, int nblk, double* out) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  double t = 0.0;
  for (int i = lane; i < nblk; i += 32) t += partial[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) *out = t;
}

__global__ void k_apply_du(int Eim, int nA, const int* __restrict__ imp_idx, const double* __restrict__ du,
                           double* __restrict__ U) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)Eim * nA) return;
  const int k = (int)(i / nA), q = (int)(i % nA);
  U[(size_t)imp_idx[k] * nA + q] += du[i];
}
__global__ void k_scatter_du(int Eim, int nA, const int* __restrict__ imp_idx, const double* __restrict__ du,
                             double* __restrict__ full) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)Eim * nA) return;
  const int k = (int)(i / nA), q = (int)(i % nA);
  full[(size_t)imp_idx[k] * nA + q] = du[i];
}
__global__ void k_axpy(size_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}
// refinement residual: res_k = r_k - (du_k - adt dR_k)    (dR = JVP of R at the linearisation point)
__global__ void k_refine_res(int Eim, int nA, const int* __restrict__ imp_idx, const double* __restrict__ r,
                             const double* __restrict__ du, const double* __restrict__ dR, double adt,
                             double* __restrict__ res) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)Eim * nA) return;
  const int k = (int)(i / nA), q = (int)(i % nA);
  res[i] = r[i] - (du[i] - adt * dR[(size_t)imp_idx[k] * nA + q]);
}

struct StageCoef {
  int nterm;
  double ci[8];  // coefficients for implicit elements (dt included)
  double ce[8];  // coefficients for explicit elements
  int hi[8];     // history index per term
};
// out = base + sum_j c_j R_hist[h_j]   (per element class)
__global__ void k_stage_combine(int E, int nA, const unsigned char* __restrict__ implicit,
                                const double* __restrict__ base, const double* __restrict__ Rh, StageCoef sc,
                                double* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t tot = (size_t)E * nA;
  if (i >= tot) return;
  const bool im = implicit[i / nA] != 0;
  double v = base[i];
  for (int j = 0; j < sc.nterm; ++j) {
    const double c = im ? sc.ci[j] : sc.ce[j];
    if (c != 0.0) v += c * Rh[(size_t)sc.hi[j] * tot + i];
  }
  out[i] = v;
}
__global__ void k_copy_implicit(int E, int nA, const unsigned char* __restrict__ implicit, int want_implicit,
                                const double* __restrict__ src, double* __restrict__ dst) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)E * nA) return;
  if ((implicit[i / nA] != 0) == (want_implicit != 0)) dst[i] = src[i];
}
__global__ void k_initial_trace(int ntrace, int npf, int NF_npf, const int* __restrict__ sides,
                                const double* __restrict__ Uf, double* __restrict__ uhat) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntrace * npf) return;
  const int t = i / npf, k = i % npf;
  const int e0 = sides[t * 4], f0 = sides[t * 4 + 1], e1 = sides[t * 4 + 2], f1 = sides[t * 4 + 3];
  const int fpn = NF_npf / 4;
  double v = Uf[(size_t)e0 * NF_npf + f0 * fpn + k];
  if (e1 >= 0) v = 0.5 * (v + Uf[(size_t)e1 * NF_npf + f1 * fpn + k]);
  uhat[i] = v;
}

static inline unsigned nblk(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------------ context
extern "C" int fr_ctx_create(const fr_mesh_desc* mesh, const fr_config* cfg, void* stream, fr_ctx** out) {
  FR_NVTX("fr_ctx_create");
  if (!mesh || !cfg || !out) return FR_ERR_INVALID_ARG;
  *out = nullptr;
  if (mesh->nelem <= 0 || !mesh->verts || !mesh->nbr || !mesh->nbr_face || !mesh->face_of || !mesh->implicit)
    return FR_ERR_INVALID_ARG;
  if (mesh->elem_type != FR_ELEM_QUAD && mesh->elem_type != FR_ELEM_HEX) return FR_ERR_UNSUPPORTED;
  if (hfr::gen::mesh_is_general(mesh) || cfg->trace_kind == FR_TRACE_EFR) {
    fr_ctx* ctx = new fr_ctx();
    memset(&ctx->err, 0, sizeof(ctx->err));
    ctx->stream = (cudaStream_t)stream;
    hfr::gen::Hooks hk;
    hk.owner = ctx;
    hk.prof_begin = hook_prof_begin;
    hk.prof_end = hook_prof_end;
    hk.set_err = hook_set_err;
    const int rc = hfr::gen::create(mesh, cfg, ctx->stream, hk, &ctx->gen);
    if (rc != FR_OK) {
      delete ctx;
      return rc;
    }
    fr_ctx_info gi;
    hfr::gen::query(ctx->gen, &gi);
    ctx->E = gi.nelem;
    ctx->Eim = gi.nimplicit;
    ctx->nv = gi.nv;
    ctx->ntrace = gi.ntrace;
    ctx->tableau = cfg->tableau;
    *out = ctx;
    return FR_OK;
  }
  fr_mesh_desc um = *mesh;  // uniform path: one degree (p_elem, when given, holds it)
  if (mesh->p_elem) um.p = mesh->p_elem[0];
  mesh = &um;
  if (mesh->p < 1 || mesh->p > 5) return FR_ERR_UNSUPPORTED;
  if (cfg->trace_kind != FR_TRACE_HFR) return FR_ERR_INVALID_ARG;
  if (cfg->physics != FR_PHYS_ADVDIFF && cfg->physics != FR_PHYS_NAVIER_STOKES && cfg->physics != FR_PHYS_EDAC)
    return FR_ERR_INVALID_ARG;
  if (cfg->physics == FR_PHYS_ADVDIFF && mesh->p > 3) return FR_ERR_UNSUPPORTED;
  if (cfg->physics == FR_PHYS_NAVIER_STOKES && mesh->p < 2) return FR_ERR_UNSUPPORTED;
  if (cfg->physics == FR_PHYS_EDAC && (mesh->p < 2 || mesh->p > 4 || !(cfg->theta > 0.0))) return FR_ERR_UNSUPPORTED;
  if (cfg->precision < FR_PREC_FP64 || cfg->precision > FR_PREC_BF16) return FR_ERR_INVALID_ARG;
  fr_ctx* ctx = new fr_ctx();
  memset(&ctx->err, 0, sizeof(ctx->err));
  ctx->stream = (cudaStream_t)stream;
  ctx->E = mesh->nelem;
  ctx->p = mesh->p;
  ctx->n = mesh->p + 1;
  ctx->ns = ctx->n * ctx->n;
  ctx->nv = cfg->physics == FR_PHYS_ADVDIFF ? 1 : (cfg->physics == FR_PHYS_EDAC ? 3 : 4);
  ctx->nA = ctx->ns * ctx->nv;
  ctx->nT = 4 * ctx->n * ctx->nv;
  ctx->prec_bytes = cfg->precision == FR_PREC_FP64 ? 8 : 4;
  const bool want_bf16 = cfg->precision == FR_PREC_BF16, want_tf32 = cfg->precision == FR_PREC_TF32;
  ctx->tableau = cfg->tableau;
  ctx->restart = cfg->gmres_restart > 0 ? std::min(cfg->gmres_restart, GM_MAXM) : 30;
  memset(&ctx->pp, 0, sizeof(ctx->pp));
  ctx->pp.kind = cfg->physics;
  ctx->pp.beta[0] = cfg->beta[0];
  ctx->pp.beta[1] = cfg->beta[1];
  ctx->pp.nu = cfg->nu;
  ctx->pp.gamma = cfg->gamma;
  ctx->pp.mu = cfg->mu;
  ctx->pp.Pr = cfg->Pr;
  ctx->pp.lref = cfg->lref > 0 ? cfg->lref : 1.0;
  ctx->pp.theta = cfg->physics == FR_PHYS_EDAC ? cfg->theta : 0.0;
  hfr::build_ref_ops(ctx->p, ctx->ref);

  const int E = ctx->E, n = ctx->n, ns = ctx->ns, NF = 4 * n;
  // connectivity checks and face kinds
  std::vector<int> kind(4 * E), tr_of(4 * E, -1);
  int max_fid = -1;
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 4; ++f) {
      const int nb = mesh->nbr[4 * e + f], nf = mesh->nbr_face[4 * e + f];
      if (nb < 0) {
        delete ctx;
        return FR_ERR_UNSUPPORTED;  // boundary faces are not implemented
      }
      if (nb >= E || nf < 0 || nf > 3 || mesh->nbr[4 * nb + nf] != e || mesh->face_of[4 * nb + nf] != mesh->face_of[4 * e + f]) {
        delete ctx;
        return FR_ERR_INVALID_ARG;
      }
      const bool ie = mesh->implicit[e] != 0, in = mesh->implicit[nb] != 0;
      kind[4 * e + f] = (ie && in) ? FK_TRACE : (ie != in ? FK_IMEX : FK_FR);
      if (kind[4 * e + f] != FK_TRACE) ctx->need_nbr = true;
      max_fid = std::max(max_fid, mesh->face_of[4 * e + f]);
    }
  ctx->has_explicit = ctx->need_nbr;
  // trace numbering: trace faces in increasing global face id
  std::vector<int> tr_of_fid(max_fid + 1, -1);
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 4; ++f)
      if (kind[4 * e + f] == FK_TRACE) tr_of_fid[mesh->face_of[4 * e + f]] = 0;
  int nt = 0;
  for (int i = 0; i <= max_fid; ++i)
    if (tr_of_fid[i] == 0) tr_of_fid[i] = nt++;
  ctx->ntrace = nt;
  std::vector<int> imp_idx, comp(E, -1);
  for (int e = 0; e < E; ++e)
    if (mesh->implicit[e]) {
      comp[e] = (int)imp_idx.size();
      imp_idx.push_back(e);
    }
  ctx->Eim = (int)imp_idx.size();
  std::vector<int> sides_e(4 * std::max(nt, 1), -1), sides_c(4 * std::max(nt, 1), -1), tr_of_c(4 * std::max(ctx->Eim, 1), -1);
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 4; ++f)
      if (kind[4 * e + f] == FK_TRACE) {
        const int t = tr_of_fid[mesh->face_of[4 * e + f]];
        tr_of[4 * e + f] = t;
        const int slot = sides_e[4 * t] < 0 ? 0 : 1;
        sides_e[4 * t + 2 * slot] = e;
        sides_e[4 * t + 2 * slot + 1] = f;
        sides_c[4 * t + 2 * slot] = comp[e];
        sides_c[4 * t + 2 * slot + 1] = f;
        tr_of_c[4 * comp[e] + f] = t;
      }
  // geometry
  std::vector<double> gsol((size_t)E * ns * 5), gface((size_t)E * NF * 3);
  ctx->xy_host.resize((size_t)E * ns * 2);
  double xg[HFR_MAXN], wg[HFR_MAXN];
  hfr::gauss_legendre_nodes(n, xg, wg);
  for (int e = 0; e < E; ++e) {
    const double* V = mesh->verts + (size_t)e * 8;
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        const int pt = a + n * b;
        double J, S[2][2];
        bilinear(V, xg[a], xg[b], &J, S, &ctx->xy_host[((size_t)e * ns + pt) * 2]);
        double* G = &gsol[((size_t)e * ns + pt) * 5];
        G[0] = 1.0 / J;
        G[1] = S[0][0];
        G[2] = S[0][1];
        G[3] = S[1][0];
        G[4] = S[1][1];
      }
    for (int f = 0; f < 4; ++f) {
      const int r = f >> 1;
      const double sg = (f & 1) ? 1.0 : -1.0;
      for (int m = 0; m < n; ++m) {
        const double xi = r == 0 ? sg : xg[m], eta = r == 0 ? xg[m] : sg;
        double J, S[2][2];
        bilinear(V, xi, eta, &J, S, nullptr);
        const double N0 = sg * S[r][0], N1 = sg * S[r][1];
        const double Jf = sqrt(N0 * N0 + N1 * N1);
        double* G = &gface[((size_t)e * NF + f * n + m) * 3];
        G[0] = Jf;
        G[1] = N0 / Jf;
        G[2] = N1 / Jf;
      }
    }
  }
  // device allocations
  int rc = FR_OK;
  const int nv = ctx->nv, nA = ctx->nA, nT = ctx->nT, Eim = ctx->Eim;
  const size_t nh = (size_t)nt * n * nv;
  const size_t pb = ctx->prec_bytes;
  ctx->geo_sol = dalloc<double>(ctx, gsol.size(), &rc);
  ctx->geo_face = dalloc<double>(ctx, gface.size(), &rc);
  ctx->nbr = dalloc<int>(ctx, 4 * E, &rc);
  ctx->nbr_face = dalloc<int>(ctx, 4 * E, &rc);
  ctx->kind = dalloc<int>(ctx, 4 * E, &rc);
  ctx->tr_of = dalloc<int>(ctx, 4 * E, &rc);
  ctx->implicit = dalloc<unsigned char>(ctx, E, &rc);
  ctx->sides_e = dalloc<int>(ctx, sides_e.size(), &rc);
  ctx->sides_c = dalloc<int>(ctx, sides_c.size(), &rc);
  ctx->imp_idx = dalloc<int>(ctx, std::max(Eim, 1), &rc);
  ctx->tr_of_c = dalloc<int>(ctx, tr_of_c.size(), &rc);
  if (ctx->need_nbr) {
    ctx->Uf_all = dalloc<double>(ctx, (size_t)E * NF * nv, &rc);
    ctx->qf_all = dalloc<double>(ctx, (size_t)E * NF * 2 * nv, &rc);
  }
  ctx->Rw = dalloc<double>(ctx, (size_t)E * nA, &rc);
  ctx->gview = dalloc<double>(ctx, (size_t)E * NF * nv, &rc);
  ctx->gw = dalloc<double>(ctx, nh, &rc);
  ctx->dUw = dalloc<double>(ctx, (size_t)E * nA, &rc);
  ctx->dRw = dalloc<double>(ctx, (size_t)E * nA, &rc);
  ctx->dgview = dalloc<double>(ctx, (size_t)E * NF * nv, &rc);
  ctx->r = dalloc<double>(ctx, (size_t)Eim * nA, &rc);
  ctx->s = dalloc<double>(ctx, (size_t)Eim * nT, &rc);
  ctx->xr = dalloc<double>(ctx, (size_t)Eim * nA, &rc);
  ctx->te = dalloc<double>(ctx, (size_t)Eim * nT, &rc);
  ctx->tg = dalloc<double>(ctx, nh, &rc);
  ctx->Pinv = dalloc<double>(ctx, (size_t)nt * (n * nv) * (n * nv), &rc);
  ctx->A = dalloc<unsigned char>(ctx, (size_t)Eim * nA * nA * pb, &rc);
  ctx->B = dalloc<unsigned char>(ctx, (size_t)Eim * nA * nT * pb, &rc);
  ctx->C = dalloc<unsigned char>(ctx, (size_t)Eim * nT * nA * pb, &rc);
  ctx->D = dalloc<unsigned char>(ctx, (size_t)Eim * nT * nT * pb, &rc);
  ctx->LU = dalloc<unsigned char>(ctx, (size_t)Eim * nA * nA * pb, &rc);
  ctx->XB = dalloc<unsigned char>(ctx, (size_t)Eim * nA * nT * pb, &rc);
  ctx->S = dalloc<unsigned char>(ctx, (size_t)Eim * nT * nT * pb, &rc);
  ctx->piv = dalloc<int>(ctx, (size_t)Eim * nA, &rc);
  ctx->status = dalloc<int>(ctx, 2, &rc);
  ctx->gm.n = nh;
  ctx->gm.V = dalloc<double>(ctx, (size_t)(GM_MAXM + 1) * std::max(nh, (size_t)1), &rc);
  ctx->gm.Z = dalloc<double>(ctx, (size_t)GM_MAXM * std::max(nh, (size_t)1), &rc);
  {
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    ctx->gm_fused_grid = fused_gmres_grid(ctx->prec_bytes, nT, n * nv);
    ctx->gm_mode = ctx->gm_fused_grid > 0 ? 1 : 0;
    ctx->cond_mode = condense_tc_available(ctx->prec_bytes, nA, nT);
    if ((want_bf16 && ctx->gm_fused_grid <= 0) || (want_tf32 && ctx->cond_mode < FR_CONDENSE_TENSOR)) {
      fr_ctx_destroy(ctx);
      return FR_ERR_UNSUPPORTED;  // the BF16 operator and single-pass TF32 exist for the fixed shapes only
    }
    if (want_tf32) ctx->cond_mode = FR_CONDENSE_TENSOR_TF32;
    if (want_bf16) ctx->S16 = dalloc<unsigned short>(ctx, (size_t)Eim * nT * nT, &rc);
    const size_t np = std::max((size_t)GM_NBLK * (GM_MAXM + 1), fused_partial_doubles(std::max(nsm, 1)));
    ctx->gm.partial = dalloc<double>(ctx, np, &rc);
    ctx->gm_bar = dalloc<unsigned>(ctx, 64, &rc);
  }
  ctx->gm.state = dalloc<GmresState>(ctx, 1, &rc);
  ctx->sdev = dalloc<StageDev>(ctx, 1, &rc);
  ctx->gm.ticket = dalloc<unsigned int>(ctx, 1, &rc);
  ctx->gm.z32 = ctx->prec_bytes == 4 ? dalloc<float>(ctx, std::max(nh, (size_t)1), &rc) : nullptr;
  ctx->duhat = dalloc<double>(ctx, nh, &rc);
  ctx->du = dalloc<double>(ctx, (size_t)Eim * nA, &rc);
  ctx->res_tmp = dalloc<double>(ctx, (size_t)Eim * nA, &rc);
  ctx->Ustar = dalloc<double>(ctx, (size_t)E * nA, &rc);
  ctx->lin_Ubuf = dalloc<double>(ctx, (size_t)E * nA, &rc);
  ctx->lin_uhbuf = dalloc<double>(ctx, std::max(nh, (size_t)1), &rc);
  ctx->red = dalloc<double>(ctx, 1024 + 8, &rc);
  ctx->filt = dalloc<double>(ctx, (size_t)ctx->ns * ctx->ns, &rc);
  if (rc != FR_OK) {
    fr_ctx_destroy(ctx);
    return rc;
  }
  cudaStream_t st = ctx->stream;
  std::vector<unsigned char> impv(mesh->implicit, mesh->implicit + E);
#define UP(dst, src, cnt)                                                                             \
  if (cudaMemcpyAsync(dst, src, (cnt) * sizeof(*(src)), cudaMemcpyHostToDevice, st) != cudaSuccess) { \
    fr_ctx_destroy(ctx);                                                                              \
    return FR_ERR_CUDA;                                                                               \
  }
  UP(ctx->geo_sol, gsol.data(), gsol.size());
  UP(ctx->geo_face, gface.data(), gface.size());
  UP(ctx->nbr, mesh->nbr, 4 * E);
  UP(ctx->nbr_face, mesh->nbr_face, 4 * E);
  UP(ctx->kind, kind.data(), 4 * E);
  UP(ctx->tr_of, tr_of.data(), 4 * E);
  UP(ctx->implicit, impv.data(), E);
  UP(ctx->sides_e, sides_e.data(), sides_e.size());
  UP(ctx->sides_c, sides_c.data(), sides_c.size());
  if (Eim) UP(ctx->imp_idx, imp_idx.data(), Eim);
  UP(ctx->tr_of_c, tr_of_c.data(), tr_of_c.size());
#undef UP
  if (cudaMemsetAsync(ctx->status, 0, 2 * sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(ctx->dUw, 0, (size_t)E * nA * sizeof(double), st) != cudaSuccess ||
      cudaMemsetAsync(ctx->gm.ticket, 0, sizeof(unsigned int), st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    fr_ctx_destroy(ctx);
    return FR_ERR_CUDA;
  }
  *out = ctx;
  return FR_OK;
}

extern "C" void fr_ctx_destroy(fr_ctx* ctx) {
  if (!ctx) return;
  if (ctx->gen) hfr::gen::destroy(ctx->gen);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  for (cudaStream_t c : ctx->cap)
    if (c) cudaStreamDestroy(c);
  for (void* p : ctx->allocs) cudaFree(p);
  for (cudaEvent_t e : ctx->evpool) cudaEventDestroy(e);
  delete ctx;
}

extern "C" int fr_ctx_query(const fr_ctx* ctx, fr_ctx_info* info) {
  if (!ctx || !info) return FR_ERR_INVALID_ARG;
  if (ctx->gen) {
    hfr::gen::query(ctx->gen, info);
    info->workspace_bytes = ctx->bytes + info->workspace_bytes;
    return FR_OK;
  }
  info->nelem = ctx->E;
  info->nimplicit = ctx->Eim;
  info->p = ctx->p;
  info->n = ctx->n;
  info->ns = ctx->ns;
  info->nv = ctx->nv;
  info->nA = ctx->nA;
  info->nT = ctx->nT;
  info->ntrace = ctx->ntrace;
  info->nstages = ctx->tableau == FR_TAB_SDIRK2 ? 2 : 1;
  info->has_explicit = ctx->has_explicit ? 1 : 0;
  info->workspace_bytes = ctx->bytes;
  info->general = 0;
  info->state_values = (size_t)ctx->E * ctx->nA;
  info->trace_values = (size_t)ctx->ntrace * ctx->n * ctx->nv;
  info->face_points = 0;
  return FR_OK;
}

extern "C" int fr_ctx_layout(const fr_ctx* ctx, long long* elem_off, long long* trace_off, int* blk_nA, int* blk_nT) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  if (ctx->gen) return hfr::gen::layout(ctx->gen, elem_off, trace_off, blk_nA, blk_nT);
  if (elem_off)
    for (int e = 0; e <= ctx->E; ++e) elem_off[e] = (long long)e * ctx->nA;
  if (trace_off)
    for (int t = 0; t <= ctx->ntrace; ++t) trace_off[t] = (long long)t * ctx->n * ctx->nv;
  for (int k = 0; k < ctx->Eim; ++k) {
    if (blk_nA) blk_nA[k] = ctx->nA;
    if (blk_nT) blk_nT[k] = ctx->nT;
  }
  return FR_OK;
}

extern "C" int fr_solution_points(fr_ctx* ctx, double* xy) {
  if (!ctx || !xy) return FR_ERR_INVALID_ARG;
  if (ctx->gen) return hfr::gen::solution_points(ctx->gen, xy);
  CK(cudaMemcpyAsync(xy, ctx->xy_host.data(), ctx->xy_host.size() * sizeof(double), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FR_OK;
}

static ResArgs res_args(fr_ctx* ctx, const double* u, const double* uhat) {
  ResArgs a;
  memset(&a, 0, sizeof(a));
  a.E = ctx->E;
  a.U = u;
  a.uhat = uhat;
  a.geo_sol = ctx->geo_sol;
  a.geo_face = ctx->geo_face;
  a.nbr = ctx->nbr;
  a.nbr_face = ctx->nbr_face;
  a.kind = ctx->kind;
  a.tr_of = ctx->tr_of;
  a.implicit = ctx->implicit;
  a.Uf_all = ctx->Uf_all;
  a.qf_all = ctx->qf_all;
  a.Uf_out = ctx->Uf_all;
  a.qf_out = ctx->qf_all;
  a.ntrace = ctx->ntrace;
  return a;
}

// R and element trace contributions (gview) at (u, uhat); g assembled if requested
static int residual_into(fr_ctx* ctx, const double* u, const double* uhat, double* R, double* gview, double* g) {
  ResArgs a = res_args(ctx, u, uhat);
  a.R = R;
  a.gview = gview;
  const int ph = prof_begin(ctx, PH_RES);
  CK(launch_residual(ctx->p, ctx->ref, ctx->pp, a, ctx->need_nbr, false, ctx->stream));
  if (g) CK(launch_trace_assemble(gview, ctx->sides_e, ctx->ntrace, ctx->n * ctx->nv, g, ctx->stream));
  prof_end(ctx, ph);
  return FR_OK;
}

extern "C" int fr_residual(fr_ctx* ctx, const double* u, const double* uhat, double* R, double* g) {
  FR_NVTX("fr_residual");
  if (!ctx || !u || !R) return set_err(ctx, FR_ERR_INVALID_ARG, "fr_residual: null argument");
  if (ctx->ntrace > 0 && !uhat) return set_err(ctx, FR_ERR_INVALID_ARG, "fr_residual: uhat required");
  if (ctx->gen) {
    const int grc = hfr::gen::residual(ctx->gen, u, uhat, R, g);
    prof_collect(ctx);
    return grc;
  }
  int rc = residual_into(ctx, u, uhat, R, ctx->gview, g);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  prof_collect(ctx);
  return FR_OK;
}

extern "C" int hfr_initial_trace(fr_ctx* ctx, const double* u, double* uhat) {
  FR_NVTX("hfr_initial_trace");
  if (!ctx || !u || (ctx->ntrace > 0 && !uhat)) return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_initial_trace: null argument");
  if (ctx->gen) return hfr::gen::initial_trace(ctx->gen, u, uhat);
  // face states of every element into a scratch buffer of the same shape (E x 4n x nv)
  ResArgs a = res_args(ctx, u, nullptr);
  a.Uf_out = ctx->gview;
  CK(launch_face_states(ctx->p, ctx->ref, ctx->pp, a, ctx->stream));
  const int npf = ctx->n * ctx->nv;
  if (ctx->ntrace) {
    (hfr::count_launch(), k_initial_trace<<<nblk((size_t)ctx->ntrace * npf), 256, 0, ctx->stream>>>(ctx->ntrace, npf, 4 * npf, ctx->sides_e,
                                                                               ctx->gview, uhat));
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return FR_OK;
}

// blocks at (u, uhat); assumes r, s were formed at the same point
static int jacobian_blocks(fr_ctx* ctx, const double* u, const double* uhat, double a_dt) {
  JacArgs j;
  memset(&j, 0, sizeof(j));
  j.Eim = ctx->Eim;
  j.imp_idx = ctx->imp_idx;
  j.U = u;
  j.uhat = uhat;
  j.geo_sol = ctx->geo_sol;
  j.geo_face = ctx->geo_face;
  j.nbr = ctx->nbr;
  j.nbr_face = ctx->nbr_face;
  j.kind = ctx->kind;
  j.tr_of = ctx->tr_of;
  j.Uf_all = ctx->Uf_all;
  j.E = ctx->E;
  j.ntrace = ctx->ntrace;
  j.a_dt = a_dt;
  j.A = ctx->A;
  j.B = ctx->B;
  j.C = ctx->C;
  j.D = ctx->D;
  if (ctx->Eim > 0) {  // no implicit element: nothing to linearise
    const int ph = prof_begin(ctx, PH_JAC);
    CK(launch_jacobian(ctx->p, ctx->prec_bytes, ctx->ref, ctx->pp, j, ctx->stream));
    prof_end(ctx, ph);
  }
  ctx->lin_U = u;
  ctx->lin_uhat = uhat;
  ctx->lin_adt = a_dt;
  return FR_OK;
}

static int form_rhs(fr_ctx* ctx, const double* u, const double* ustar, double a_dt) {
  const size_t tot = (size_t)ctx->Eim * (ctx->nA + ctx->nT);
  if (tot == 0) return FR_OK;
  (hfr::count_launch(), k_form_rhs<<<nblk(tot), 256, 0, ctx->stream>>>(ctx->Eim, ctx->nA, ctx->nT, ctx->imp_idx, u, ustar, ctx->Rw,
                                                 ctx->gview, a_dt, ctx->r, ctx->s));
  CK(cudaGetLastError());
  return FR_OK;
}

extern "C" int hfr_local_jacobian(fr_ctx* ctx, const double* u, const double* uhat, const double* ustar,
                                  double a_dt) {
  FR_NVTX("hfr_local_jacobian");
  if (!ctx || !u || (ctx->ntrace > 0 && !uhat)) return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_local_jacobian: null argument");
  if (ctx->gen) {
    const int grc = hfr::gen::local_jacobian(ctx->gen, u, uhat, ustar, a_dt);
    prof_collect(ctx);
    return grc;
  }
  ctx->keep_valid = 0;  // the blocks no longer belong to an imex_stage linearisation
  // keep a copy of the linearisation point for later refinement sweeps
  CK(cudaMemcpyAsync(ctx->lin_Ubuf, u, (size_t)ctx->E * ctx->nA * sizeof(double), cudaMemcpyDeviceToDevice,
                     ctx->stream));
  const size_t nh = (size_t)ctx->ntrace * ctx->n * ctx->nv;
  if (nh) CK(cudaMemcpyAsync(ctx->lin_uhbuf, uhat, nh * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  int rc = residual_into(ctx, u, uhat, ctx->Rw, ctx->gview, nullptr);
  if (!rc) rc = form_rhs(ctx, u, ustar, a_dt);
  if (!rc) rc = jacobian_blocks(ctx, u, uhat, a_dt);
  ctx->lin_U = ctx->lin_Ubuf;
  ctx->lin_uhat = nh ? ctx->lin_uhbuf : nullptr;
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  prof_collect(ctx);
  return FR_OK;
}

static TraceArgs trace_args(fr_ctx* ctx) {
  TraceArgs t;
  t.ntrace = ctx->ntrace;
  t.n = ctx->n;
  t.nv = ctx->nv;
  t.nT = ctx->nT;
  t.sides = ctx->sides_c;
  t.tr_of_c = ctx->tr_of_c;
  t.S = ctx->S;
  return t;
}

// FP64 refinement sweep(s) of X = A^{-1} rhs against the exact linearisation:
// x <- x + LU^{-1} (rhs - A x - B y), A x + B y evaluated as x - adt dR(U, u^)[x, y]
static int refine_local(fr_ctx* ctx, const double* rhs, double* x, const double* y_trace, int sweeps) {
  const int Eim = ctx->Eim, nA = ctx->nA, E = ctx->E;
  const size_t nloc = (size_t)Eim * nA;
  for (int sw = 0; sw < sweeps; ++sw) {
    (hfr::count_launch(), k_scatter_du<<<nblk(nloc), 256, 0, ctx->stream>>>(Eim, nA, ctx->imp_idx, x, ctx->dUw));
    CK(cudaGetLastError());
    ResArgs a = res_args(ctx, ctx->lin_U, ctx->lin_uhat);
    a.dU = ctx->dUw;
    a.duhat = y_trace;
    a.dR = ctx->dRw;
    CK(launch_residual(ctx->p, ctx->ref, ctx->pp, a, ctx->need_nbr, true, ctx->stream));
    (hfr::count_launch(), k_refine_res<<<nblk(nloc), 256, 0, ctx->stream>>>(Eim, nA, ctx->imp_idx, rhs, x, ctx->dRw, ctx->lin_adt,
                                                      ctx->res_tmp));
    CK(cudaGetLastError());
    CK(launch_lu_solve(ctx->prec_bytes, Eim, nA, ctx->nT, ctx->LU, ctx->piv, ctx->res_tmp, ctx->stream));
    (hfr::count_launch(), k_axpy<<<nblk(nloc), 256, 0, ctx->stream>>>(nloc, 1.0, ctx->res_tmp, x));
    CK(cudaGetLastError());
  }
  (void)E;
  return FR_OK;
}

static int check_status(fr_ctx* ctx, const char* where) {
  int hs[2];
  CK(cudaMemcpyAsync(hs, ctx->status, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (hs[0] & DEV_ERR_SINGULAR) {
    CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
    return set_err(ctx, FR_ERR_SINGULAR, where, hs[1]);
  }
  if (hs[0] & DEV_ERR_TIMEOUT) {
    CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
    return set_err(ctx, FR_ERR_TIMEOUT, "hfr_condense: tensor-core completion wait timed out");
  }
  return FR_OK;
}

// the trace operator in BF16 (round to nearest even) for the GMRES mat-vec of FR_PREC_BF16
__global__ void k_s_to_bf16(size_t n, const float* __restrict__ S, unsigned short* __restrict__ S16) {
  const size_t i = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (i + 3 < n) {
    const float4 v = *reinterpret_cast<const float4*>(S + i);
    const __nv_bfloat16 b0 = __float2bfloat16_rn(v.x), b1 = __float2bfloat16_rn(v.y), b2 = __float2bfloat16_rn(v.z),
                        b3 = __float2bfloat16_rn(v.w);
    ushort4 o;
    o.x = __bfloat16_as_ushort(b0);
    o.y = __bfloat16_as_ushort(b1);
    o.z = __bfloat16_as_ushort(b2);
    o.w = __bfloat16_as_ushort(b3);
    *reinterpret_cast<ushort4*>(S16 + i) = o;
  } else {
    for (size_t j = i; j < n; ++j) S16[j] = __bfloat16_as_ushort(__float2bfloat16_rn(S[j]));
  }
}

__global__ void k_status_reset(int* status) {
  status[0] = 0;
  status[1] = 0x7fffffff;
}

static int condense_impl(fr_ctx* ctx, int refine) {
  // (a kernel, not a copy from host memory: a pageable host-to-device copy would wait for the stream)
  (hfr::count_launch(), k_status_reset<<<1, 1, 0, ctx->stream>>>(ctx->status));
  CK(cudaGetLastError());
  if (ctx->Eim == 0) return FR_OK;  // no implicit element (and so no trace)
  CondArgs c;
  c.Eim = ctx->Eim;
  c.nA = ctx->nA;
  c.nT = ctx->nT;
  c.A = ctx->A;
  c.B = ctx->B;
  c.C = ctx->C;
  c.D = ctx->D;
  c.r = ctx->r;
  c.s = ctx->s;
  c.LU = ctx->LU;
  c.piv = ctx->piv;
  c.XB = ctx->XB;
  c.xr = ctx->xr;
  c.S = ctx->S;
  c.t = ctx->te;
  c.status = ctx->status;
  c.tc_mode = ctx->cond_mode;
  c.inv_ctas = ctx->inv_ctas;
  int ph = prof_begin(ctx, PH_COND);
  CK(launch_condense_part(ctx->prec_bytes, c, ctx->stream, 0));
  prof_end(ctx, ph);
  ph = prof_begin(ctx, PH_CPROD);
  CK(launch_condense_part(ctx->prec_bytes, c, ctx->stream, 1));
  if (ctx->S16) {
    const size_t ns16 = (size_t)ctx->Eim * ctx->nT * ctx->nT;
    (hfr::count_launch(), k_s_to_bf16<<<nblk((ns16 + 3) / 4), 256, 0, ctx->stream>>>(ns16, (const float*)ctx->S, ctx->S16));
    CK(cudaGetLastError());
  }
  prof_end(ctx, ph);
  if (refine > 0 && ctx->lin_U) {
    // FP64 refinement of x_r against the exact linearisation (used by the back-substitution)
    ph = prof_begin(ctx, PH_REFX);
    int rc = refine_local(ctx, ctx->r, ctx->xr, nullptr, refine);
    prof_end(ctx, ph);
    if (rc) return rc;
  }
  TraceArgs t = trace_args(ctx);
  ph = prof_begin(ctx, PH_PREC);
  CK(launch_assemble_t(t, ctx->te, ctx->tg, ctx->stream));
  CK(launch_precond_build(ctx->prec_bytes, t, ctx->Pinv, ctx->status, ctx->stream));
  prof_end(ctx, ph);
  return FR_OK;
}

// New right-hand sides with the blocks of an earlier condensation (chord Newton iterations):
// x_r = A^{-1} r with the stored factorisation, t_k = s - C x_r, t = sum scatter(t_k).  S_k, X_B and
// the face preconditioner are kept.
static int condense_rhs_impl(fr_ctx* ctx) {
  if (ctx->Eim == 0) return FR_OK;
  const size_t nrA = (size_t)ctx->Eim * ctx->nA;
  int ph = prof_begin(ctx, PH_COND);
  CK(cudaMemcpyAsync(ctx->xr, ctx->r, nrA * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  CK(launch_lu_solve(ctx->prec_bytes, ctx->Eim, ctx->nA, ctx->nT, ctx->LU, ctx->piv, ctx->xr, ctx->stream));
  CK(launch_rhs_condense(ctx->prec_bytes, ctx->Eim, ctx->nA, ctx->nT, ctx->C, ctx->xr, ctx->s, ctx->te, ctx->stream));
  prof_end(ctx, ph);
  ph = prof_begin(ctx, PH_PREC);
  CK(launch_assemble_t(trace_args(ctx), ctx->te, ctx->tg, ctx->stream));
  prof_end(ctx, ph);
  return FR_OK;
}

extern "C" int hfr_condense(fr_ctx* ctx, int refine) {
  FR_NVTX("hfr_condense");
  if (!ctx) return FR_ERR_INVALID_ARG;
  if (ctx->gen) {
    const int grc = hfr::gen::condense(ctx->gen, refine);
    prof_collect(ctx);
    return grc;
  }
  ctx->keep_valid = 0;
  int rc = condense_impl(ctx, refine);
  if (rc) return rc;
  rc = check_status(ctx, "hfr_condense: zero pivot");
  prof_collect(ctx);
  return rc;
}

// GMRES callbacks
static void cb_matvec(void* c, const double* x, double* y, cudaStream_t s) {
  fr_ctx* ctx = (fr_ctx*)c;
  const int ph = prof_begin(ctx, PH_MATVEC);
  launch_trace_matvec(ctx->prec_bytes, trace_args(ctx), x, y, s);
  prof_end(ctx, ph);
}
static void cb_gmatvec(void* c, const GmresState* st, int j, const double* x, const float* x32, double* y,
                       cudaStream_t s) {
  fr_ctx* ctx = (fr_ctx*)c;
  launch_trace_matvec(ctx->prec_bytes, trace_args(ctx), x, y, s, &st->kdone, j, x32);
}
static void cb_precond(void* c, const GmresState* st, int j, double* x, double* y, float* y32, cudaStream_t s) {
  fr_ctx* ctx = (fr_ctx*)c;
  launch_precond_apply(ctx->prec_bytes, trace_args(ctx), ctx->Pinv, x, y, s, &st->kdone, j,
                       j > 0 ? &st->inv_hn : nullptr, y32);
}

// true_res: report the true final residual ||t - L du^|| / ||t|| (else the GMRES estimate, which
// the Newton iteration does not need)
// cond_status (host, nullable): receives the condensation status words, read back with the
// GMRES result instead of at a synchronisation of their own
static int gmres_impl(fr_ctx* ctx, double* duhat, double rtol, int maxit, int* iters, double* final_rel,
                      bool true_res = true, int* cond_status = nullptr) {
  GmresOps ops;
  ops.ctx = ctx;
  ops.matvec = cb_matvec;
  ops.gated_matvec = cb_gmatvec;
  ops.precond = cb_precond;
  GmresResult res;
  memset(&res, 0, sizeof(res));
  if (ctx->ntrace == 0) {
    if (iters) *iters = 0;
    if (final_rel) *final_rel = 0.0;
    if (cond_status) {
      CK(cudaMemcpyAsync(cond_status, ctx->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    }
    return FR_OK;
  }
  const int ph = prof_begin(ctx, PH_GMRES);
  int grc = 0, timed_out = 0;
  if (ctx->gm_mode == 1) {
    FusedArgs fa;
    fa.ntrace = ctx->ntrace;
    fa.nT = ctx->nT;
    fa.sides = ctx->sides_c;
    fa.tr_of_c = ctx->tr_of_c;
    fa.S = ctx->S16 ? (const void*)ctx->S16 : ctx->S;
    fa.s_bf16 = ctx->S16 ? 1 : 0;
    fa.S_bytes = (size_t)ctx->Eim * ctx->nT * ctx->nT * (ctx->S16 ? 2 : ctx->prec_bytes);
    fa.Pinv = ctx->Pinv;
    fa.t = ctx->tg;
    fa.x = duhat;
    fa.V = ctx->gm.V;
    fa.z = ctx->prec_bytes == 4 ? (void*)ctx->gm.z32 : (void*)ctx->gm.Z;
    fa.partial = ctx->gm.partial;
    fa.bar = ctx->gm_bar;
    fa.st = ctx->gm.state;
    fa.n = ctx->gm.n;
    fa.m = ctx->restart;
    fa.rtol = rtol;
    fa.x_zero = 1;
    fa.true_res = true_res ? 1 : 0;
    grc = run_gmres_fused(fa, ctx->prec_bytes, ctx->gm_fused_grid, rtol, ctx->restart, maxit, &res, &timed_out,
                          ctx->stream, cond_status ? ctx->status : nullptr, cond_status);
  } else {
    grc = run_gmres(ops, ctx->gm, ctx->tg, duhat, rtol, ctx->restart, maxit, 4, &res, ctx->stream);
    if (grc == 0 && cond_status) {
      CK(cudaMemcpyAsync(cond_status, ctx->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
    }
  }
  prof_end(ctx, ph);
  if (grc != 0) return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  if (timed_out) return set_err(ctx, FR_ERR_TIMEOUT, "hfr_trace_gmres: grid barrier wait timed out", -1, res.iterations);
  CK(cudaGetLastError());
  if (iters) *iters = res.iterations;
  if (final_rel) *final_rel = res.rel;
  if (res.nan) return set_err(ctx, FR_ERR_DIVERGED, "hfr_trace_gmres: non-finite residual", -1, res.iterations);
  if (!res.converged && res.rel > rtol)
    return set_err(ctx, FR_ERR_NOT_CONVERGED, "hfr_trace_gmres: iteration limit", -1, res.iterations, res.rel);
  return FR_OK;
}

extern "C" int imex_set_jacobian_policy(fr_ctx* ctx, int policy) {
  if (!ctx || (policy != FR_JAC_EVERY_NEWTON && policy != FR_JAC_ONCE_PER_STAGE && policy != FR_JAC_KEEP))
    return set_err(ctx, FR_ERR_INVALID_ARG, "imex_set_jacobian_policy: bad argument");
  if (ctx->gen && policy != FR_JAC_EVERY_NEWTON)
    return set_err(ctx, FR_ERR_UNSUPPORTED, "imex_set_jacobian_policy: general meshes re-linearise at every Newton iterate");
  ctx->jac_policy = policy;
  return FR_OK;
}

extern "C" int imex_refresh_jacobian(fr_ctx* ctx) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  ctx->keep_refresh = 1;
  return FR_OK;
}

extern "C" int hfr_gmres_set_mode(fr_ctx* ctx, int mode) {
  if (ctx && ctx->gen && mode == FR_GMRES_MULTI) return FR_OK;
  NOT_GENERAL(ctx, "hfr_gmres_set_mode (single-launch cycle)");
  if (!ctx || (mode != FR_GMRES_MULTI && mode != FR_GMRES_FUSED))
    return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_gmres_set_mode: bad argument");
  if (mode == FR_GMRES_FUSED && ctx->gm_fused_grid <= 0)
    return set_err(ctx, FR_ERR_UNSUPPORTED, "hfr_gmres_set_mode: no single-launch cycle for this shape or device");
  ctx->gm_mode = mode;
  return FR_OK;
}

extern "C" int hfr_gmres_get_mode(const fr_ctx* ctx) { return ctx ? ctx->gm_mode : -1; }

extern "C" int hfr_condense_set_mode(fr_ctx* ctx, int mode) {
  NOT_GENERAL(ctx, "hfr_condense_set_mode");
  if (!ctx || mode < FR_CONDENSE_FMA || mode > FR_CONDENSE_TENSOR_TF32)
    return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_condense_set_mode: bad argument");
  if ((mode == FR_CONDENSE_TENSOR_TF32 ? FR_CONDENSE_TENSOR : mode) >
      condense_tc_available(ctx->prec_bytes, ctx->nA, ctx->nT))
    return set_err(ctx, FR_ERR_UNSUPPORTED, "hfr_condense_set_mode: no tensor-core form for this precision or shape");
  ctx->cond_mode = mode;
  return FR_OK;
}

extern "C" int hfr_condense_get_mode(const fr_ctx* ctx) { return ctx ? ctx->cond_mode : -1; }

// Autotuner: time the compiled alternatives on the context's own blocks and keep the fastest.
static int autotune_uniform(fr_ctx* ctx, const double* u, const double* uhat, const double* ustar, double a_dt,
                            fr_tune_report* out);
extern "C" int hfr_autotune(fr_ctx* ctx, const double* u, const double* uhat, const double* ustar, double a_dt,
                            fr_tune_report* out) {
  FR_NVTX("hfr_autotune");
  NOT_GENERAL(ctx, "hfr_autotune");
  return autotune_uniform(ctx, u, uhat, ustar, a_dt, out);
}
static int autotune_uniform(fr_ctx* ctx, const double* u, const double* uhat, const double* ustar, double a_dt,
                            fr_tune_report* out) {
  if (!ctx || !u || (ctx->ntrace > 0 && !uhat) || !ustar) return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_autotune: null argument");
  fr_tune_report rep;
  memset(&rep, 0, sizeof(rep));
  for (int i = 0; i < 3; ++i) rep.condense_ms[i] = -1.0;
  for (int i = 0; i < 4; ++i) rep.inverse_ms[i] = -1.0;
  for (int i = 0; i < 2; ++i) rep.gmres_ms[i] = -1.0;
  if (ctx->Eim == 0) {
    if (out) *out = rep;
    return FR_OK;
  }
  int rc = hfr_local_jacobian(ctx, u, uhat, ustar, a_dt);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const bool prof = ctx->prof;
  ctx->prof = false;
  auto time_it = [&](auto&& fn, double* ms_out) -> int {
    int r = fn();  // warm-up (first-use attributes, caches)
    if (r) return r;
    float best = 1e30f;
    for (int rep_i = 0; rep_i < 2; ++rep_i) {
      CK(cudaEventRecord(e0, ctx->stream));
      r = fn();
      if (r) return r;
      CK(cudaEventRecord(e1, ctx->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      best = ms < best ? ms : best;
    }
    *ms_out = best;
    return FR_OK;
  };
  auto condense = [&]() -> int {
    const int r = condense_impl(ctx, 0);
    if (r) return r;
    return check_status(ctx, "hfr_autotune: zero pivot");
  };
  // condensation: every available mode; for the tensor-core inverse every residency 1..4 CTAs per SM
  const int avail = condense_tc_available(ctx->prec_bytes, ctx->nA, ctx->nT);
  int best_mode = ctx->cond_mode, best_ctas = ctx->inv_ctas;
  double best_ms = 1e30;
  for (int mode = 0; mode <= avail && !rc; ++mode) {
    ctx->cond_mode = mode;
    const int nv = mode == 2 ? 4 : 1;
    for (int v = 0; v < nv && !rc; ++v) {
      ctx->inv_ctas = mode == 2 ? v + 1 : 0;
      double ms = 0.0;
      rc = time_it(condense, &ms);
      if (rc) break;
      if (mode == 2) rep.inverse_ms[v] = ms;
      if (rep.condense_ms[mode] < 0.0 || ms < rep.condense_ms[mode]) rep.condense_ms[mode] = ms;
      if (ms < best_ms) {
        best_ms = ms;
        best_mode = mode;
        best_ctas = ctx->inv_ctas;
      }
    }
  }
  ctx->cond_mode = best_mode;
  ctx->inv_ctas = best_ctas;
  // GMRES cycle form (same iteration either way): on the condensed system of the chosen mode
  int best_gm = ctx->gm_mode;
  if (!rc && ctx->ntrace > 0) rc = condense();
  if (!rc && ctx->ntrace > 0) {
    double bg = 1e30;
    for (int mode = 1; mode >= 0 && !rc; --mode) {
      if (mode == 1 && ctx->gm_fused_grid <= 0) continue;
      ctx->gm_mode = mode;
      double ms = 0.0;
      rc = time_it([&]() -> int {
        int its = 0;
        double rel = 0.0;
        const int r = gmres_impl(ctx, ctx->duhat, 1e-4, 500, &its, &rel, false, nullptr);
        return r == FR_ERR_NOT_CONVERGED ? FR_OK : r;
      }, &ms);
      if (rc) break;
      rep.gmres_ms[mode] = ms;
      if (ms < bg) {
        bg = ms;
        best_gm = mode;
      }
    }
  }
  ctx->gm_mode = best_gm;
  ctx->gvalid = false;
  ctx->prof = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  rep.condense_mode = ctx->cond_mode;
  rep.inverse_ctas_per_sm = ctx->inv_ctas;
  rep.gmres_mode = ctx->gm_mode;
  if (out) *out = rep;
  return FR_OK;
}

// ------------------------------------------------------------------ modal filter (Appendix B)
// u[e][i][v] <- sum_k F[i][k] u[e][k][v] on the selected elements, F = V Lambda* V^{-1}; one thread
// per (element, variable) holds its column, so the update is in place.
template <int NS>
__global__ void k_modal_filter(int E, int nv, const double* __restrict__ F, const unsigned char* __restrict__ implicit,
                               int which, double* __restrict__ U) {
  __shared__ double sF[NS * NS];
  for (int i = threadIdx.x; i < NS * NS; i += blockDim.x) sF[i] = F[i];
  __syncthreads();
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)E * nv) return;
  const int e = (int)(t / nv), v = (int)(t % nv);
  if (which == 1 && !implicit[e]) return;
  if (which == 2 && implicit[e]) return;
  double* u = U + (size_t)e * NS * nv + v;
  double x[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) x[k] = u[(size_t)k * nv];
#pragma unroll 4
  for (int i = 0; i < NS; ++i) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < NS; ++k) acc += sF[i * NS + k] * x[k];
    u[(size_t)i * nv] = acc;
  }
}

// F = V Lambda* V^{-1} with V^{-1} = V^T W (the orthonormal basis is orthonormal under the tensor
// Gauss rule), V the tensor products of psi_k = sqrt((2k+1)/2) P_k at the Gauss points, Lambda* =
// sigma(i + j)^dt_ratio
static void modal_filter_operator(int p, double alpha, double s, int eta_c, double dt_ratio, double* F) {
  const int n = p + 1, ns = n * n, eta_max = 2 * p;
  double x[HFR_MAXN], w[HFR_MAXN], psi[HFR_MAXN][HFR_MAXN];  // psi[a][k] = psi_k(x_a)
  hfr::gauss_legendre_nodes(n, x, w);
  for (int a = 0; a < n; ++a) {
    double pm = 1.0, pk = x[a];
    for (int k = 0; k < n; ++k) {
      double P;
      if (k == 0) P = 1.0;
      else if (k == 1) P = x[a];
      else {
        const double pn = ((2.0 * k - 1.0) * x[a] * pk - (k - 1.0) * pm) / k;
        pm = pk;
        pk = pn;
        P = pn;
      }
      psi[a][k] = sqrt((2.0 * k + 1.0) / 2.0) * P;
    }
  }
  double lam[2 * HFR_MAXN];
  for (int eta = 0; eta <= eta_max; ++eta) {
    double sg = 1.0;
    if (eta >= eta_c) sg = eta_max > eta_c ? exp(-alpha * pow((double)(eta - eta_c) / (eta_max - eta_c), s)) : exp(-alpha);
    lam[eta] = pow(sg, dt_ratio);
  }
  for (int i = 0; i < ns; ++i) {
    const int a = i % n, b = i / n;
    for (int k = 0; k < ns; ++k) {
      const int ak = k % n, bk = k / n;
      double acc = 0.0;
      for (int jj = 0; jj < n; ++jj)
        for (int ii = 0; ii < n; ++ii) acc += psi[a][ii] * psi[b][jj] * lam[ii + jj] * psi[ak][ii] * psi[bk][jj];
      F[i * ns + k] = acc * w[ak] * w[bk];
    }
  }
}

extern "C" int fr_modal_filter(fr_ctx* ctx, double* u, double alpha, double s, int eta_c, double dt_ratio, int which) {
  FR_NVTX("fr_modal_filter");
  NOT_GENERAL(ctx, "fr_modal_filter");
  if (!ctx || !u || !(alpha >= 0.0) || !(s > 0.0) || eta_c < 0 || !(dt_ratio > 0.0) || which < 0 || which > 2)
    return set_err(ctx, FR_ERR_INVALID_ARG, "fr_modal_filter: bad argument");
  const int ns = ctx->ns;
  std::vector<double> F((size_t)ns * ns);
  modal_filter_operator(ctx->p, alpha, s, eta_c, dt_ratio, F.data());
  CK(cudaMemcpyAsync(ctx->filt, F.data(), F.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  const size_t nt = (size_t)ctx->E * ctx->nv;
  if (nt == 0) return FR_OK;
  const unsigned grid = nblk(nt, 128);
  switch (ns) {
    case 4: (hfr::count_launch(), k_modal_filter<4><<<grid, 128, 0, ctx->stream>>>(ctx->E, ctx->nv, ctx->filt, ctx->implicit, which, u)); break;
    case 9: (hfr::count_launch(), k_modal_filter<9><<<grid, 128, 0, ctx->stream>>>(ctx->E, ctx->nv, ctx->filt, ctx->implicit, which, u)); break;
    case 16: (hfr::count_launch(), k_modal_filter<16><<<grid, 128, 0, ctx->stream>>>(ctx->E, ctx->nv, ctx->filt, ctx->implicit, which, u)); break;
    case 25: (hfr::count_launch(), k_modal_filter<25><<<grid, 128, 0, ctx->stream>>>(ctx->E, ctx->nv, ctx->filt, ctx->implicit, which, u)); break;
    case 36: (hfr::count_launch(), k_modal_filter<36><<<grid, 128, 0, ctx->stream>>>(ctx->E, ctx->nv, ctx->filt, ctx->implicit, which, u)); break;
    default: return set_err(ctx, FR_ERR_UNSUPPORTED, "fr_modal_filter: degree");
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));  // the host operator buffer is released on return
  return FR_OK;
}

extern "C" int hfr_condense_uneven(int nelem, const int* nA, const int* nT, int precision, const void* A, const void* B,
                                   const void* C, const void* D, const double* r, const double* s, void* LU, int* piv,
                                   void* XB, double* xr, void* S, double* t, int* status, void* stream,
                                   int* failed_element) {
  FR_NVTX("hfr_condense_uneven");
  if (failed_element) *failed_element = -1;
  if (nelem < 0 || (nelem > 0 && (!nA || !nT || !A || !B || !C || !D || !r || !s || !LU || !piv || !XB || !xr || !S ||
                                  !t || !status)) ||
      (precision != FR_PREC_FP64 && precision != FR_PREC_FP32))
    return FR_ERR_INVALID_ARG;
  if (nelem == 0) return FR_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int init[2] = {0, 0x7fffffff};
  if (cudaMemcpyAsync(status, init, sizeof(init), cudaMemcpyHostToDevice, st) != cudaSuccess) return FR_ERR_CUDA;
  const cudaError_t e = launch_condense_uneven(precision == FR_PREC_FP64 ? 8 : 4, nelem, nA, nT, A, B, C, D, r, s, LU,
                                               piv, XB, xr, S, t, status, st);
  if (e == cudaErrorInvalidValue) {
    cudaGetLastError();
    return FR_ERR_INVALID_ARG;
  }
  if (e != cudaSuccess) return FR_ERR_CUDA;
  int hs[2] = {0, 0};
  if (cudaMemcpyAsync(hs, status, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FR_ERR_CUDA;
  if (hs[0] & DEV_ERR_SINGULAR) {
    if (failed_element) *failed_element = hs[1];
    return FR_ERR_SINGULAR;
  }
  return FR_OK;
}

extern "C" int fr_barrier_selftest(int nblocks, int absent_block, int rounds, double timeout_s,
                                   int* barriers_passed, void* stream) {
  if (!barriers_passed || !(timeout_s > 0.0) || timeout_s > 10.0) return FR_ERR_INVALID_ARG;
  int timed_out = 0;
  const int rc = hfr::barrier_selftest(nblocks, absent_block, rounds, timeout_s, barriers_passed, &timed_out,
                                       (cudaStream_t)stream);
  if (rc == -2) return FR_ERR_INVALID_ARG;
  if (rc != 0) return FR_ERR_CUDA;
  return timed_out ? FR_ERR_TIMEOUT : FR_OK;
}

extern "C" int hfr_trace_gmres(fr_ctx* ctx, double* duhat, double rtol, int maxit, int* iters, double* final_rel) {
  FR_NVTX("hfr_trace_gmres");
  if (ctx && ctx->gen) {
    if (!duhat) return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_trace_gmres: null argument");
    const int grc = hfr::gen::trace_gmres(ctx->gen, duhat, rtol, maxit, iters, final_rel);
    prof_collect(ctx);
    return grc;
  }
  if (!ctx || !duhat || rtol < 0 || maxit < 1) return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_trace_gmres: bad argument");
  const int rc = gmres_impl(ctx, duhat, rtol, maxit, iters, final_rel);
  prof_collect(ctx);
  return rc;
}

static int backsolve_impl(fr_ctx* ctx, const double* duhat, double* du, int refine) {
  if (ctx->Eim == 0) return FR_OK;
  TraceArgs t = trace_args(ctx);
  const int ph = prof_begin(ctx, PH_BACK);
  CK(launch_backsolve(ctx->prec_bytes, t, ctx->Eim, ctx->nA, ctx->XB, ctx->xr, duhat, du, ctx->stream));
  int rc = FR_OK;
  if (refine > 0 && ctx->lin_U) rc = refine_local(ctx, ctx->r, du, duhat, refine);
  prof_end(ctx, ph);
  return rc;
}

extern "C" int hfr_backsolve(fr_ctx* ctx, const double* duhat, double* du, int refine) {
  FR_NVTX("hfr_backsolve");
  if (ctx && ctx->gen) {
    if (!du || (ctx->ntrace > 0 && !duhat)) return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_backsolve: null argument");
    const int grc = hfr::gen::backsolve(ctx->gen, duhat, du, refine);
    prof_collect(ctx);
    return grc;
  }
  if (!ctx || !du || (ctx->ntrace > 0 && !duhat)) return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_backsolve: null argument");
  int rc = backsolve_impl(ctx, duhat, du, refine);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  prof_collect(ctx);
  return FR_OK;
}

// the context array `which` of hfr_export / hfr_import and its size in bytes (nullptr: unknown)
static void* ctx_array(fr_ctx* ctx, int which, size_t* need) {
  const size_t pb = ctx->prec_bytes, Eim = ctx->Eim, nA = ctx->nA, nT = ctx->nT;
  switch (which) {
    case 0: *need = Eim * nA * nA * pb; return ctx->A;
    case 1: *need = Eim * nA * nT * pb; return ctx->B;
    case 2: *need = Eim * nT * nA * pb; return ctx->C;
    case 3: *need = Eim * nT * nT * pb; return ctx->D;
    case 4: *need = Eim * nT * nT * pb; return ctx->S;
    case 5: *need = Eim * nA * nT * pb; return ctx->XB;
    case 6: *need = Eim * nA * 8; return ctx->xr;
    case 7: *need = Eim * nT * 8; return ctx->te;
    case 8: *need = Eim * nA * 8; return ctx->r;
    case 9: *need = Eim * nT * 8; return ctx->s;
    case 10: *need = (size_t)ctx->ntrace * ctx->n * ctx->nv * 8; return ctx->tg;
    case 11: *need = (size_t)ctx->ntrace * (ctx->n * ctx->nv) * (ctx->n * ctx->nv) * pb; return ctx->Pinv;
  }
  *need = 0;
  return nullptr;
}

extern "C" int hfr_import(fr_ctx* ctx, int which, const void* src, size_t bytes) {
  if (!ctx || !src) return FR_ERR_INVALID_ARG;
  if (ctx->gen) {
#ifdef FR_CHECKED
    const bool map = which == 64;  // the face-point trace map, a planted defect in checked builds
#else
    const bool map = false;
#endif
    if ((which < 0 || which > 9) && !map) return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_import: array not importable");
    return hfr::gen::export_array(ctx->gen, which, const_cast<void*>(src), bytes, true);
  }
  if (which < 0 || which > 9) return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_import: array not importable");
  size_t need = 0;
  void* dst = ctx_array(ctx, which, &need);
  if (!dst) return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_import: unknown array");
  if (bytes != need) return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_import: size differs from the context array");
  ctx->keep_valid = 0;  // a held condensation no longer matches the blocks
  CK(cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FR_OK;
}

extern "C" int hfr_export(fr_ctx* ctx, int which, void* dst, size_t bytes) {
  if (!ctx || !dst) return FR_ERR_INVALID_ARG;
  if (ctx->gen) return hfr::gen::export_array(ctx->gen, which, dst, bytes, false);
  size_t need = 0;
  const void* src = ctx_array(ctx, which, &need);
  if (!src) return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_export: unknown array");
  if (bytes < need) return set_err(ctx, FR_ERR_INVALID_ARG, "hfr_export: destination too small");
  CK(cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FR_OK;
}

// ------------------------------------------------------------------------ tableaux
struct Tab {
  int s;
  double a[2][2], b[2], ah[3][3], bh[3];
};
static Tab tableau(int which) {
  Tab t;
  memset(&t, 0, sizeof(t));
  if (which == FR_TAB_SDIRK2) {
    const double g = 1.0 - sqrt(2.0) / 2.0, dl = -2.0 * sqrt(2.0) / 3.0;
    t.s = 2;
    t.a[0][0] = g;
    t.a[1][0] = 1.0 - g;
    t.a[1][1] = g;
    t.b[0] = 1.0 - g;
    t.b[1] = g;
    t.ah[1][0] = g;
    t.ah[2][0] = dl;
    t.ah[2][1] = 1.0 - dl;
    t.bh[1] = 1.0 - g;
    t.bh[2] = g;
  } else {
    t.s = 1;
    t.a[0][0] = 1.0;
    t.b[0] = 1.0;
    t.ah[1][0] = 1.0;
    t.bh[1] = 1.0;
  }
  return t;
}

static int sumsq(fr_ctx* ctx, const double* a, size_t na, const double* b, size_t nb, double* out_host) {
  const int nbk = 256;
  (hfr::count_launch(), k_sumsq_part<<<nbk, 256, 0, ctx->stream>>>(a, na, b, nb, ctx->red));
  (hfr::count_launch(), k_sumsq_final<<<1, 32, 0, ctx->stream>>>(ctx->red, nbk, ctx->red + 1024));
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out_host, ctx->red + 1024, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FR_OK;
}

// ------------------------------------------------------------------ whole-stage CUDA graph
// The implicit stage as one executable graph: the Newton loop is a WHILE node, its linear solve
// an IF node (skipped on the iteration that finds the residual converged) and the GMRES restart
// cycles a nested WHILE node.  Small kernels decide on the device what the host decides in the
// stream path (same tests, same order), so one graph launch runs the whole stage and the host
// reads the counters once at the end.
__global__ void k_stage_init(StageDev* sd) {
  sd->norm0 = -1.0;
  sd->norm = 0.0;
  sd->it = 0;
  sd->gtot = 0;
  sd->conv = 0;
  sd->err = 0;
  sd->gm_total = 0;
  sd->cycles = 0;
}

__global__ void k_newton_check(StageDev* sd, const double* ss, double tol, int maxit, cudaGraphConditionalHandle hn,
                               cudaGraphConditionalHandle hs) {
  const double nrm = sqrt(*ss);
  if (sd->norm0 < 0.0) sd->norm0 = nrm;
  sd->norm = nrm;
  if (!(nrm == nrm)) sd->err |= 1;
  const int conv = (nrm <= tol * sd->norm0 || nrm == 0.0) ? 1 : 0;
  sd->conv = conv;
  const int cont = (!conv && sd->err == 0 && sd->it < maxit) ? 1 : 0;
  if (cont) sd->it += 1;
  cudaGraphSetConditional(hn, (unsigned)cont);
  cudaGraphSetConditional(hs, (unsigned)cont);
}

__global__ void k_gmres_begin(StageDev* sd, int m, int maxit, cudaGraphConditionalHandle hg) {
  sd->gm_total = 0;
  sd->dyn[0] = 1;
  sd->dyn[1] = m < maxit ? m : maxit;
  cudaGraphSetConditional(hg, 1u);
}

__global__ void k_gmres_after(StageDev* sd, const GmresState* st, const unsigned* bar, int m, int maxit,
                              cudaGraphConditionalHandle hg) {
  int cont = 0;
  if (bar[1] != 0u) {
    sd->err |= 4;
  } else {
    sd->gm_total += st->k;
    sd->cycles += 1;
    if (st->nan) sd->err |= 2;
    cont = (st->nan || st->converged || sd->gm_total >= maxit || st->k == 0) ? 0 : 1;
    const int rem = maxit - sd->gm_total;
    sd->dyn[0] = 0;
    sd->dyn[1] = m < rem ? m : rem;
  }
  cudaGraphSetConditional(hg, (unsigned)cont);
}

__global__ void k_gmres_end(StageDev* sd) { sd->gtot += sd->gm_total; }

// a conditional node after the work captured so far on s; returns its body graph
cudaError_t hfr::graph_add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                       cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  // zeroed storage (the struct's union has no default constructor)
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams& p = *reinterpret_cast<cudaGraphNodeParams*>(raw);
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p)) != cudaSuccess) return e;
  *body = p.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// a conditional handle of the graph that s is capturing into
cudaError_t hfr::graph_conditional_handle(cudaStream_t s, unsigned dflt, unsigned flags, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  return cudaGraphConditionalHandleCreate(h, g, dflt, flags);
}
using hfr::graph_add_conditional;
static inline cudaError_t add_conditional(cudaStream_t s, cudaGraphConditionalHandle h,
                                          cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  return graph_add_conditional(s, h, type, body);
}

static int stage_graph_capture(fr_ctx* ctx, const StageGraphKey& key) {
  const Tab tb = tableau(ctx->tableau);
  const int i = key.stage, E = ctx->E, nA = ctx->nA;
  const size_t tot = (size_t)E * nA;
  const size_t nh = (size_t)ctx->ntrace * ctx->n * ctx->nv;
  for (auto& c : ctx->cap)
    if (!c) CK(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
  cudaStream_t user = ctx->stream;
  const bool prof = ctx->prof;
  ctx->prof = false;
  cudaGraph_t g = nullptr, bn = nullptr, bs = nullptr, bg = nullptr;
  int depth = 0;  // capture streams currently capturing
  int rc = FR_OK;
  unsigned long long l0 = 0, l1 = 0, l2 = 0, l3 = 0, l4 = 0, l5 = 0, l6 = 0;
  auto fail = [&](int code) {
    for (int d = depth - 1; d >= 0; --d) {
      cudaGraph_t tmp = nullptr;
      cudaStreamEndCapture(ctx->cap[d], &tmp);
    }
    ctx->stream = user;
    ctx->prof = prof;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return code ? code : FR_ERR_CUDA;
  };
#define GK(x)                                                         \
  do {                                                                \
    cudaError_t e_ = (x);                                             \
    if (e_ != cudaSuccess) {                                          \
      set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e_));              \
      return fail(FR_ERR_CUDA);                                       \
    }                                                                 \
  } while (0)
#define GR(x)                     \
  do {                            \
    const int r_ = (x);           \
    if (r_ != FR_OK) return fail(r_); \
  } while (0)
  GK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle hn;
  GK(cudaGraphConditionalHandleCreate(&hn, g, 1u, cudaGraphCondAssignDefault));
  // ---- top level: stage combination, u*, counters
  GK(cudaStreamBeginCaptureToGraph(ctx->cap[0], g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  depth = 1;
  ctx->stream = ctx->cap[0];
  l0 = fr_kernel_launches();
  {
    StageCoef sc;
    memset(&sc, 0, sizeof(sc));
    sc.nterm = i;
    for (int j = 0; j < i; ++j) {
      sc.hi[j] = j;
      sc.ce[j] = key.dt * tb.ah[i][j];
      sc.ci[j] = j >= 1 ? key.dt * tb.a[i - 1][j - 1] : 0.0;
    }
    (hfr::count_launch(), k_stage_combine<<<nblk(tot), 256, 0, ctx->stream>>>(E, nA, ctx->implicit, key.u_n, key.R_hist,
                                                                                sc, const_cast<double*>(key.u_stage)));
    GK(cudaGetLastError());
  }
  GK(cudaMemcpyAsync(ctx->Ustar, key.u_stage, tot * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  (hfr::count_launch(), k_stage_init<<<1, 1, 0, ctx->stream>>>(ctx->sdev));
  GK(cudaGetLastError());
  const double adt = key.dt * tb.a[i - 1][i - 1];
  double* u_stage = const_cast<double*>(key.u_stage);
  double* uhat = const_cast<double*>(key.uhat);
  GK(add_conditional(ctx->cap[0], hn, cudaGraphCondTypeWhile, &bn));
  l1 = fr_kernel_launches();
  // ---- Newton body: residual, right-hand sides, norm test
  cudaGraphConditionalHandle hs;
  GK(cudaGraphConditionalHandleCreate(&hs, bn, 0u, 0u));
  GK(cudaStreamBeginCaptureToGraph(ctx->cap[1], bn, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  depth = 2;
  ctx->stream = ctx->cap[1];
  GR(residual_into(ctx, u_stage, uhat, ctx->Rw, ctx->gview, ctx->gw));
  GR(form_rhs(ctx, u_stage, ctx->Ustar, adt));
  {
    const int nbk = 256;
    (hfr::count_launch(), k_sumsq_part<<<nbk, 256, 0, ctx->stream>>>(ctx->r, (size_t)ctx->Eim * nA, ctx->gw, nh, ctx->red));
    (hfr::count_launch(), k_sumsq_final<<<1, 32, 0, ctx->stream>>>(ctx->red, nbk, ctx->red + 1024));
    (hfr::count_launch(), k_newton_check<<<1, 1, 0, ctx->stream>>>(ctx->sdev, ctx->red + 1024, key.ntol, key.nmax, hn, hs));
    GK(cudaGetLastError());
  }
  GK(add_conditional(ctx->cap[1], hs, cudaGraphCondTypeIf, &bs));
  l2 = fr_kernel_launches();
  // ---- solve body: blocks, condensation, GMRES cycles, back-substitution, update
  GK(cudaStreamBeginCaptureToGraph(ctx->cap[2], bs, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  depth = 3;
  ctx->stream = ctx->cap[2];
  GR(jacobian_blocks(ctx, u_stage, uhat, adt));
  GR(condense_impl(ctx, 0));
  if (ctx->ntrace > 0) {
    FusedArgs fa;
    fa.ntrace = ctx->ntrace;
    fa.nT = ctx->nT;
    fa.sides = ctx->sides_c;
    fa.tr_of_c = ctx->tr_of_c;
    fa.S = ctx->S16 ? (const void*)ctx->S16 : ctx->S;
    fa.s_bf16 = ctx->S16 ? 1 : 0;
    fa.S_bytes = (size_t)ctx->Eim * ctx->nT * ctx->nT * (ctx->S16 ? 2 : ctx->prec_bytes);
    fa.Pinv = ctx->Pinv;
    fa.t = ctx->tg;
    fa.x = ctx->duhat;
    fa.V = ctx->gm.V;
    fa.z = ctx->prec_bytes == 4 ? (void*)ctx->gm.z32 : (void*)ctx->gm.Z;
    fa.partial = ctx->gm.partial;
    fa.bar = ctx->gm_bar;
    fa.st = ctx->gm.state;
    fa.n = ctx->gm.n;
    fa.m = ctx->restart > GM_MAXM ? GM_MAXM : ctx->restart;
    fa.rtol = key.grtol;
    fa.x_zero = 1;
    fa.true_res = 0;
    fa.dyn = ctx->sdev->dyn;
    cudaGraphConditionalHandle hg;
    GK(cudaGraphConditionalHandleCreate(&hg, bs, 0u, 0u));
    GK(cudaMemsetAsync(ctx->duhat, 0, nh * sizeof(double), ctx->stream));
    (hfr::count_launch(), k_gmres_begin<<<1, 1, 0, ctx->stream>>>(ctx->sdev, fa.m, key.gmax, hg));
    GK(cudaGetLastError());
    GK(add_conditional(ctx->cap[2], hg, cudaGraphCondTypeWhile, &bg));
    l3 = fr_kernel_launches();
    // ---- GMRES body: one restart cycle and the device-side restart decision
    GK(cudaStreamBeginCaptureToGraph(ctx->cap[3], bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    depth = 4;
    ctx->stream = ctx->cap[3];
    GK(cudaMemsetAsync(ctx->gm_bar, 0, 2 * sizeof(unsigned), ctx->stream));
    GK(launch_gmres_cycle(fa, ctx->prec_bytes, ctx->gm_fused_grid, ctx->stream));
    (hfr::count_launch(), k_gmres_after<<<1, 1, 0, ctx->stream>>>(ctx->sdev, ctx->gm.state, ctx->gm_bar, fa.m, key.gmax, hg));
    GK(cudaGetLastError());
    GK(cudaStreamEndCapture(ctx->cap[3], &bg));
    depth = 3;
    l4 = fr_kernel_launches();
    ctx->stream = ctx->cap[2];
    (hfr::count_launch(), k_gmres_end<<<1, 1, 0, ctx->stream>>>(ctx->sdev));
    GK(cudaGetLastError());
  } else {
    l3 = l4 = fr_kernel_launches();
  }
  GR(backsolve_impl(ctx, ctx->duhat, ctx->du, key.refine));
  (hfr::count_launch(), k_apply_du<<<nblk((size_t)ctx->Eim * nA), 256, 0, ctx->stream>>>(ctx->Eim, nA, ctx->imp_idx, ctx->du, u_stage));
  GK(cudaGetLastError());
  if (nh) {
    (hfr::count_launch(), k_axpy<<<nblk(nh), 256, 0, ctx->stream>>>(nh, 1.0, ctx->duhat, uhat));
    GK(cudaGetLastError());
  }
  GK(cudaStreamEndCapture(ctx->cap[2], &bs));
  depth = 2;
  l5 = fr_kernel_launches();
  GK(cudaStreamEndCapture(ctx->cap[1], &bn));
  depth = 1;
  // ---- after the loop: R_hist[i] = R(u_i, u^_i), the last residual the loop evaluated
  ctx->stream = ctx->cap[0];
  GK(cudaMemcpyAsync(const_cast<double*>(key.R_hist) + (size_t)i * tot, ctx->Rw, tot * sizeof(double),
                     cudaMemcpyDeviceToDevice, ctx->stream));
  GK(cudaStreamEndCapture(ctx->cap[0], &g));
  depth = 0;
  l6 = fr_kernel_launches();
  ctx->stream = user;
  ctx->prof = prof;
  cudaGraphExec_t ex = nullptr;
  {
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      cudaGetLastError();
      return set_err(ctx, FR_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->graph = g;
  ctx->gexec = ex;
  ctx->gkey = key;
  ctx->gvalid = true;
  // capture counted each kernel once: the launches of one replay follow from the iteration counts
  g_launches.fetch_sub(l6 - l0, std::memory_order_relaxed);
  ctx->gl_top = (int)((l1 - l0) + (l6 - l5));
  ctx->gl_newton = (int)(l2 - l1);
  ctx->gl_cycle = (int)(l4 - l3);
  ctx->gl_solve = (int)((l5 - l2) - (l4 - l3));
#undef GK
#undef GR
  return rc;
}

static int imex_stage_graph(fr_ctx* ctx, const StageGraphKey& key, fr_stage_stats* stats) {
  if (!ctx->gvalid || !(ctx->gkey == key)) {
    const int rc = stage_graph_capture(ctx, key);
    if (rc) return rc;
  }
  cudaStream_t st = ctx->stream;
  CK(cudaGraphLaunch(ctx->gexec, st));
  StageDev h;
  int hs[2] = {0, 0};
  CK(cudaMemcpyAsync(&h, ctx->sdev, sizeof(h), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hs, ctx->status, sizeof(hs), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const unsigned long long n = (unsigned long long)ctx->gl_top + (unsigned long long)(h.it + 1) * ctx->gl_newton +
                               (unsigned long long)h.it * ctx->gl_solve + (unsigned long long)h.cycles * ctx->gl_cycle;
  g_launches.fetch_add(n, std::memory_order_relaxed);
  if (stats) {
    stats->newton_iterations = h.it;
    stats->gmres_iterations = h.gtot;
    stats->residual0 = h.norm0;
    stats->residual = h.norm;
    stats->converged = h.conv;
  }
  if (hs[0] & DEV_ERR_SINGULAR) {
    CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), st));
    return set_err(ctx, FR_ERR_SINGULAR, "imex_stage: zero pivot in condensation", hs[1]);
  }
  if ((hs[0] & DEV_ERR_TIMEOUT) || (h.err & 4)) {
    CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), st));
    return set_err(ctx, FR_ERR_TIMEOUT, "imex_stage: a bounded device wait timed out", -1, h.it);
  }
  if (h.err & 1) return set_err(ctx, FR_ERR_DIVERGED, "imex_stage: non-finite Newton residual", -1, h.it);
  if (h.err & 2) return set_err(ctx, FR_ERR_DIVERGED, "imex_stage: non-finite GMRES residual", -1, h.it);
  if (!h.conv) return set_err(ctx, FR_ERR_NOT_CONVERGED, "imex_stage: Newton iteration limit", -1, h.it, h.norm);
  return FR_OK;
}

extern "C" int imex_stage_set_graph(fr_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return set_err(ctx, FR_ERR_INVALID_ARG, "imex_stage_set_graph: bad argument");
  if (ctx->gen) {
    const int rc = hfr::gen::set_graph(ctx->gen, on);
    if (rc == FR_OK) ctx->use_graph = on;
    return rc;
  }
  if (on && (ctx->Eim == 0 || (ctx->ntrace > 0 && ctx->gm_mode != 1)))
    return set_err(ctx, FR_ERR_UNSUPPORTED, "imex_stage_set_graph: needs implicit elements and the single-launch GMRES cycle");
  ctx->use_graph = on;
  ctx->gvalid = false;
  return FR_OK;
}

extern "C" int imex_stage_get_graph(const fr_ctx* ctx) { return ctx ? ctx->use_graph : -1; }

extern "C" int imex_stage(fr_ctx* ctx, int stage, double dt, const double* u_n, double* u_stage, double* uhat,
                          double* R_hist, double newton_tol, int newton_maxit, double gmres_rtol, int gmres_maxit,
                          int refine, fr_stage_stats* stats) {
  FR_NVTX("imex_stage");
  if (!ctx || !u_n || !u_stage || !R_hist || (ctx->ntrace > 0 && !uhat))
    return set_err(ctx, FR_ERR_INVALID_ARG, "imex_stage: null argument");
  if (ctx->gen) {
    const int grc = hfr::gen::stage(ctx->gen, stage, dt, u_n, u_stage, uhat, R_hist, newton_tol, newton_maxit,
                                    gmres_rtol, gmres_maxit, refine, stats);
    prof_collect(ctx);
    return grc;
  }
  const Tab tb = tableau(ctx->tableau);
  if (stage < 0 || stage > tb.s + 1) return set_err(ctx, FR_ERR_INVALID_ARG, "imex_stage: stage out of range");
  const int E = ctx->E, nA = ctx->nA;
  const size_t tot = (size_t)E * nA;
  cudaStream_t st = ctx->stream;
  if (stats) memset(stats, 0, sizeof(*stats));
  if (stage == 0) {
    int rc = residual_into(ctx, u_n, uhat, R_hist, ctx->gview, nullptr);
    if (rc) return rc;
    CK(cudaStreamSynchronize(st));
    return FR_OK;
  }
  if (stage == tb.s + 1) {
    StageCoef sc;
    memset(&sc, 0, sizeof(sc));
    sc.nterm = tb.s + 1;
    for (int j = 0; j <= tb.s; ++j) {
      sc.hi[j] = j;
      sc.ci[j] = j >= 1 ? dt * tb.b[j - 1] : 0.0;  // implicit: b_j R(u_j)
      sc.ce[j] = dt * tb.bh[j];                    // explicit: bhat_{j+1} R(u_j)
    }
    (hfr::count_launch(), k_stage_combine<<<nblk(tot), 256, 0, st>>>(E, nA, ctx->implicit, u_n, R_hist, sc, u_stage));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return FR_OK;
  }
  if (ctx->use_graph) {
    if (ctx->jac_policy != FR_JAC_EVERY_NEWTON || (ctx->ntrace > 0 && ctx->gm_mode != 1))
      return set_err(ctx, FR_ERR_UNSUPPORTED, "imex_stage: the graph runs the exact-Newton, single-launch GMRES stage");
    StageGraphKey key{stage, newton_maxit, gmres_maxit, refine, dt, newton_tol, gmres_rtol, u_n, u_stage, uhat, R_hist};
    return imex_stage_graph(ctx, key, stats);
  }
  const int i = stage;
  // explicit elements: u_i = u_n + dt sum_{j<=i} ahat_{i+1,j} R_hist[j-1];
  // implicit elements: u* = u_n + dt sum_{j<i} a_ij R_hist[j]  (also the Newton start)
  StageCoef sc;
  memset(&sc, 0, sizeof(sc));
  sc.nterm = i;
  for (int j = 0; j < i; ++j) {
    sc.hi[j] = j;
    sc.ce[j] = dt * tb.ah[i][j];
    sc.ci[j] = j >= 1 ? dt * tb.a[i - 1][j - 1] : 0.0;
  }
  (hfr::count_launch(), k_stage_combine<<<nblk(tot), 256, 0, st>>>(E, nA, ctx->implicit, u_n, R_hist, sc, u_stage));
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(ctx->Ustar, u_stage, tot * sizeof(double), cudaMemcpyDeviceToDevice, st));
  const double adt = dt * tb.a[i - 1][i - 1];
  const size_t nh = (size_t)ctx->ntrace * ctx->n * ctx->nv;
  double norm0 = -1.0, normk = 0.0;
  int it = 0, gtot = 0;
  bool conv = false;
  for (;; ++it) {
    int rc = residual_into(ctx, u_stage, uhat, ctx->Rw, ctx->gview, ctx->gw);
    const int phn = prof_begin(ctx, PH_NEWTON);
    if (!rc) rc = form_rhs(ctx, u_stage, ctx->Ustar, adt);
    double ss = 0.0;
    if (!rc) rc = sumsq(ctx, ctx->r, (size_t)ctx->Eim * nA, ctx->gw, nh, &ss);
    prof_end(ctx, phn);
    if (rc) return rc;
    normk = sqrt(ss);
    if (!(normk == normk)) return set_err(ctx, FR_ERR_DIVERGED, "imex_stage: non-finite Newton residual", -1, it);
    if (norm0 < 0) norm0 = normk;
    if (normk <= newton_tol * norm0 || normk == 0.0) {
      conv = true;
      break;
    }
    if (it >= newton_maxit) break;
    bool fresh;
    if (ctx->jac_policy == FR_JAC_KEEP)
      fresh = it == 0 && (!ctx->keep_valid || ctx->keep_adt != adt || ctx->keep_refresh);
    else
      fresh = it == 0 || ctx->jac_policy == FR_JAC_EVERY_NEWTON;
    if (fresh) {
      ctx->keep_valid = 0;
      rc = jacobian_blocks(ctx, u_stage, uhat, adt);
      // the local solves are refined once, at the back-substitution (du = A^{-1}(r - B du^));
      // refining x_r as well would not change the converged step
      if (!rc) rc = condense_impl(ctx, 0);
      ++ctx->jac_refreshes;
    } else {
      // chord iteration: blocks, factors, S_k and preconditioner of an earlier iterate (this
      // stage's first, or with FR_JAC_KEEP an earlier stage's or step's)
      rc = condense_rhs_impl(ctx);
    }
    if (rc) return rc;
    int its = 0;
    double rel = 0.0;
    int cst[2] = {0, 0};
    rc = gmres_impl(ctx, ctx->duhat, gmres_rtol, gmres_maxit, &its, &rel, false, cst);
    if (cst[0] & DEV_ERR_SINGULAR) {
      CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), st));
      return set_err(ctx, FR_ERR_SINGULAR, "imex_stage: zero pivot in condensation", cst[1]);
    }
    if (cst[0] & DEV_ERR_TIMEOUT) {
      CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), st));
      return set_err(ctx, FR_ERR_TIMEOUT, "imex_stage: tensor-core completion wait timed out");
    }
    if (fresh) {  // a factorisation without a zero pivot: held for later chord iterations
      ctx->keep_valid = 1;
      ctx->keep_adt = adt;
      ctx->keep_refresh = 0;
    }
    gtot += its;
    if (rc && rc != FR_ERR_NOT_CONVERGED) return rc;
    rc = backsolve_impl(ctx, ctx->duhat, ctx->du, refine);
    if (rc) return rc;
    const int phu = prof_begin(ctx, PH_NEWTON);
    (hfr::count_launch(), k_apply_du<<<nblk((size_t)ctx->Eim * nA), 256, 0, st>>>(ctx->Eim, nA, ctx->imp_idx, ctx->du, u_stage));
    CK(cudaGetLastError());
    if (nh) {
      (hfr::count_launch(), k_axpy<<<nblk(nh), 256, 0, st>>>(nh, 1.0, ctx->duhat, uhat));
      CK(cudaGetLastError());
    }
    prof_end(ctx, phu);
  }
  // R_hist[i] = R(u_i, u^_i): the loop leaves right after evaluating R at the final state
  CK(cudaMemcpyAsync(R_hist + (size_t)i * tot, ctx->Rw, tot * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  prof_collect(ctx);
  if (stats) {
    stats->newton_iterations = it;
    stats->gmres_iterations = gtot;
    stats->residual0 = norm0;
    stats->residual = normk;
    stats->converged = conv ? 1 : 0;
  }
  if (!conv) return set_err(ctx, FR_ERR_NOT_CONVERGED, "imex_stage: Newton iteration limit", -1, it, normk);
  return FR_OK;
}

// nsteps IMEX steps in place: per step, stage 0 (R at u_n), the implicit stages 1..s and the
// final combination into u_stage, copied back to u.  With FR_JAC_KEEP the held condensation is
// refreshed at every refresh_every-th step (and whenever a_ii dt changes or none is held).
extern "C" int imex_steps(fr_ctx* ctx, int nsteps, double dt, double* u, double* uhat, double* R_hist,
                          double* u_stage, int refresh_every, double newton_tol, int newton_maxit,
                          double gmres_rtol, int gmres_maxit, int refine, fr_steps_stats* stats) {
  FR_NVTX("imex_steps");
  if (!ctx || !u || !R_hist || !u_stage || (ctx->ntrace > 0 && !uhat) || nsteps < 0 || !(dt > 0.0))
    return set_err(ctx, FR_ERR_INVALID_ARG, "imex_steps: bad argument");
  const Tab tb = tableau(ctx->tableau);
  if (ctx->gen && ctx->jac_policy != FR_JAC_EVERY_NEWTON)
    return set_err(ctx, FR_ERR_UNSUPPORTED, "imex_steps: general meshes re-linearise at every Newton iterate");
  fr_steps_stats acc;
  memset(&acc, 0, sizeof(acc));
  acc.converged = 1;
  const long long r0 = ctx->jac_refreshes;
  int rc = FR_OK;
  for (int k = 0; k < nsteps && rc == FR_OK; ++k) {
    if (ctx->jac_policy == FR_JAC_KEEP && refresh_every > 0 && k % refresh_every == 0) ctx->keep_refresh = 1;
    rc = imex_stage(ctx, 0, dt, u, u_stage, uhat, R_hist, newton_tol, newton_maxit, gmres_rtol, gmres_maxit,
                    refine, nullptr);
    for (int i = 1; i <= tb.s && rc == FR_OK; ++i) {
      fr_stage_stats ss;
      rc = imex_stage(ctx, i, dt, u, u_stage, uhat, R_hist, newton_tol, newton_maxit, gmres_rtol, gmres_maxit,
                      refine, &ss);
      acc.newton_iterations += ss.newton_iterations;
      acc.gmres_iterations += ss.gmres_iterations;
      const double rel = ss.residual0 > 0.0 ? ss.residual / ss.residual0 : 0.0;
      if (rel > acc.max_rel_residual) acc.max_rel_residual = rel;
      if (!ss.converged) acc.converged = 0;
    }
    if (rc == FR_OK)
      rc = imex_stage(ctx, tb.s + 1, dt, u, u_stage, uhat, R_hist, newton_tol, newton_maxit, gmres_rtol,
                      gmres_maxit, refine, nullptr);
    if (rc == FR_OK) {
      const size_t nst = ctx->gen ? hfr::gen::state_values(ctx->gen) : (size_t)ctx->E * ctx->nA;
      if (cudaMemcpyAsync(u, u_stage, nst * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
        rc = set_err(ctx, FR_ERR_CUDA, "imex_steps: copy of u_{n+1}");
      else
        ++acc.steps;
    }
  }
  if (rc != FR_OK) acc.converged = 0;
  acc.jacobian_refreshes = (int)(ctx->jac_refreshes - r0);
  CK(cudaStreamSynchronize(ctx->stream));
  if (stats) *stats = acc;
  return rc;
}

extern "C" int fr_profile_enable(fr_ctx* ctx, int on) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  prof_collect(ctx);
  if (on && ctx->evpool.empty()) {
    ctx->evpool.resize(4096);
    for (auto& e : ctx->evpool) CK(cudaEventCreate(&e));
  }
  ctx->prof = on != 0;
  if (on)
    for (int i = 0; i < 10; ++i) {
      ctx->pms[i] = 0.0;
      ctx->pcnt[i] = 0;
    }
  return FR_OK;
}

extern "C" int fr_profile_read(const fr_ctx* ctx, fr_profile* out) {
  if (!ctx || !out) return FR_ERR_INVALID_ARG;
  for (int i = 0; i < 10; ++i) {
    out->ms[i] = ctx->pms[i];
    out->count[i] = ctx->pcnt[i];
  }
  return FR_OK;
}

extern "C" unsigned long long fr_kernel_launches(void) { return g_launches.load(); }

extern "C" int fr_checked_status(unsigned long long* first, unsigned long long* count) {
  if (!first || !count) return FR_ERR_INVALID_ARG;
  *first = 0;
  *count = 0;
#ifdef FR_CHECKED
  for (ChkCollect f : checked_units()) {
    unsigned long long a = 0, c = 0;
    if (f(&a, &c) != 0) return FR_ERR_CUDA;
    if (*first == 0 && a != 0) *first = a;
    *count += c;
  }
  return FR_OK;
#else
  return FR_ERR_UNSUPPORTED;
#endif
}

extern "C" int fr_last_error(const fr_ctx* ctx, fr_error_info* info) {
  if (!ctx || !info) return FR_ERR_INVALID_ARG;
  *info = ctx->err;
  return FR_OK;
}

extern "C" const char* fr_status_string(int code) {
  switch (code) {
    case FR_OK: return "ok";
    case FR_ERR_INVALID_ARG: return "invalid argument";
    case FR_ERR_CUDA: return "CUDA error";
    case FR_ERR_SINGULAR: return "singular block";
    case FR_ERR_NOT_CONVERGED: return "not converged";
    case FR_ERR_DIVERGED: return "diverged";
    case FR_ERR_TIMEOUT: return "timeout";
    case FR_ERR_OOM: return "out of device memory";
    case FR_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}
