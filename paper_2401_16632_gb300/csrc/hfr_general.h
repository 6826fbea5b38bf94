// General quadrilateral meshes (internal): per-element polynomial degree, faces between unequal
// degrees, and wall / far-field boundary faces, through the whole hybridized stage.  The context
// of hfr_api.cu owns one GenCtx when its mesh needs it and forwards its entry points here.
#pragma once

#include "../../include/hfr.h"
#include "hfr_internal.h"
#include "hfr_krylov.h"

namespace hfr {
namespace gen {

struct GenCtx;

// hooks into the owning context: per-phase event timing and error reporting
struct Hooks {
  void* owner = nullptr;
  int (*prof_begin)(void* owner, int phase) = nullptr;
  void (*prof_end)(void* owner, int handle) = nullptr;
  int (*set_err)(void* owner, int code, const char* msg, int elem, int it, double val) = nullptr;
};

// true when the mesh needs the general path (per-element degrees that differ, or boundary faces)
bool mesh_is_general(const fr_mesh_desc* mesh);
int create(const fr_mesh_desc* mesh, const fr_config* cfg, cudaStream_t st, const Hooks& hooks, GenCtx** out);
void destroy(GenCtx* g);
void query(const GenCtx* g, fr_ctx_info* info);
int layout(const GenCtx* g, long long* elem_off, long long* trace_off, int* blk_nA, int* blk_nT);
int solution_points(GenCtx* g, double* xy);
int residual(GenCtx* g, const double* u, const double* uhat, double* R, double* gtrace);
int initial_trace(GenCtx* g, const double* u, double* uhat);
int local_jacobian(GenCtx* g, const double* u, const double* uhat, const double* ustar, double a_dt);
int condense(GenCtx* g, int refine);
int trace_gmres(GenCtx* g, double* duhat, double rtol, int maxit, int* iters, double* final_rel);
int backsolve(GenCtx* g, const double* duhat, double* du, int refine);
int export_array(GenCtx* g, int which, void* dst, size_t bytes, bool import);
int stage(GenCtx* g, int stage, double dt, const double* u_n, double* u_stage, double* uhat, double* R_hist,
          double newton_tol, int newton_maxit, double gmres_rtol, int gmres_maxit, int refine, fr_stage_stats* st);
// the implicit stages as one CUDA graph each (captured on the first call with a new key)
int set_graph(GenCtx* g, int on);
int nstages(const GenCtx* g);
size_t state_values(const GenCtx* g);

}  // namespace gen
}  // namespace hfr
