/*
 * hfr.h -- C ABI of the GB300 (sm_103a) hybridized implicit-explicit flux-reconstruction
 * stage library.
 *
 * The operations follow C. A. Pereira and B. C. Vermeire, "Hybridized Implicit-Explicit Flux
 * Reconstruction Methods", arXiv 2401.16632:
 *   fr_residual         Sec. 2.1 eq. (freq1) and Sec. 2.2 eqs. (hfrriemann, hfr1, hfr2);
 *                       Sec. 4 eq. (hfrimex) on implicit/explicit interface faces
 *   hfr_local_jacobian  Sec. 3.2 eqs. (elemA, elemsystem, elemsystemB)
 *   hfr_condense        Sec. 3.2, L^k = D^k - C^k A_k^{-1} B^k, t^k = s^k - C^k A_k^{-1} r^k
 *   hfr_trace_gmres     Sec. 3.2, L du^ = t with L assembled by eqs. (assembly, assembly2)
 *   hfr_backsolve       Sec. 3.2 eq. (localproblems), du_k = A_k^{-1}(r_k - B_k du^_k)
 *   imex_stage          Sec. 3.1 eqs. (9oind, 23nffsd) inside Algorithm 1 (alg:imex) with the
 *                       domain split of Sec. 4 (eq. explicitimex)
 *   imex_steps          Algorithm 1 over whole steps, the Jacobian optionally kept across steps
 *                       as in Sec. 5 (turbulent cylinder: refreshed every 100 steps)
 *   fr_modal_filter     Appendix B (modal filter of the EDAC runs)
 *
 * Conventions
 *   - Every array argument is a DEVICE pointer owned by the caller unless it is marked
 *     "host".  The library never frees caller memory.  The library owns the workspace it
 *     allocates in fr_ctx_create (freed by fr_ctx_destroy); no entry point that takes a context
 *     allocates device memory after creation.  Two context-free calls do: hfr_condense_uneven
 *     (a stream-ordered work buffer of 28 bytes per element, freed before it returns),
 *     fr_barrier_selftest (its barrier words); the allocation-free condensation
 *     hfr_condense_noalloc allocates nothing.
 *   - All work is enqueued on the CUDA stream given to fr_ctx_create.  Calls that report
 *     scalars to the host (norms, iteration counts) synchronise that stream.
 *   - Quadrilateral meshes, tensor-product Gauss-Legendre solution points, p = 1..5.
 *     E elements, Ns = (p+1)^2, nv variables (1 advection-diffusion, 4 Navier-Stokes),
 *     nA = Ns nv, n = p + 1 points per face, nT = 4 n nv.
 *   - State layout u[e][pt][v], pt = a + n b (a along xi).  Trace layout uhat[t][m][v] for the
 *     trace faces t = 0..ntrace-1, numbered in increasing global face id (mesh face_of).
 *   - Element-local block indices: unknown i = pt nv + v; trace unknown l = (f n + m) nv + v
 *     over the four local faces (f: 0 xi=-1, 1 xi=+1, 2 eta=-1, 3 eta=+1).
 *   - Implicit elements are addressed by their compact index k (increasing element id).
 *   - Return value: FR_OK (0) or an FR_ERR_* code; fr_last_error gives details.  No entry
 *     point aborts, traps or spins without bound.
 */
#ifndef HFR_H_
#define HFR_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HFR_ABI_VERSION 2

enum fr_status {
  FR_OK = 0,
  FR_ERR_INVALID_ARG = 1,
  FR_ERR_CUDA = 2,
  FR_ERR_SINGULAR = 3,      /* zero pivot in an element block or face preconditioner block */
  FR_ERR_NOT_CONVERGED = 4, /* GMRES or Newton hit its iteration limit */
  FR_ERR_DIVERGED = 5,      /* non-finite residual */
  FR_ERR_TIMEOUT = 6,
  FR_ERR_OOM = 7,
  FR_ERR_UNSUPPORTED = 8    /* configuration outside what the library implements */
};

/* FR_PHYS_EDAC: entropically damped artificial compressibility (Appendix A), u = (P, v_x, v_y),
 * parameters theta = 1 / M^2 and nu = 1 / Re; p = 2..4; the velocity must not vanish at a trace
 * point (the hybridized stabilisation of Sec. 5.4 contains |v^|). */
enum fr_physics { FR_PHYS_ADVDIFF = 0, FR_PHYS_NAVIER_STOKES = 1, FR_PHYS_EDAC = 2 };
/* Precision of the element blocks, their factorisation and condensation, and the stored S^k
 * (the Newton residual, right-hand sides and updates, the GMRES Hessenberg / Givens state and the
 * trace solution stay FP64 in every mode; every mode stops on the same FP64 Newton test).
 *   FR_PREC_FP64  everything in FP64 (LU with partial pivoting; FP64 trace operator)
 *   FR_PREC_FP32  FP32 blocks; the condensation on the tensor cores in 3xTF32 (FP32-accurate) for
 *                 the fixed shapes (see hfr_condense_set_mode), else FP32 FMA; FP32 S and Krylov basis
 *   FR_PREC_TF32  as FP32 with the single-pass TF32 condensation (FR_CONDENSE_TENSOR_TF32); only
 *                 for the tensor-core shapes (else FR_ERR_UNSUPPORTED at creation)
 *   FR_PREC_BF16  as FP32, and S^k also stored in BF16 (rounded to nearest) for the mat-vecs of the
 *                 single-launch GMRES cycle, accumulated in FP32: half the bytes of the memory-bound
 *                 trace operator; the face-block preconditioner and the multi-kernel cycle keep FP32
 *                 S; only for the single-launch shapes (else FR_ERR_UNSUPPORTED) */
enum fr_precision { FR_PREC_FP64 = 0, FR_PREC_FP32 = 1, FR_PREC_TF32 = 2, FR_PREC_BF16 = 3 };
enum fr_tableau { FR_TAB_BE = 0, FR_TAB_SDIRK2 = 1 };

typedef struct fr_ctx fr_ctx;

/* Trace space of the hybridized elements (Sec. 2.2).  FR_TRACE_HFR: a discontinuous trace per face,
 * at the face's Gauss points.  FR_TRACE_EFR (interior-embedded FR): on interior trace faces the
 * trace is continuous, with nodes at the Gauss-Lobatto points of the faces (vertex nodes shared by
 * every trace face meeting there); each side evaluates its state, gradient, one-sided flux and J_f
 * at those points, and the values of J_f F^.n and of u^ - u_f are interpolated to the element's
 * Gauss-aligned face points for the lift; the transmission condition of a node sums w^GLL J_f F^.n
 * over every face and side that carries it; boundary faces keep discontinuous traces at their
 * Gauss points.  EFR runs on the general path (quadrilaterals, one degree); its trace vector holds
 * one node per unit (fr_ctx_layout: ntrace = nodes) in the numbering of efr_trace_nodes, and its
 * GMRES preconditioner is node-block Jacobi (nv x nv blocks: the nodes' blocks overlap faces). */
enum fr_trace_kind { FR_TRACE_HFR = 0, FR_TRACE_EFR = 1 };

/* Boundary tags of fr_mesh_desc.bc (where nbr < 0). */
enum fr_boundary { FR_BC_WALL = 1, FR_BC_FARFIELD = 2 };
/* Element types of fr_mesh_desc.elem_type.  FR_ELEM_HEX (the paper's 3D runs, Sec. 5.3; Navier-Stokes
 * only, one degree p = 1..3, general path): verts nelem x 8 x 3 with corner k = a + 2b + 4c at
 * (2a-1, 2b-1, 2c-1); nbr, nbr_face, face_of, bc nelem x 6 with faces 0/1 xi = -1/+1, 2/3 eta,
 * 4/5 zeta; solution point pt = a + n b + n^2 c; face point m = i + n j along the lower then the
 * higher tangential axis, met in the same order from both sides of a face (conforming meshes of
 * one orientation); u = (rho, rho v_x, rho v_y, rho v_z, E), nv = 5.  Its element blocks are
 * stored column-major (hfr_export / hfr_import: A^T, B^T, C^T, D^T row-major). */
enum fr_elem_type { FR_ELEM_QUAD = 0, FR_ELEM_HEX = 1 };

/* Mesh description (all HOST arrays, copied by fr_ctx_create).
 * A mesh whose elements all share one degree and that has no boundary face runs the uniform
 * path (fixed-shape kernels: tensor-core condensation, single-launch GMRES, stage graph).  A mesh
 * with per-element degrees (p_elem not all equal) or with boundary faces runs the general path
 * (packed layouts, see fr_ctx_layout): faces between unequal degrees carry the Gauss points of
 * the higher one (the element blocks admit faces with different numbers of trace points, Sec. 3.2
 * eq. elemsystemB), boundary faces carry the boundary rows of the transmission conditions
 * (Sec. 2.2 eq. hfr2): a hybridized far field (trace = average of the element state and u_inf) and
 * a no-slip adiabatic wall (Navier-Stokes; momentum rows set the trace velocity to zero, mass and
 * energy rows are the element's own normal fluxes).  Explicit elements may meet the far field
 * (Rusanov against u_inf), not a wall. */
typedef struct {
  int nelem;
  int p;                         /* polynomial degree 1..5 (all elements, unless p_elem is given) */
  const double* verts;           /* nelem x 4 x 2 corner coordinates, corner k = a + 2b at (2a-1, 2b-1) (hex: see fr_elem_type) */
  const int* nbr;                /* nelem x 4 (hex: 6) neighbour element across each local face, -1 on a boundary */
  const int* nbr_face;           /* nelem x 4 (6) neighbour's local face */
  const int* face_of;            /* nelem x 4 (6) global face id (first-appearance numbering), < 4 (6) nelem */
  const unsigned char* implicit; /* nelem: 1 = hybridized implicit, 0 = explicit FR */
  const int* p_elem;             /* nullable: nelem degrees 1..5 (general path: advection-diffusion, Navier-Stokes) */
  const int* bc;                 /* nullable: nelem x 4 fr_boundary tags where nbr < 0 (required when there are) */
  int elem_type;                 /* fr_elem_type */
} fr_mesh_desc;

typedef struct {
  int physics;     /* fr_physics */
  double beta[2];  /* advection velocity */
  double nu;       /* diffusivity (advection-diffusion), 1 / Re (EDAC) */
  double gamma;    /* ratio of specific heats */
  double mu;       /* dynamic viscosity */
  double Pr;       /* Prandtl number */
  double lref;     /* length in the viscous part of the hybridized stabilisation s */
  int precision;   /* fr_precision */
  int tableau;     /* fr_tableau: implicit DIRK + explicit partner of the IMEX pair */
  int gmres_restart; /* m <= 64 */
  double theta;    /* EDAC: 1 / M^2 of the artificial Mach number */
  double u_inf[5]; /* free-stream state of far-field faces (conserved variables) */
  int trace_kind;  /* fr_trace_kind */
} fr_config;

/* Sizes of a context.  Uniform path: as named.  General path: p, n, ns the largest degree and its
 * point counts, nA / nT the largest element blocks; the state, R and R_hist hold state_values
 * values per copy, uhat and g trace_values (layouts from fr_ctx_layout). */
typedef struct {
  int nelem, nimplicit, p, n, ns, nv, nA, nT, ntrace, nstages;
  int has_explicit;       /* mesh has FR faces / interface faces */
  size_t workspace_bytes; /* device memory held by the context */
  int general;            /* 1: general path (packed layouts) */
  size_t state_values;    /* values of one state copy (nelem ns nv on the uniform path) */
  size_t trace_values;    /* values of one trace vector (ntrace n nv on the uniform path) */
  int face_points;        /* general path: entries of the face-point trace map (hfr_export 64) */
} fr_ctx_info;

typedef struct {
  int newton_iterations;
  int gmres_iterations;   /* summed over Newton iterations */
  double residual0;       /* ||[h; g]||_2 at the initial guess */
  double residual;        /* final ||[h; g]||_2 */
  int converged;
} fr_stage_stats;

typedef struct {
  int code;
  int element;      /* failing implicit element (compact index) or -1 */
  int iteration;    /* failing Newton / GMRES iteration or -1 */
  double value;     /* residual or pivot magnitude where relevant */
  char message[160];
} fr_error_info;

/* Create a context: builds reference operators, metrics, face classification, trace numbering,
 * and allocates all device workspace.  stream: a cudaStream_t (0 = legacy default stream).
 * Errors: FR_ERR_INVALID_ARG (bad sizes / inconsistent connectivity), FR_ERR_UNSUPPORTED
 * (boundary faces, p outside 1..5, combinations not compiled), FR_ERR_OOM, FR_ERR_CUDA. */
int fr_ctx_create(const fr_mesh_desc* mesh, const fr_config* cfg, void* stream, fr_ctx** out);
void fr_ctx_destroy(fr_ctx* ctx);
int fr_ctx_query(const fr_ctx* ctx, fr_ctx_info* info /* host */);
/* Physical coordinates (nelem x Ns x 2, device; general path: element after element, Ns_e
 * points each) of the solution points. */
int fr_solution_points(fr_ctx* ctx, double* xy);

/* Packed layouts of a context (host arrays; NULL skips one).  elem_off (nelem + 1): element e's
 * state values start at elem_off[e] (uniform path: e ns nv); trace_off (ntrace + 1): trace t's
 * values (points x nv, the points of face t in order) start at trace_off[t]; blk_nA, blk_nT
 * (nimplicit): the block sizes of each implicit element.  General path, per implicit element k
 * (increasing element id): the local trace unknowns are the four faces' points in local face
 * order (point count m_f = max(p_e, p_neighbour) + 1, p_e + 1 on boundaries; rows and columns of
 * faces without a trace are zero), l = (sum_{f' < f} m_f') nv + q nv + v; hfr_export packs the
 * element arrays one after another in k (A: nA_k^2, B, C, X_B: nA_k nT_k, D, S: nT_k^2, r, x_r:
 * nA_k, s, t_k: nT_k) and the face-block inverses per trace ((m_t nv)^2).  FR_OK. */
int fr_ctx_layout(const fr_ctx* ctx, long long* elem_off, long long* trace_off, int* blk_nA, int* blk_nT);

/* Spatial residual du/dt = R(u, u^) at every element (R: nelem x nA) and, if g != NULL, the
 * trace residual g (ntrace x n x nv) = sum over the two sides of w_q J_f F^.n (eq. hfr2).
 * uhat may be NULL only when the mesh has no trace faces. */
int fr_residual(fr_ctx* ctx, const double* u, const double* uhat, double* R, double* g);

/* Element blocks A_k, B_k, C_k, D_k of the stage residual h = u - u* - a_dt R(u, u^) at (u, u^)
 * for every implicit element, kept in the context (FP64 or FP32 per cfg.precision), together
 * with the Newton right-hand sides r_k = -h_k and s_k = -g^k (FP64).  ustar: nelem x nA
 * (NULL means u* = u). */
int hfr_local_jacobian(fr_ctx* ctx, const double* u, const double* uhat, const double* ustar, double a_dt);

/* Per implicit element: LU with partial pivoting of A_k, X = A_k^{-1}[B_k | r_k],
 * S_k = D_k - C_k X_B, t_k = s_k - C_k x_r; assembles the global t and the face-block Jacobi
 * preconditioner.  refine: number of FP64 refinement sweeps of x_r against the exact FP64
 * linearisation (0 = none).  Errors: FR_ERR_SINGULAR (element in fr_last_error). */
int hfr_condense(fr_ctx* ctx, int refine);

/* Restarted right-preconditioned GMRES(m) on L du^ = t (L applied matrix-free from the S_k).
 * duhat: ntrace x n x nv output.  Stops when the estimated ||t - L du^|| <= rtol ||t|| or after
 * maxit inner iterations (then FR_ERR_NOT_CONVERGED, duhat holds the last iterate).
 * iters / final_rel (host, nullable): iterations and true final relative residual. */
int hfr_trace_gmres(fr_ctx* ctx, double* duhat, double rtol, int maxit, int* iters, double* final_rel);

/* When imex_stage re-linearises.  FR_JAC_EVERY_NEWTON (default): element blocks, condensation and
 * preconditioner at every Newton iterate (exact Newton on the blocks).  FR_JAC_ONCE_PER_STAGE:
 * at the stage's first iterate only; later iterations are chord iterations that reuse the blocks,
 * their factorisation, S_k, X_B and the preconditioner, and recompute only x_r = A^{-1} r,
 * t_k = s - C x_r and t.  FR_JAC_KEEP: the condensation is held across stages and steps (the
 * paper keeps its Jacobian for 100 steps; Sec. 5, turbulent cylinder) and every Newton iteration
 * is a chord iteration, except that the first iterate of a stage re-linearises when no
 * condensation is held, when a_ii dt differs from the held one, or after imex_refresh_jacobian;
 * hfr_local_jacobian, hfr_condense and hfr_autotune drop the held one.  All policies stop on the
 * same FP64 Newton residual test.  FR_ERR_INVALID_ARG for another value. */
enum fr_jacobian_policy { FR_JAC_EVERY_NEWTON = 0, FR_JAC_ONCE_PER_STAGE = 1, FR_JAC_KEEP = 2 };
int imex_set_jacobian_policy(fr_ctx* ctx, int policy);
/* FR_JAC_KEEP: re-linearise at the next stage's first Newton iterate.  FR_OK. */
int imex_refresh_jacobian(fr_ctx* ctx);

/* How hfr_trace_gmres (and imex_stage) run a restart cycle.  FR_GMRES_FUSED (the default where
 * available): the whole cycle -- preconditioner, mat-vecs, Gram-Schmidt, Givens rotations and the
 * solution update -- is one cooperative launch with one CTA per SM that meets at grid barriers;
 * available for trace blocks (nT, n nv) = (64,16), (80,20), (48,12) on devices with cooperative
 * launch.  Each barrier wait is bounded (about 2 s); a wait that runs out ends the launch and
 * hfr_trace_gmres returns FR_ERR_TIMEOUT.  FR_GMRES_MULTI: one short kernel per step with the
 * Krylov state on the device (any shape).  Both compute the same iteration (classical
 * Gram-Schmidt with a conditional second pass); their results agree to rounding.
 * set: FR_ERR_UNSUPPORTED if FR_GMRES_FUSED is not available for the context.
 * get: the mode in effect, -1 for a null context.  This switch has no counterpart in the paper. */
enum fr_gmres_mode { FR_GMRES_MULTI = 0, FR_GMRES_FUSED = 1 };
int hfr_gmres_set_mode(fr_ctx* ctx, int mode);
int hfr_gmres_get_mode(const fr_ctx* ctx);

/* Which pipes run the FP32 condensation (Sec. 3.2; this switch has no counterpart in the paper).
 * FR_CONDENSE_TENSOR (the default where available: FP32 blocks of shape (nA, nT) = (100, 80),
 * (64, 64), (36, 48)): the Gauss-Jordan factorisation as 16-column panels whose trailing updates
 * are rank-16 products, and the products X = (PA)^{-1}[P B | P r], S = D - C X_B, t = s - C x_r,
 * all on the tensor cores (tcgen05; TF32 operands split into high and low parts, three products
 * accumulated in FP32: about 2^-21 relative per product term).  FR_CONDENSE_TENSOR_PRODUCTS: the
 * products on the tensor cores, the factorisation on the FP32 FMA pipes.  FR_CONDENSE_FMA: both
 * on the FP32 FMA pipes.  FR_CONDENSE_TENSOR_TF32: the FR_CONDENSE_TENSOR kernels with the single
 * TF32 product hi*hi (about 2^-11 relative per product term; the FP64 Newton residual still decides
 * convergence, which may take more iterations; hfr_autotune never chooses it).  set:
 * FR_ERR_UNSUPPORTED where the requested form does not exist for the context; get: the mode in
 * effect, -1 for a null context. */
enum fr_condense_mode {
  FR_CONDENSE_FMA = 0,
  FR_CONDENSE_TENSOR_PRODUCTS = 1,
  FR_CONDENSE_TENSOR = 2,
  FR_CONDENSE_TENSOR_TF32 = 3
};
int hfr_condense_set_mode(fr_ctx* ctx, int mode);
int hfr_condense_get_mode(const fr_ctx* ctx);

/* Self-test of the bounded grid barrier that the single-launch GMRES cycle meets at (no
 * counterpart in the paper; failure detection of that cycle).  One cooperative launch of nblocks
 * CTAs on `stream` passes `rounds` grid barriers; if 0 <= absent_block < nblocks that CTA leaves
 * without arriving, so the others' wait runs out after timeout_s seconds (0 < timeout_s <= 10),
 * they raise the abort flag and return.  *barriers_passed (host) = the barriers passed, summed
 * over CTAs.  Returns FR_OK (no wait ran out), FR_ERR_TIMEOUT (the abort flag was raised; the
 * CUDA context stays usable), FR_ERR_INVALID_ARG (arguments, or more CTAs than can be resident
 * at once) or FR_ERR_CUDA. */
int fr_barrier_selftest(int nblocks, int absent_block, int rounds, double timeout_s, int* barriers_passed,
                        void* stream);

/* du_k = x_r - X_B du^_k = A_k^{-1}(r_k - B_k du^_k) for every implicit element (du: nimplicit x nA,
 * compact order), followed by `refine` FP64 refinement sweeps against the exact FP64 linearisation. */
int hfr_backsolve(fr_ctx* ctx, const double* duhat, double* du, int refine);

/* Copy a context block array to a caller device buffer (for inspection / parity tests).
 * which: 0 A, 1 B, 2 C, 3 D, 4 S, 5 X_B, 6 x_r (FP64), 7 t_k (FP64), 8 r (FP64), 9 s (FP64),
 * 10 global t (FP64), 11 face-block-Jacobi inverses (ntrace x bs x bs, bs = n nv); general-mesh
 * contexts also 64: the trace point of every element face point (int32, nface x nelem x face-point
 * stride, -1 off traces).  Block arrays are in the context precision; dst must hold `bytes`. */
int hfr_export(fr_ctx* ctx, int which, void* dst, size_t bytes);
/* The reverse of hfr_export for the arrays 0..9 (A, B, C, D, S, X_B, x_r, t_k, r, s): overwrite the
 * context array with `bytes` (exactly its size) from the caller device buffer src, e.g. to condense
 * blocks formed elsewhere or to plant a defective block in a test.  A condensation held for
 * FR_JAC_KEEP is dropped.  In a bounds-checked build (FR_CHECKED) a general-mesh context also takes
 * array 64 (the face-point trace map), to plant a corrupted index that the device checks must catch.
 * FR_ERR_INVALID_ARG for another array or size. */
int hfr_import(fr_ctx* ctx, int which, const void* src, size_t bytes);

/* One stage of the IMEX step (Algorithm 1):
 *   stage 0      : R_hist[0] = R(u_n, u^)                             (start of a step)
 *   1 <= i <= s  : explicit elements u_i = u_n + dt sum_{j<=i} ahat_{i+1,j} R_hist[j-1];
 *                  implicit elements solve u_i - u* - a_ii dt R(u_i, u^_i) = 0, g = 0 by Newton
 *                  from u* = u_n + dt sum_{j<i} a_ij R_hist[j], updating uhat in place;
 *                  then R_hist[i] = R(u_i, u^_i)
 *   i = s + 1    : u_stage = u_{n+1} = u_n + dt sum_j b_j R_hist[j] (implicit elements)
 *                                      + dt sum_j bhat_j R_hist[j-1] (explicit elements)
 * u_n, u_stage: nelem x nA; R_hist: (s + 1) x nelem x nA.  Newton stops when
 * ||[h; g]||_2 <= newton_tol ||[h; g]^0||_2 (FR_ERR_NOT_CONVERGED after newton_maxit).
 * gmres_rtol / gmres_maxit: inner linear solve; refine: FP64 refinement sweeps of the local solves. */
int imex_stage(fr_ctx* ctx, int stage, double dt, const double* u_n, double* u_stage, double* uhat,
               double* R_hist, double newton_tol, int newton_maxit, double gmres_rtol, int gmres_maxit,
               int refine, fr_stage_stats* stats /* host, nullable */);

/* Totals of imex_steps. */
typedef struct fr_steps_stats {
  int steps;               /* steps completed */
  int newton_iterations;   /* over all implicit stages */
  int gmres_iterations;
  int jacobian_refreshes;  /* linearisations (element blocks + condensation) made */
  double max_rel_residual; /* largest final ||[h; g]|| / ||[h; g]^0|| of the implicit stages */
  int converged;           /* 1 when every stage met newton_tol */
} fr_steps_stats;

/* nsteps whole IMEX steps of size dt (Algorithm 1, all stages and the final combination), in
 * place: u (nelem x nA) holds u_n on entry and u_{n+nsteps} on return, uhat the traces.  R_hist
 * ((s + 1) x nelem x nA) and u_stage (nelem x nA) are caller-owned device scratch.  With
 * FR_JAC_KEEP the held condensation is refreshed at steps 0, refresh_every, 2 refresh_every, ...
 * (refresh_every <= 0: only when needed, see imex_set_jacobian_policy); other policies ignore it.
 * Stops at the first failing stage with its status (stats then count the completed steps).
 * Newton and GMRES arguments as for imex_stage.  Synchronises the stream. */
int imex_steps(fr_ctx* ctx, int nsteps, double dt, double* u, double* uhat, double* R_hist, double* u_stage,
               int refresh_every, double newton_tol, int newton_maxit, double gmres_rtol, int gmres_maxit,
               int refine, fr_steps_stats* stats /* host, nullable */);

/* Condensation of elements of uneven block shapes (e.g. several polynomial degrees) in one
 * persistent launch (Sec. 3.2; batching has no counterpart in the paper).  Element k has blocks of
 * nA[k] x nA[k] (A), nA[k] x nT[k] (B), nT[k] x nA[k] (C), nT[k] x nT[k] (D), each row-major,
 * packed element after element in each array (element k's A starts after sum_{j<k} nA[j]^2
 * values, its B and C after sum nA[j] nT[j], its D after sum nT[j]^2, its r after sum nA[j], its
 * s after sum nT[j]); outputs packed the same way: LU (((PA)^{-1})^T, A-sized), piv (nA-sized),
 * XB (B-sized), xr (nA-sized), S (D-sized), t (nT-sized).  nA, nT: HOST arrays; every other
 * array a caller-owned DEVICE buffer in the block precision (r, s, xr, t FP64); status: 2 device
 * ints of scratch.  The CTAs walk the elements from the most to the least expensive (shared-memory
 * Gauss-Jordan with partial pivoting, S = D - C X_B, t = s - C x_r).  A stream-ordered work
 * buffer of 28 bytes per element is allocated and freed inside; the call synchronises the stream.
 * Shapes whose working set exceeds the 227 KB of shared memory (FP32 beyond (144, 96), FP64
 * beyond about (100, 80)) are condensed by a global-memory kernel in the same call (LU with
 * partial pivoting of A in place, one CTA per element; LU then holds the LU factors and piv the
 * row interchanges instead of the inverse).  Returns FR_OK, FR_ERR_SINGULAR (*failed_element: an
 * element with a zero pivot), FR_ERR_INVALID_ARG (null array, bad precision, nA or nT < 1, nT >
 * 16384) or FR_ERR_CUDA. */
int hfr_condense_uneven(int nelem, const int* nA, const int* nT, int precision, const void* A, const void* B,
                        const void* C, const void* D, const double* r, const double* s, void* LU, int* piv, void* XB,
                        double* xr, void* S, double* t, int* status, void* stream, int* failed_element);

/* Modal filter of Appendix B, in place on u (device, nelem x ns x nv): on every element of the
 * selection (which: 0 all, 1 implicit, 2 explicit) and every variable, u <- F u with
 * F = V Lambda* V^{-1}, V the tensor-product orthonormal Legendre basis at the solution points,
 * Lambda = diag(sigma(i + j)) for the mode of degrees (i, j): sigma = 1 below eta_c,
 * exp(-alpha ((eta - eta_c) / (2p - eta_c))^s) from eta_c to 2p.  Lambda* = Lambda^dt_ratio with
 * dt_ratio = dt / dt_ref (a reading of the paper's time-step normalisation; 1 for Lambda* = Lambda).
 * Keeps each element's mean.  FR_ERR_INVALID_ARG for alpha < 0, s <= 0, eta_c < 0, dt_ratio <= 0. */
int fr_modal_filter(fr_ctx* ctx, double* u, double alpha, double s, int eta_c, double dt_ratio, int which);

/* Autotuner (no counterpart in the paper): forms the element blocks at (u, uhat, ustar, a_dt) as
 * hfr_local_jacobian does, then times on them, with CUDA events on the context stream (best of
 * two after a warm-up), every condensation form available for the context's precision and block
 * shape -- FMA, tensor-core products, tensor-core factorisation and products with 1 to 4 resident
 * CTAs per SM for the factorisation -- and both GMRES cycle forms on the condensed system
 * (rtol 1e-4, at most 500 iterations), and keeps the fastest of each in the context.  out (host,
 * nullable): the times (ms, -1 where not available) and the choices. */
typedef struct {
  int condense_mode;        /* fr_condense_mode chosen */
  int inverse_ctas_per_sm;  /* 0 = default residency */
  int gmres_mode;           /* fr_gmres_mode chosen */
  double condense_ms[3];    /* per fr_condense_mode (best residency for the tensor-core form) */
  double inverse_ms[4];     /* tensor-core form, 1..4 CTAs per SM */
  double gmres_ms[2];       /* per fr_gmres_mode */
} fr_tune_report;
int hfr_autotune(fr_ctx* ctx, const double* u, const double* uhat, const double* ustar, double a_dt,
                 fr_tune_report* out);

/* Run each implicit stage of imex_stage as one CUDA graph (on = 1; no counterpart in the paper).
 * The graph holds the whole stage: the Newton loop as a conditional WHILE node, its linear solve
 * (blocks, condensation, GMRES restart cycles as a nested WHILE node, back-substitution, update)
 * as a conditional IF node, with the convergence tests of Algorithm 1 and of GMRES taken by small
 * device kernels, so that the host launches the stage once and reads its counters once.  The
 * first call with a given (stage, dt, buffers, tolerances, limits, refine) captures and
 * instantiates the graph; later calls with the same arguments replay it.  Results equal the
 * stream path's.  Uniform meshes: requires implicit elements, FR_JAC_EVERY_NEWTON and (with a
 * trace) FR_GMRES_FUSED.  General meshes (mixed degree, boundary faces, hexahedra, EFR): requires
 * implicit elements; the GMRES restart cycle is the multi-kernel one, its m iterations enqueued
 * in the graph and skipped on the device once the cycle has ended, its restart decision taken on
 * the device, and the iteration limit checked per cycle.  FR_ERR_UNSUPPORTED otherwise.
 * Per-phase profiling (fr_profile_*) sees no phases of a graph stage. */
int imex_stage_set_graph(fr_ctx* ctx, int on);
int imex_stage_get_graph(const fr_ctx* ctx);

/* Initial trace guess: average of both sides' interpolated states (uhat: ntrace x n x nv). */
int hfr_initial_trace(fr_ctx* ctx, const double* u, double* uhat);

/* Per-phase device time of the context's calls, measured with CUDA events on its stream.
 * Phases: 0 residual (incl. trace assembly), 1 element Jacobian blocks, 2 condensation: the
 * factorisation kernel (the whole condensation where it is a single kernel), 3 trace right-hand
 * side + preconditioner build, 4 trace GMRES solve, 5 back-substitution and refinement, 6 Newton
 * bookkeeping (right-hand sides, norms, updates), 7 FP64 refinement of x_r, 8 one trace mat-vec
 * kernel (multi-kernel GMRES: the restart / final-residual products), 9 condensation: the
 * products X = A^{-1}[B | r], S = D - C X_B of the two-kernel FP32 path. */
typedef struct {
  double ms[10];
  long long count[10];
} fr_profile;
/* on != 0 enables event timing (and resets the totals); off stops it. */
int fr_profile_enable(fr_ctx* ctx, int on);
int fr_profile_read(const fr_ctx* ctx, fr_profile* out /* host */);
/* Number of kernels this library has launched in this process (all contexts). */
unsigned long long fr_kernel_launches(void);

/* Bounds-checked build (library compiled with FR_CHECKED; no counterpart in the paper: the
 * substitute for a memory checker on devices where none may run).  Every mesh-derived gather /
 * scatter index of the residual, the element blocks, the trace assembly, the element-view
 * mat-vec and the back-substitution is checked on the device: an index outside its array is
 * counted, the first one recorded, and the access redirected to entry 0 (no trap, the kernel goes
 * on; results are then meaningless).  Reads and clears the record of every kernel so far: first =
 * (site << 48) | index of the first failure (0: none), count = failures.  FR_ERR_UNSUPPORTED in a
 * build without the checks. */
int fr_checked_status(unsigned long long* first, unsigned long long* count);

/* Allocation-free condensation, for callers that cannot let a library allocate device memory
 * (a host code with its own pooled device-memory budget, a plugin handed pre-allocated buffers).
 * The paper has no counterpart; the operation is that of hfr_condense on caller-provided blocks:
 * X = A^{-1}[B | r], S = D - C X_B, t = s - C x_r for nimplicit elements, blocks row-major in the
 * given precision (A: nA x nA, B: nA x nT, C: nT x nA, D, S: nT x nT, XB: nA x nT; r, xr: nA and
 * s, t: nT per element in FP64).  All pointers are device pointers; stream is a cudaStream_t.
 * The factors and pivots are kept in one file-scope device array of HFR_NOALLOC_SCRATCH_BYTES
 * (held by every GPU that loads the library until the process exits).  Limit:
 *   256 + round_up_256(nimplicit nA 4) + nimplicit nA^2 (8 for FP64, 4 for FP32) <= 16 MiB,
 * larger requests, nA outside 1..160 and nT outside 1..16384 return FR_ERR_INVALID_ARG before any
 * work is enqueued.  The first call on a device looks up the
 * array's device address; make that first call before any stream capture.  Every call uses the
 * same array, so calls that overlap on the GPU (other streams, other threads) race.  No
 * cudaMalloc / cudaFree is made.  Synchronises the stream; FR_ERR_SINGULAR on a zero pivot. */
#define HFR_NOALLOC_SCRATCH_BYTES (16u << 20)
int hfr_condense_noalloc(int nimplicit, int nA, int nT, int precision, const void* A, const void* B, const void* C,
                         const void* D, const double* r, const double* s, void* XB, double* xr, void* S, double* t,
                         void* stream);

/* Peak rate of one arithmetic pipe of the current device, measured now with CUDA events on
 * `stream` (no counterpart in the paper; the denominators of roofline fractions).  which:
 * 0 FP64 FMA, 1 FP32 FMA (8 independent FMA chains per thread, 8 CTAs of 256 threads per SM),
 * 2 TF32 tensor core (tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, issued back to back by one
 * thread per CTA, two CTAs per SM).  *tflops (host): dense TFLOP/s, 2 flops per multiply-add.  A
 * warm-up launch precedes the timed one; about 0.1-0.5 s in all.  Allocates nothing.  Returns
 * FR_OK, FR_ERR_INVALID_ARG, FR_ERR_TIMEOUT (the bounded wait for the MMAs ran out) or
 * FR_ERR_CUDA.  Synchronises the stream. */
int fr_measure_peak(int which, void* stream, double* tflops);

int fr_last_error(const fr_ctx* ctx, fr_error_info* info /* host */);
const char* fr_status_string(int code);

/* Trace-node layout of the interior-embedded variant EFR (Sec. 2.2: the trace is continuous on
 * the implicit skeleton, with nodes at the p + 1 Gauss-Lobatto points of every trace face; a
 * face's end points are the mesh vertices it shares with the other trace faces meeting there;
 * boundary faces keep discontinuous traces).  Host only: needs no device and no context.
 *   nbr, nbr_face, face_of  host, (nelem, 4) each: neighbour element (-1 on a boundary), its local
 *                           face, global face id (the mesh arrays of fr_mesh_desc); all elements
 *                           share one orientation, so the first point of a face meets the
 *                           neighbour's first
 *   bc                      host, (nelem, 4), nullable: FR_BC_WALL / FR_BC_FARFIELD where nbr < 0
 *                           (required when the mesh has boundary faces)
 *   implicit                host, (nelem,): nonzero for implicit elements; a trace face has both
 *                           sides implicit
 *   node_of                 host, (nelem, 4, p + 1) out: the node at each point of each element
 *                           face, -1 on faces without a trace.  Vertex nodes first, in increasing
 *                           smallest element corner 4 e + c of the vertex (corner c = a + 2 b), then
 *                           the interior Gauss-Lobatto points m = 1..p-1 of trace face t (trace faces
 *                           in increasing global face id) at nvert + t (p - 1) + m - 1, then the
 *                           p + 1 Gauss points of each boundary face of an implicit element (in
 *                           increasing global face id) at nvert + ntrace (p - 1) + b (p + 1) + m
 *   nvert_out, nnode_out    host out: vertex nodes and all nodes
 * Errors: FR_ERR_INVALID_ARG (null pointer, nelem <= 0, p outside 1..5, indices out of range, a
 * neighbour relation that is not symmetric, a boundary tag that is neither wall nor far field),
 * FR_ERR_UNSUPPORTED (boundary faces without bc). */
int efr_trace_nodes(int nelem, const int* nbr, const int* nbr_face, const int* face_of, const int* bc,
                    const unsigned char* implicit, int p, int* node_of, int* nvert_out, int* nnode_out);

/* Trace layout of a quad mesh whose elements carry different degrees p_e (Sec. 3.2: the element
 * blocks admit faces with different numbers of trace points), with wall and far-field faces.
 * A face between degrees p- and p+ carries the max(p-, p+) + 1 Gauss points of the higher degree;
 * a boundary face the p_e + 1 of its element.  A face has a trace when both sides are implicit,
 * or when it is a boundary face of an implicit element.  Host only.
 *   nbr, nbr_face, face_of, bc  host, (nelem, 4): connectivity as in fr_mesh_desc; bc = 1 (wall)
 *                               or 2 (far field) where nbr < 0
 *   implicit, p                 host, (nelem,): implicit flags, degrees 1..5
 *   face_pts                    host, (nelem, 4) out: points of each element face
 *   trace_of                    host, (nelem, 4) out: trace index of each element face, or -1;
 *                               traces numbered in increasing global face id
 *   trace_off                   host, (4 nelem + 1) capacity, out: trace t's points start at
 *                               trace_off[t] (trace_off[ntrace] = all trace points)
 *   ntrace_out                  host out
 * Errors: FR_ERR_INVALID_ARG (null pointer, nelem <= 0, a degree outside 1..5, indices out of
 * range, asymmetric connectivity, a boundary face that is neither wall nor far field). */
int mixed_trace_layout(int nelem, const int* nbr, const int* nbr_face, const int* face_of, const int* bc,
                       const unsigned char* implicit, const int* p, int* face_pts, int* trace_of, int* trace_off,
                       int* ntrace_out);

#ifdef __cplusplus
}
#endif
#endif /* HFR_H_ */
