// Internal (non-ABI) declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "hfr_common.cuh"

namespace hfr {

// NVTX range around one C-ABI call (host timeline of the enqueued work; a no-op without a tool)
struct NvtxScope {
  explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
  NvtxScope(const NvtxScope&) = delete;
  NvtxScope& operator=(const NvtxScope&) = delete;
};
#define FR_NVTX(name) ::hfr::NvtxScope fr_nvtx_scope_(name)

// Stream-capture helpers of the whole-stage graphs: a conditional handle of the graph that s is
// capturing into, and a conditional node (WHILE / IF) after the work captured so far on s, whose
// body graph is returned for capture on another stream
cudaError_t graph_conditional_handle(cudaStream_t s, unsigned dflt, unsigned flags, cudaGraphConditionalHandle* h);
cudaError_t graph_add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                  cudaGraph_t* body);

// counts every kernel launch of the library (reported by fr_kernel_launches); launch_count reads
// the counter, launch_count_add corrects it for graphs (a capture counts its kernels once, a
// replay runs them as often as its loops turn)
void count_launch();
// bounds-checked build: the collectors of the translation units' device words (FR_IDX)
void checked_register(int (*collect)(unsigned long long* first, unsigned long long* count));
unsigned long long launch_count();
void launch_count_add(long long delta);

// n-point Gauss-Legendre nodes and weights (Newton on P_n), and the 1D reference operators of
// degree p (barycentric Lagrange derivatives, DG-recovering correction lift l_i(+-1)/w_i)
void gauss_legendre_nodes(int n, double* x, double* w);
void build_ref_ops(int p, RefOps& R);

// Arguments of the element residual kernels.  All pointers are device pointers; nullable
// ones are marked.  U: E x Ns x nv; uhat: ntrace x n x nv; Uf_all: E x 4n x nv;
// qf_all: E x 4n x 2 x nv; gview: E x 4n x nv.
struct ResArgs {
  int E;
  const double* U;
  const double* dU;     // nullable: tangent of U (JVP mode)
  const double* uhat;   // nullable when the mesh has no trace faces
  const double* duhat;  // nullable
  const double* geo_sol;
  const double* geo_face;
  const int* nbr;
  const int* nbr_face;
  const int* kind;
  const int* tr_of;
  const unsigned char* implicit;
  const double* Uf_all;  // neighbour face states (read), nullable for all-trace meshes
  const double* qf_all;  // neighbour face gradients (read)
  double* Uf_out;        // MODE_UF output
  double* qf_out;        // MODE_QF output
  double* R;             // nullable
  double* dR;            // nullable (JVP)
  double* gview;         // nullable: w_q J_f F^.n on trace faces
  double* dgview;        // nullable (JVP)
  int ntrace;            // trace faces (bounds of tr_of in the checked build)
};

cudaError_t launch_residual(int p, const RefOps& ref, const PhysParams& pp, const ResArgs& a, bool need_nbr,
                            bool jvp, cudaStream_t st);
cudaError_t launch_face_states(int p, const RefOps& ref, const PhysParams& pp, const ResArgs& a, cudaStream_t st);
cudaError_t launch_trace_assemble(const double* gview, const int* sides, int ntrace, int npf, double* g,
                                  cudaStream_t st);

// Element Jacobian blocks of the implicit elements (row-major, per implicit element k):
// A: nA x nA, B: nA x nT, C: nT x nA, D: nT x nT.
struct JacArgs {
  int Eim;
  const int* imp_idx;  // Eim element ids
  const double* U;
  const double* uhat;
  const double* geo_sol;
  const double* geo_face;
  const int* nbr;
  const int* nbr_face;
  const int* kind;
  const int* tr_of;
  const double* Uf_all;  // neighbour face states for interface faces
  int E, ntrace;         // elements and trace faces (bounds in the checked build)
  double a_dt;
  void* A;
  void* B;
  void* C;
  void* D;
};
cudaError_t launch_jacobian(int p, int prec_bytes, const RefOps& ref, const PhysParams& pp, const JacArgs& a,
                            cudaStream_t st);

// Condensation: per implicit element, LU with partial pivoting of A (in place into LU),
// X = A^{-1}[B | r], S = D - C X_B, t = s - C x_r.
struct CondArgs {
  int Eim, nA, nT;
  const void* A;
  const void* B;
  const void* C;
  const void* D;
  const double* r;  // Eim x nA (FP64 right-hand side -h)
  const double* s;  // Eim x nT (FP64 -g^k)
  void* LU;
  int* piv;
  void* XB;
  double* xr;       // Eim x nA
  void* S;
  double* t;        // Eim x nT
  int* status;      // device status word (DEV_ERR_*), first failing element in status[1]
  // FP32 blocks: 0 = factorisation and products on the FP32 FMA pipes, 1 = products on the tensor
  // cores (3xTF32), 2 = factorisation and products on the tensor cores
  int tc_mode = 0;
  int inv_ctas = 0;  // resident CTAs per SM of the tensor-core inverse (0: as many as fit, at most 4)
};
cudaError_t launch_condense(int prec_bytes, const CondArgs& a, cudaStream_t st);
// the same in two parts: 0 = factorisation (the whole condensation where it is one kernel),
// 1 = the products X = A^{-1}[B | r], S = D - C X_B of the two-kernel FP32 path (else nothing)
cudaError_t launch_condense_part(int prec_bytes, const CondArgs& a, cudaStream_t st, int part);

// Elements of uneven shapes (nA[k], nT[k], host arrays) condensed in one persistent launch with
// the shared-memory Gauss-Jordan kernel; blocks packed element after element (see hfr.h)
cudaError_t launch_condense_uneven(int prec_bytes, int n, const int* nA, const int* nT, const void* A, const void* B,
                                   const void* C, const void* D, const double* r, const double* s, void* LU, int* piv,
                                   void* XB, double* xr, void* S, double* t, int* status, cudaStream_t st);

// The same with the tables built once (host) and kept on the device, e.g. by a context whose
// element shapes do not change: per element 5 offsets (A, B/C, D, nA-vector, nT-vector) and the
// shape; the shared-memory elements in launch order with their bundles; the elements whose working
// set exceeds shared memory, condensed by the global-memory kernel (FP64 LU factors in LU).
struct UnevenTables {
  std::vector<long long> off;
  std::vector<int> shape, order, bundle, global;
  size_t smem = 0;
  int gmax_nA = 0, gmax_nT = 0;  // largest shape of the global-memory elements
};
struct UnevenDev {
  const long long* off = nullptr;
  const int *order = nullptr, *shape = nullptr, *bundle = nullptr, *global = nullptr;
  int nb = 0, nglobal = 0;
  size_t smem = 0;
  int colmajor = 0;  // the blocks are stored column-major (hexahedra); all go to the global kernel
  int gmax_nA = 0, gmax_nT = 0;
};
// skip (nullable): elements condensed elsewhere keep their offsets but are not scheduled
int uneven_tables(int prec_bytes, int n, const int* nA, const int* nT, UnevenTables* tb,
                  const unsigned char* skip = nullptr);
// One shape class of a packed uneven FP32 batch (list: its elements, off: the batch's per-element
// offsets as uploaded with its tables) through the fixed-shape kernels of that shape, in chunks of
// cap elements staged in scratch (class_scratch_bytes; one buffer may serve every shape: its
// leading status words, set once by class_scratch_init_status, are where every shape expects
// them).  The chunk's failures go to status with packed element ids.  contig_k0 >= 0: the class is
// the consecutive elements contig_k0.. (uniform strides from the host offsets contig_off of its
// first element: A, B/C, D, nA-vector, nT-vector), condensed in place without the scratch batch.
size_t class_scratch_bytes(int nA, int nT, int cap);
cudaError_t class_scratch_init_status(void* scratch, cudaStream_t st);
cudaError_t launch_condense_class(const int* list, int count, int nA, int nT, const long long* off, const void* A,
                                  const void* B, const void* C, const void* D, const double* r, const double* s,
                                  void* LU, int* piv, void* XB, double* xr, void* S, double* t, int* status,
                                  void* scratch, int cap, int tc_mode, cudaStream_t st, int contig_k0 = -1,
                                  const long long* contig_off = nullptr);
size_t uneven_dev_bytes(const UnevenTables& tb);
cudaError_t uneven_upload(const UnevenTables& tb, void* dbuf, UnevenDev* dv, cudaStream_t st);
cudaError_t launch_condense_uneven_dev(int prec_bytes, const UnevenDev& dv, const void* A, const void* B, const void* C,
                                       const void* D, const double* r, const double* s, void* LU, int* piv, void* XB,
                                       double* xr, void* S, double* t, int* status, cudaStream_t st);
bool uneven_fits_smem(int prec_bytes, int nA, int nT);

// x = A^{-1} b with the stored factorisation (LU + interchanges or in-place inverse, as chosen
// by condense_uses_lu), in place on b (Eim x nA, FP64 vectors).
bool condense_uses_lu(int prec_bytes, int nA, int nT);
// a condensation kernel exists for this precision and block shape (launch_condense succeeds)
bool condense_feasible(int prec_bytes, int nA, int nT);
// highest CondArgs::tc_mode available for this precision and block shape (0: none)
int condense_tc_available(int prec_bytes, int nA, int nT);
cudaError_t launch_lu_solve(int prec_bytes, int Eim, int nA, int nT, const void* LU, const int* piv, double* b,
                            cudaStream_t st);

// Trace operators
struct TraceArgs {
  int ntrace, n, nv, nT;  // nT = 4 n nv
  const int* sides;       // ntrace x 4 (e0, f0, e1, f1) with compact implicit element ids
  const int* tr_of_c;     // Eim x 4 trace id of each face of a compact implicit element (-1 none)
  const void* S;          // Eim x nT x nT
};
// x32 (nullable): FP32 copy of x read instead of x by the FP32 fixed-shape kernels
cudaError_t launch_trace_matvec(int prec_bytes, const TraceArgs& a, const double* x, double* y, cudaStream_t st,
                                const int* gate = nullptr, int gj = 0, const float* x32 = nullptr);
cudaError_t launch_precond_build(int prec_bytes, const TraceArgs& a, double* Pinv, int* status, cudaStream_t st);
// Pinv holds the inverses in the block precision (double or float storage in the same buffer)
// inv_h (nullable): x is first scaled in place by *inv_h; y32 (nullable): FP32 copy of y
cudaError_t launch_precond_apply(int prec_bytes, const TraceArgs& a, const double* Pinv, double* x, double* y,
                                 cudaStream_t st, const int* gate = nullptr, int gj = 0, const double* inv_h = nullptr,
                                 float* y32 = nullptr);
cudaError_t launch_assemble_t(const TraceArgs& a, const double* te, double* t, cudaStream_t st);
// t_k = s_k - C_k x_r for every implicit element (C in the block precision)
cudaError_t launch_rhs_condense(int prec_bytes, int Eim, int nA, int nT, const void* C, const double* xr,
                                const double* s, double* t, cudaStream_t st);
cudaError_t launch_backsolve(int prec_bytes, const TraceArgs& a, int Eim, int nA, const void* XB, const double* xr,
                             const double* duhat, double* du, cudaStream_t st);


}  // namespace hfr
