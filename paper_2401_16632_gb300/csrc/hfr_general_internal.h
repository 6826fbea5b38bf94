// Internal definitions shared by the general-mesh translation units (quadrilaterals in
// hfr_general.cu, hexahedra in hfr_hex.cu): reference data, kernel arguments and the context.
#pragma once

#include <vector>

#include "hfr_general.h"

namespace hfr {
namespace gen {

constexpr int GN = HFR_MAXN;  // points per line / face (p <= 5)
constexpr int GNS = GN * GN;
constexpr int GF = 4 * GN;
constexpr int GEPB = 4;       // elements (warps) per CTA of the residual passes
constexpr int JT = 256;       // threads of the block kernel
constexpr int JW = JT / 32;
constexpr int HEX_PMAX = 3;                          // hexahedra: p <= 3
constexpr int HEX_FS = (HEX_PMAX + 1) * (HEX_PMAX + 1);  // face-point stride of a hexahedron face
enum { FK_WALL = 3, FK_FAR = 4 };
enum { BC_WALL = 1, BC_FAR = 2 };

// Reference operators of every degree, and the face interpolation / projection of every pair
// (n nodes, m >= n face points).  Built on the host, read from global memory.
struct GenRef {
  double M[GN + 1][GN][GN];
  double lm[GN + 1][GN], lp[GN + 1][GN], dgL[GN + 1][GN], dgR[GN + 1][GN], w[GN + 1][GN];
  double T[GN + 1][GN + 1][GN][GN];  // [n][m][q][b] = l_b(s_q): node b of n -> face point q of m
  double P[GN + 1][GN + 1][GN][GN];  // [n][m][b][q] = w_q l_b(s_q) / w_b: face points -> nodes
  // EFR faces: the n Gauss-Lobatto points of a face (interpolation both ways, GLL weights)
  double TL[GN + 1][GN][GN];  // [n][q][b] = l_b(x^GLL_q): Gauss node b -> GLL point q
  double PL[GN + 1][GN][GN];  // [n][b][q] = l^GLL_q(x_b): GLL point q -> Gauss node b
  double wl[GN + 1][GN];      // GLL weights
};

struct GArgs {
  int E;
  const int* deg;         // E: points per line n_e
  const long long* uoff;  // E: state offset
  const long long* goff;  // E: first solution point of the element in geo_sol
  const double* geo_sol;  // [point][5] = {1/J, S00, S01, S10, S11}
  const double* geo_face; // [(4 e + f) GN + q][3] = {J_f, n0, n1}
  const int *nbr, *nbr_face, *kind, *tr_of, *nfp;  // 4 E
  const long long* toff;  // trace value offsets
  const int* fnode;       // (e nface + f) fs + q: trace point of each element face point, -1 off traces
  const unsigned char* fset;  // e nface + f: 1 where the face points are Gauss-Lobatto (EFR faces)
  const unsigned char* implicit;
  const GenRef* ref;
  const double* U;
  const double* uhat;
  const double* Uf_all;   // face-point states of every element (FR / IMEX neighbours)
  const double* qf_all;   // face-point gradients
  double* Uf_out;
  double* qf_out;
  double* R;
  double* gview;          // element trace rows w_q J_f (row)_q at face points, zero off traces
  double uinf[5];
  int nface, fs;          // faces per element, face-point stride per face
  long long npts;         // trace points (bound of fnode in the checked build)
  const int* elist;       // nullable: the elements of this pass (nlist of them) instead of 0..E-1
  int nlist;
};


struct JArgs {
  int Eim;
  const int* imp_idx;
  const long long* offA;
  const long long* offB;
  const long long* offD;
  const int* lto;  // nface Eim: local offset of each face's trace unknowns
  double a_dt;
  void *A, *B, *C, *D;
  void* scratch = nullptr;  // hexahedra: per-CTA slabs of pointwise Jacobians
};

struct GenCtx {
  Hooks hk;
  cudaStream_t st = 0;
  int E = 0, Eim = 0, nv = 0, ntrace = 0, pb = 8, tableau = 0, restart = 30, pmax = 0;
  int maxA = 0, maxT = 0;
  bool need_nbr = false, has_explicit = false;
  PhysParams pp;
  double uinf[5] = {0, 0, 0, 0, 0};
  int dim = 2, nface = 4, fs = GN;  // dimension, faces per element, face-point stride per face
  int efr = 0;                      // trace continuous at GLL points on interior trace faces
  size_t npts = 0;                  // trace points (units: HFR trace faces, EFR nodes)
  size_t nstate = 0, nh = 0, sumA = 0, sumT = 0, sumAA = 0, sumAT = 0, sumTT = 0, sumP = 0;
  int bsmax = 0;  // largest face block of the preconditioner
  size_t bytes = 0;
  std::vector<void*> allocs;
  std::vector<long long> h_uoff, h_toff;
  std::vector<int> h_nA, h_nT, h_deg;
  std::vector<double> xy;
  // device
  GenRef* ref = nullptr;
  int *deg = nullptr, *nbr = nullptr, *nbr_face = nullptr, *kind = nullptr, *tr_of = nullptr, *nfp = nullptr;
  long long *uoff = nullptr, *goff = nullptr, *toff = nullptr;
  double *geo_sol = nullptr, *geo_face = nullptr;
  unsigned char *implicit = nullptr, *dof_imp = nullptr;
  int *tpts = nullptr, *sides = nullptr, *pside = nullptr;
  long long* poff = nullptr;
  int *imp_idx = nullptr, *lto = nullptr, *nAk = nullptr, *nTk = nullptr, *gmap = nullptr;
  long long *offA = nullptr, *offB = nullptr, *offD = nullptr, *offr = nullptr, *offs = nullptr;
  int* fnode = nullptr;            // per element face point: its trace point (-1 off traces)
  unsigned char* fset = nullptr;   // per element face: 1 = GLL points (EFR)
  long long *gptr = nullptr, *gidx = nullptr;  // trace point <- element face points (CSR)
  long long *vptr = nullptr, *vidx = nullptr;  // trace value <- element-view entries (CSR)
  long long* nptr = nullptr;       // EFR node blocks: entries (implicit element, local row) per node
  int *nent_k = nullptr, *nent_l = nullptr;
  double *Uf_all = nullptr, *qf_all = nullptr, *Rw = nullptr, *gview = nullptr, *gw = nullptr, *Ustar = nullptr;
  double *r = nullptr, *s = nullptr, *xr = nullptr, *te = nullptr, *tg = nullptr, *yv = nullptr;
  double *duhat = nullptr, *du = nullptr, *red = nullptr;
  void *A = nullptr, *B = nullptr, *C = nullptr, *D = nullptr, *LU = nullptr, *XB = nullptr, *S = nullptr, *Pinv = nullptr;
  int* piv = nullptr;
  int* status = nullptr;
  int* exp_list = nullptr;  // the explicit elements (Eex)
  int Eex = 0;
  UnevenDev udev;
  // FP32 quadrilaterals: shape classes with the fixed-shape tensor-core condensation, condensed
  // through a contiguous scratch batch (the other elements by the uneven launch)
  struct TcClass {
    int nA, nT, count;
    int* list;          // device: compact implicit ids of the class
    int k0 = -1;        // >= 0: the class is the consecutive elements k0.. (condensed in place)
    long long off0[5];  // host: the offsets of element k0 (A, B/C, D, nA-vector, nT-vector)
  };
  std::vector<TcClass> tc_classes;
  void* cscratch = nullptr;
  int ccap = 0;
  GmresBuffers gm;
  bool lin_valid = false;
  void* jscratch = nullptr;  // hexahedra: pointwise Jacobians, one slab per CTA of the block kernel
  int jgrid = 0;
  // the implicit stage as one CUDA graph (imex_stage_set_graph), captured per key
  struct GKey {
    int stage = -1;
    double dt = 0.0;
    const double *u_n = nullptr, *u_stage = nullptr, *uhat = nullptr, *R_hist = nullptr;
    double ntol = 0.0, grtol = 0.0;
    int nmax = 0, gmax = 0;
    bool operator==(const GKey& o) const {
      return stage == o.stage && dt == o.dt && u_n == o.u_n && u_stage == o.u_stage && uhat == o.uhat &&
             R_hist == o.R_hist && ntol == o.ntol && grtol == o.grtol && nmax == o.nmax && gmax == o.gmax;
    }
  };
  int use_graph = 0;
  bool gvalid = false, capturing = false;
  GKey gkey;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cap[5] = {};
  void* gdev = nullptr;  // the stage's and the GMRES solve's device counters
  int gl_top = 0, gl_newton = 0, gl_solve = 0;
  GmresGraphLaunches gl_gm;
};

// hexahedra (hfr_hex.cu): the residual passes (mode GM_UF / GM_QF / GM_RES) and the element
// blocks, stored column-major
enum { GM_UF = 0, GM_QF = 1, GM_RES = 2 };
cudaError_t hex_elem_pass(GenCtx* g, const GArgs& a, int mode);
// metrics of a hexahedral mesh of one degree: per solution point {1/J, S[3][3]} (S = adjugate of
// dx/dxi, F~_r = sum_c S[r][c] F_c), per face point {J_f, n}, solution-point coordinates
void hex_geometry(const double* verts, int E, const int* deg, const long long* goff, double* gsol, double* gface,
                  double* xyz);
cudaError_t hex_jacobian(GenCtx* g, const GArgs& a, const JArgs& j);
size_t hex_jacobian_scratch_bytes(int prec_bytes, int grid);
int hex_jacobian_grid(int prec_bytes);

}  // namespace gen
}  // namespace hfr
