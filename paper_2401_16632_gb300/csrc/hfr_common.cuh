// Shared device-side definitions of the hybridized FR library.
//
// Discretisation (Pereira & Vermeire, arXiv 2401.16632, Sec. 2): tensor-product
// Gauss-Legendre solution points, DG-recovering correction functions.  With the
// 1D lift l_i(+-1)/w_i of those correction functions, the corrected gradient and
// the flux divergence along every reference axis use the same 1D operator
//     M = D - dgL lm^T - dgR lp^T,   dgL = -lm / w,  dgR = lp / w,
// (D the Lagrange derivative matrix, lm / lp the interpolation to xi = -1 / +1):
//     Q~_r  = M U|_line + dgL u_bar_L + dgR u_bar_R           (gradient, eq. fluxcorrection)
//     div   = sum_r M F~_r|_line - dgL Fn_L + dgR Fn_R          (eqs. correctedflux, freq1)
// where Fn = J_f F^.n is the common normal flux (eq. 8923i).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define HFR_MAXN 6  // up to p = 5

// -------------------------------------------------------------------------------------------
// Reference 1D operators for one polynomial degree, passed by value as a kernel parameter.
struct RefOps {
  double D[HFR_MAXN][HFR_MAXN];
  double M[HFR_MAXN][HFR_MAXN];
  double lm[HFR_MAXN], lp[HFR_MAXN];
  double dgL[HFR_MAXN], dgR[HFR_MAXN];
  double w[HFR_MAXN];
};

struct PhysParams {
  int kind;  // 0 advection-diffusion, 1 Navier-Stokes 2D, 2 EDAC 2D, 3 Navier-Stokes 3D
  double beta[3];
  double nu;
  double gamma, mu, Pr;
  double lref;
  double theta;  // EDAC: 1 / M^2 of the artificial Mach number
};
// viscous terms present (advection-diffusion and EDAC: nu; Navier-Stokes: mu)
__host__ __device__ inline bool phys_viscous(const PhysParams& pp) {
  return (pp.kind == 1 || pp.kind == 3) ? pp.mu != 0.0 : pp.nu != 0.0;
}

// face kinds of an element face
enum { FK_FR = 0, FK_TRACE = 1, FK_IMEX = 2 };

// -------------------------------------------------------------------------------------------
// Forward-mode dual number with one tangent (exact pointwise Jacobians and JVPs).
template <typename T>
struct Dual {
  T v, d;
  __host__ __device__ Dual() {}
  __host__ __device__ Dual(T a) : v(a), d(T(0)) {}
  __host__ __device__ Dual(T a, T b) : v(a), d(b) {}
};
template <typename T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return Dual<T>(a.v + b.v, a.d + b.d); }
template <typename T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return Dual<T>(a.v - b.v, a.d - b.d); }
template <typename T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return Dual<T>(-a.v, -a.d); }
template <typename T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return Dual<T>(a.v * b.v, a.d * b.v + a.v * b.d); }
template <typename T> __device__ __forceinline__ Dual<T> operator/(Dual<T> a, Dual<T> b) {
  T inv = T(1) / b.v;
  T q = a.v * inv;
  return Dual<T>(q, (a.d - q * b.d) * inv);
}
template <typename T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, T b) { return Dual<T>(a.v + b, a.d); }
template <typename T> __device__ __forceinline__ Dual<T> operator+(T a, Dual<T> b) { return Dual<T>(a + b.v, b.d); }
template <typename T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, T b) { return Dual<T>(a.v - b, a.d); }
template <typename T> __device__ __forceinline__ Dual<T> operator-(T a, Dual<T> b) { return Dual<T>(a - b.v, -b.d); }
template <typename T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, T b) { return Dual<T>(a.v * b, a.d * b); }
template <typename T> __device__ __forceinline__ Dual<T> operator*(T a, Dual<T> b) { return Dual<T>(a * b.v, a * b.d); }
template <typename T> __device__ __forceinline__ Dual<T> operator/(Dual<T> a, T b) { T inv = T(1) / b; return Dual<T>(a.v * inv, a.d * inv); }
template <typename T> __device__ __forceinline__ Dual<T> operator/(T a, Dual<T> b) {
  T inv = T(1) / b.v;
  T q = a * inv;
  return Dual<T>(q, -q * b.d * inv);
}

__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
template <typename T> __device__ __forceinline__ Dual<T> dsqrt(Dual<T> a) {
  T s = dsqrt(a.v);
  return Dual<T>(s, a.d / (T(2) * s));
}
// |x| with the branch taken on the value
__device__ __forceinline__ double dabs(double x) { return fabs(x); }
__device__ __forceinline__ float dabs(float x) { return fabsf(x); }
template <typename T> __device__ __forceinline__ Dual<T> dabs(Dual<T> a) { return a.v >= T(0) ? a : -a; }
__device__ __forceinline__ double dval(double x) { return x; }
__device__ __forceinline__ float dval(float x) { return x; }
template <typename T> __device__ __forceinline__ T dval(Dual<T> a) { return a.v; }
template <typename S> __device__ __forceinline__ S dmax(S a, S b) { return dval(a) >= dval(b) ? a : b; }

// underlying real type of a scalar
template <typename S> struct RealOf { typedef S type; };
template <typename T> struct RealOf<Dual<T>> { typedef T type; };

// -------------------------------------------------------------------------------------------
// Physics.  Fluxes F[c][v] (c = physical direction, v = variable).  q[c][v] = du_v/dx_c.
// Same readings as the oracle: advection-diffusion F^c = beta u, F^v = nu grad u,
// s = |beta.n| + nu/lref; Navier-Stokes ideal gas R = 1, constant mu, Stokes hypothesis,
// kappa = mu gamma / ((gamma - 1) Pr), wave speed |v.n| + c, s = |v^.n| + c^ + mu/(rho^ lref).
// Physics constants in the compute precision R, derived once per thread from PhysParams so
// that no double arithmetic or conversion happens inside the flux evaluations of FP32 kernels.
template <typename R>
struct PhysConst {
  R beta0, beta1, nu, nu_lref;          // advection-diffusion
  R gamma, gm1, mu, kappa, mu_lref;     // Navier-Stokes
  R theta;                              // EDAC
};
template <typename R>
__host__ __device__ inline PhysConst<R> phys_const(const PhysParams& pp) {
  PhysConst<R> c;
  c.beta0 = R(pp.beta[0]);
  c.beta1 = R(pp.beta[1]);
  c.nu = R(pp.nu);
  c.nu_lref = R(pp.nu / pp.lref);
  c.gamma = R(pp.gamma);
  c.gm1 = R(pp.gamma - 1.0);
  c.mu = R(pp.mu);
  c.kappa = (pp.kind == 1 || pp.kind == 3) ? R(pp.mu * pp.gamma / ((pp.gamma - 1.0) * pp.Pr)) : R(0);
  c.mu_lref = R(pp.mu / pp.lref);
  c.theta = R(pp.theta);
  return c;
}

template <int PHYS> struct Phys;

template <> struct Phys<0> {
  static constexpr int NV = 1;
  template <typename S, typename R>
  __device__ static void conv(const PhysConst<R>& pc, const S* u, S F[2][1]) {
    F[0][0] = pc.beta0 * u[0];
    F[1][0] = pc.beta1 * u[0];
  }
  template <typename S, typename R>
  __device__ static void visc(const PhysConst<R>& pc, const S* u, const S q[2][1], S F[2][1]) {
    F[0][0] = pc.nu * q[0][0];
    F[1][0] = pc.nu * q[1][0];
  }
  template <typename S, typename R>
  __device__ static S wave(const PhysConst<R>& pc, const S* u, R n0, R n1) {
    R bn = pc.beta0 * n0 + pc.beta1 * n1;
    return S(dabs(bn)) + R(0) * u[0];
  }
  template <typename S, typename R>
  __device__ static S stab(const PhysConst<R>& pc, const S* u, R n0, R n1) {
    return wave<S, R>(pc, u, n0, n1) + pc.nu_lref;
  }
};

template <> struct Phys<1> {
  static constexpr int NV = 4;
  template <typename S, typename R>
  __device__ static void conv(const PhysConst<R>& pc, const S* u, S F[2][4]) {
    S rho = u[0];
    S ir = R(1) / rho;
    S vx = u[1] * ir, vy = u[2] * ir;
    S p = pc.gm1 * (u[3] - R(0.5) * (u[1] * vx + u[2] * vy));
    S Ep = u[3] + p;
    F[0][0] = u[1];
    F[0][1] = u[1] * vx + p;
    F[0][2] = u[2] * vx;
    F[0][3] = Ep * vx;
    F[1][0] = u[2];
    F[1][1] = u[1] * vy;
    F[1][2] = u[2] * vy + p;
    F[1][3] = Ep * vy;
  }
  template <typename S, typename R>
  __device__ static void visc(const PhysConst<R>& pc, const S* u, const S q[2][4], S F[2][4]) {
    const R mu = pc.mu;
    S rho = u[0];
    S ir = R(1) / rho;
    S vx = u[1] * ir, vy = u[2] * ir;
    S e = u[3] * ir;
    S dvx[2], dvy[2], dT[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      dvx[c] = (q[c][1] - vx * q[c][0]) * ir;
      dvy[c] = (q[c][2] - vy * q[c][0]) * ir;
      dT[c] = pc.gm1 * ((q[c][3] - e * q[c][0]) * ir - vx * dvx[c] - vy * dvy[c]);
    }
    S div = dvx[0] + dvy[1];
    S txx = mu * (R(2) * dvx[0] - R(2.0 / 3.0) * div);
    S tyy = mu * (R(2) * dvy[1] - R(2.0 / 3.0) * div);
    S txy = mu * (dvx[1] + dvy[0]);
    F[0][0] = S(R(0));
    F[0][1] = txx;
    F[0][2] = txy;
    F[0][3] = vx * txx + vy * txy + pc.kappa * dT[0];
    F[1][0] = S(R(0));
    F[1][1] = txy;
    F[1][2] = tyy;
    F[1][3] = vx * txy + vy * tyy + pc.kappa * dT[1];
  }
  template <typename S, typename R>
  __device__ static S wave(const PhysConst<R>& pc, const S* u, R n0, R n1) {
    S rho = u[0];
    S ir = R(1) / rho;
    S vx = u[1] * ir, vy = u[2] * ir;
    S p = pc.gm1 * (u[3] - R(0.5) * (u[1] * vx + u[2] * vy));
    S c = dsqrt(pc.gamma * p * ir);
    return dabs(vx * n0 + vy * n1) + c;
  }
  template <typename S, typename R>
  __device__ static S stab(const PhysConst<R>& pc, const S* u, R n0, R n1) {
    return wave<S, R>(pc, u, n0, n1) + pc.mu_lref / u[0];
  }
};

// EDAC (Appendix A): u = (P, v_x, v_y), F^c_i = (v_i (P + Theta), v_i v_x + P delta_ix,
// v_i v_y + P delta_iy), F^v_i = nu du/dx_i.  Rusanov speed: the largest eigenvalue magnitude of
// the normal flux Jacobian, 3/2 |v.n| + sqrt((v.n)^2/4 + P + Theta); hybridized stabilisation
// (Sec. 5.4): 3/2 |v| + sqrt(|v|^2/4 + P + Theta), isotropic, plus nu / lref.
template <> struct Phys<2> {
  static constexpr int NV = 3;
  template <typename S, typename R>
  __device__ static void conv(const PhysConst<R>& pc, const S* u, S F[2][3]) {
    const S Pt = u[0] + pc.theta;
    F[0][0] = u[1] * Pt;
    F[0][1] = u[1] * u[1] + u[0];
    F[0][2] = u[1] * u[2];
    F[1][0] = u[2] * Pt;
    F[1][1] = u[2] * u[1];
    F[1][2] = u[2] * u[2] + u[0];
  }
  template <typename S, typename R>
  __device__ static void visc(const PhysConst<R>& pc, const S* u, const S q[2][3], S F[2][3]) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int v = 0; v < 3; ++v) F[c][v] = pc.nu * q[c][v];
  }
  template <typename S, typename R>
  __device__ static S wave(const PhysConst<R>& pc, const S* u, R n0, R n1) {
    const S vn = u[1] * n0 + u[2] * n1;
    return R(1.5) * dabs(vn) + dsqrt(R(0.25) * vn * vn + u[0] + pc.theta);
  }
  template <typename S, typename R>
  __device__ static S stab(const PhysConst<R>& pc, const S* u, R n0, R n1) {
    const S v2 = u[1] * u[1] + u[2] * u[2];
    return R(1.5) * dsqrt(v2) + dsqrt(R(0.25) * v2 + u[0] + pc.theta) + pc.nu_lref;
  }
};

// -------------------------------------------------------------------------------------------
// Geometry layout (double, per element):
//   sol: [Ns][5] = {1/J, S00, S01, S10, S11}  (S = adjugate of dx/dxi, F~_r = sum_c S[r][c] F_c)
//   face: [4][n][3] = {J_f, n0, n1}            (unit outward normal, face Jacobian)
// Element face f: axis r = f >> 1, side sigma = (f & 1) ? +1 : -1.  Face point m is the line
// index along the other axis.  Solution point pt = a + n b.
__device__ __forceinline__ int face_axis(int f) { return f >> 1; }

// index of the solution point at coordinate c along axis r on line m
template <int N>
__device__ __forceinline__ int line_pt(int r, int m, int c) {
  return r == 0 ? (c + N * m) : (m + N * c);
}

// status word bits written by kernels (never trap)
enum { DEV_ERR_SINGULAR = 1, DEV_ERR_NAN = 2, DEV_ERR_INDEX = 4, DEV_ERR_TIMEOUT = 8 };

// -------------------------------------------------------------------------------------------
// Bounds-checked build (compile flag FR_CHECKED): every mesh-derived gather / scatter index of
// the general path (trace point of an element face point, neighbour element and face, element
// face point of a trace point, element-view entry of a trace value, trace value of an
// element-view entry) and of the uniform path's residual and blocks (trace face, neighbour) goes
// through FR_IDX(i, n, site): an index outside [0, n) is recorded in this translation unit's
// device word (the first one: site and index; and a count) and replaced by 0, so the access
// stays in bounds and the kernel goes on (never a trap).  fr_checked_status reads and clears the
// words of every unit.  Without the flag FR_IDX is the index itself.
#ifdef FR_CHECKED
namespace fr_chk {
static __device__ unsigned long long g_first;  // (site << 48) | (index & (2^48 - 1)), 0 = none
static __device__ unsigned long long g_count;
__device__ __forceinline__ long long idx(long long i, long long n, int site) {
  if (i >= 0 && i < n) return i;
  atomicCAS(&g_first, 0ull, ((unsigned long long)(site & 0xFFFF) << 48) | ((unsigned long long)i & 0xFFFFFFFFFFFFull));
  atomicAdd(&g_count, 1ull);
  return 0;
}
}  // namespace fr_chk
#define FR_IDX(i, n, site) ::fr_chk::idx((long long)(i), (long long)(n), (site))
#else
#define FR_IDX(i, n, site) (i)
#endif
