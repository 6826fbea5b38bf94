"""Element Jacobian blocks (Sec. 3.2, eqs. elemA, elemsystem, elemsystemB).

For the stage residuals (eqs. 9oind, 23nffsd)

    h(u, u^) = u - u* - a_ii dt R(u, u^),        g(u, u^) = 0,

the Newton matrix is [A B; C D] with, per implicit element k,
A_k = dh_k/du_k, B_k = dh_k/du^_k, C_k = dg^k/du_k, D_k = dg^k/du^_k where g^k
is element k's contribution w_q J_f F^_k . n_k to the trace residual.  Sign
reading: the paper's eq. elemA prints A = delta - dt a (1/J)[...] and
eq. 9oind writes u - u* - a dt f with eq. 099io defining u_t + f = 0; here R is
the time derivative, so A = I - a dt dR/du and B = -a dt dR/du^, which makes
A -> I as dt -> 0.

Derivatives are taken by complex-step differentiation of the element residual,
d/dx f(x) = Im f(x + i eps) / eps with eps = 1e-30, exact to rounding for the
real-analytic (piecewise) fluxes.  Local index conventions (also those of the
GPU library's block layout):

* element unknown i = pt * nv + v  (pt = a + n b),
* element trace unknown l = (f * n + m) * nv + v over all four faces (columns /
  rows of faces without a trace are zero).
"""

from __future__ import annotations

import numpy as np

EPS = 1.0e-30


def element_blocks(disc, U, uhat, a_dt: float, view=None):
    """A, B, C, D for every element, shapes (E, nA, nA), (E, nA, nT),
    (E, nT, nA), (E, nT, nT).  Only implicit elements' blocks are meaningful.
    view (optional): per element-face trace values (E, 4, n, nv) used instead of
    disc.trace_view(uhat) (the blocks of a hybridized element depend only on its
    own state and its own faces' traces)."""
    E = disc.mesh.nelem
    nv, ns, n = disc.nv, disc.ns, disc.n
    nA = ns * nv
    nT = 4 * n * nv
    if view is None:
        view = disc.trace_view(uhat)
    Uc = U.astype(np.complex128)
    Vc = view.astype(np.complex128)
    imp = disc.imp
    dRdu = np.zeros((E, nA, nA))
    dGdu = np.zeros((E, nT, nA))
    for j in range(nA):
        pt, v = divmod(j, nv)
        Up = Uc.copy()
        Up[imp, pt, v] += 1j * EPS
        R, Fn = disc.residual(Up, Vc)
        dRdu[:, :, j] = R.imag.reshape(E, nA) / EPS
        dGdu[:, :, j] = disc.trace_weights(Fn).imag.reshape(E, nT) / EPS
    dRdh = np.zeros((E, nA, nT))
    dGdh = np.zeros((E, nT, nT))
    for l in range(nT):
        fm, v = divmod(l, nv)
        f, m = divmod(fm, n)
        Vp = Vc.copy()
        Vp[imp, f, m, v] += 1j * EPS
        R, Fn = disc.residual(Uc, Vp)
        dRdh[:, :, l] = R.imag.reshape(E, nA) / EPS
        dGdh[:, :, l] = disc.trace_weights(Fn).imag.reshape(E, nT) / EPS
    A = np.eye(nA)[None] - a_dt * dRdu
    B = -a_dt * dRdh
    return A, B, dGdu, dGdh


def global_jacobian(disc, U, uhat, a_dt: float):
    """Monolithic Jacobian of [h; g] with respect to [u_im; u^] (dense), for
    tiny meshes only.  Unknown order: implicit elements in increasing index,
    each element's nA unknowns, then the global trace (t, m, v)."""
    imp_idx = disc.imp_idx
    nA = disc.ns * disc.nv
    nu = len(imp_idx) * nA
    nh = disc.ntrace * disc.n * disc.nv
    N = nu + nh
    Jm = np.zeros((N, N))
    Uc = U.astype(np.complex128)
    Hc = uhat.astype(np.complex128)
    for col in range(N):
        Up = Uc.copy()
        Hp = Hc.copy()
        if col < nu:
            k, j = divmod(col, nA)
            pt, v = divmod(j, disc.nv)
            Up[imp_idx[k], pt, v] += 1j * EPS
        else:
            t, r = divmod(col - nu, disc.n * disc.nv)
            m, v = divmod(r, disc.nv)
            Hp[t, m, v] += 1j * EPS
        R, g = disc.full_residual(Up, Hp)
        dh = Up[imp_idx].imag / EPS - a_dt * R[imp_idx].imag / EPS
        Jm[:nu, col] = dh.reshape(-1)
        Jm[nu:, col] = g.imag.reshape(-1) / EPS
    return Jm
