"""Element mapping and metric terms (Sec. 2, eqs. d9sfxda, 3289u4, 8923i).

Quadrilaterals use the bilinear map x = sum_k M_k(xi) x^g_k over the four
corners (Sec. 2: x = M_k(x~) = sum_i M_i(x~) x^g_i).  With the Jacobian
matrix J[c, r] = dx_c / dxi_r and determinant J, the metric stored is the
adjugate S = J J^{-1}, S[r, c] = J dxi_r / dx_c, so that the transformed flux is
F~_r = sum_c S[r, c] F_c (eq. d9sfxda).  On a face with reference outward
normal n~ (axis r, sign sigma) the scaled physical normal is
N = J J^{-T} n~, N_c = sigma S[r, c]; then J_f = |N| and n = N / J_f, so that
F^~ . n~ = J_f F^ . n (eq. 8923i).

Local numbering: solution point pt = a + n b (a along xi); faces
0: xi=-1, 1: xi=+1, 2: eta=-1, 3: eta=+1; on xi-faces point m = b, on
eta-faces m = a.
"""

from __future__ import annotations

import numpy as np

from .basis import RefElement1D

# (axis, sign) of each local face
FACES_2D = ((0, -1.0), (0, +1.0), (1, -1.0), (1, +1.0))


def _bilinear_derivs(verts: np.ndarray, xi: np.ndarray, eta: np.ndarray):
    """dx/dxi, dx/deta at reference points (xi, eta) for every element.
    verts (E, 4, 2); xi, eta (P,) -> (E, P, 2) each."""
    sa = np.array([-1.0, 1.0, -1.0, 1.0])
    sb = np.array([-1.0, -1.0, 1.0, 1.0])
    dNdxi = 0.25 * sa[None, :] * (1.0 + sb[None, :] * eta[:, None])  # (P, 4)
    dNdeta = 0.25 * sb[None, :] * (1.0 + sa[None, :] * xi[:, None])
    x_xi = np.einsum("pk,ekc->epc", dNdxi, verts)
    x_eta = np.einsum("pk,ekc->epc", dNdeta, verts)
    return x_xi, x_eta


def _adjugate(x_xi: np.ndarray, x_eta: np.ndarray):
    """Determinant and adjugate S[r, c] of J[c, r] = (x_xi, x_eta)."""
    J = x_xi[..., 0] * x_eta[..., 1] - x_eta[..., 0] * x_xi[..., 1]
    S = np.empty(x_xi.shape[:-1] + (2, 2))
    S[..., 0, 0] = x_eta[..., 1]
    S[..., 0, 1] = -x_eta[..., 0]
    S[..., 1, 0] = -x_xi[..., 1]
    S[..., 1, 1] = x_xi[..., 0]
    return J, S


class QuadGeometry:
    """Metric terms at solution points and flux points of every element."""

    def __init__(self, verts: np.ndarray, ref: RefElement1D):
        n = ref.n
        self.n = n
        self.ns = n * n
        x = ref.x
        xi = np.tile(x, n)
        eta = np.repeat(x, n)
        x_xi, x_eta = _bilinear_derivs(verts, xi, eta)
        self.J, self.S = _adjugate(x_xi, x_eta)  # (E, Ns), (E, Ns, 2, 2)
        # physical coordinates of the solution points
        sa = np.array([-1.0, 1.0, -1.0, 1.0])
        sb = np.array([-1.0, -1.0, 1.0, 1.0])
        N = 0.25 * (1 + sa[None, :] * xi[:, None]) * (1 + sb[None, :] * eta[:, None])
        self.xy = np.einsum("pk,ekc->epc", N, verts)
        # flux points
        E = verts.shape[0]
        self.Nf = np.zeros((E, 4, n, 2))
        for f, (r, sg) in enumerate(FACES_2D):
            if r == 0:
                fx, fe = np.full(n, sg), x
            else:
                fx, fe = x, np.full(n, sg)
            a, b = _bilinear_derivs(verts, fx, fe)
            _, Sf = _adjugate(a, b)
            self.Nf[:, f] = sg * Sf[:, :, r, :]
        self.Jf = np.sqrt(np.sum(self.Nf**2, axis=-1))  # (E, 4, n)
        self.normal = self.Nf / self.Jf[..., None]
        self.wface = ref.w.copy()  # quadrature weights of the face points
