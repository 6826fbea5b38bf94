"""Interior-embedded FR (EFR): the hybridized residual with a trace that is continuous on the
implicit skeleton (Sec. 2.2; Secs. 4-5 pair it with explicit FR).  Test infrastructure: plain
FP64, only ``tests/`` use it.

The paper fixes: trace nodal basis continuous across interior faces, placed at the
Gauss-Lobatto-Legendre (GLL) points of each face; Gauss solution points; tensor-product
correction functions as for HFR, with an extra interpolation in the lift because face and flux
points differ; discontinuous (no) traces on the IMEX interface, which carries the FR flux.  It
defers the rest to its EFR reference.  Readings used here:

* trace unknowns: one node per vertex of the implicit skeleton (vertices joined through trace
  faces are one node) and the p - 1 interior GLL points of every trace face;
* on a trace face each side evaluates its state, gradient, one-sided flux
  F^ = F(u^) + s (u_f - u^) n - F^v(u^, q_f) (eq. hfrriemann) and J_f at the GLL points; the
  element's own state and gradient there are its polynomials evaluated at those points
  (interpolation along the face from its Gauss-aligned face values);
* the lift works at the element's Gauss-aligned face points: the GLL values of J_f F^.n and of
  the gradient jump u^ - u_f are interpolated there (degree-p Lagrange interpolation, exact for
  the element's own polynomials) before the DG-recovering corrections spread them;
* transmission condition of node i: g_i = sum over the trace faces f that carry node i and over
  both sides of w^GLL_q J_f,q (F^.n)_q at the face point q of node i, the GLL rule applied to
  the nodal basis function of i (collocated).  Summed over all nodes this is the face integral
  of the interpolated flux jump, so the implicit region is conservative as a whole, as the paper
  states for EFR, while single elements are not.

Boundary faces of implicit elements keep a discontinuous trace at their Gauss points with the wall
and far-field rows of ``oracle.boundary``; their nodes are their own.

Element-local trace layout is that of HFR (4 faces x (p+1) points x nv, a corner node appearing
once on each of its two faces); the condensed system gathers both copies into one unknown.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .basis import gauss_lobatto, lagrange
from .blocks import element_blocks, EPS
from .boundary import FARFIELD_FACE, WALL_FACE, BoundaryDiscretisation
from .fr import IMEX_FACE, TRACE_FACE
from .geometry import FACES_2D, _adjugate, _bilinear_derivs
from .physics import cmax
from .solve import condense, backsolve

# corners (a + 2 b in the element's vertex order) at the first and last point of each face
FACE_CORNERS = ((0, 2), (1, 3), (0, 1), (2, 3))


class EmbeddedDiscretisation(BoundaryDiscretisation):
    """EFR operators for a quad mesh with a single polynomial degree p >= 1: the continuous GLL
    trace on interior trace faces; on wall and far-field faces of implicit elements the
    discontinuous trace at the Gauss points with the boundary rows of ``oracle.boundary`` (the
    paper keeps discontinuous traces on boundaries, Sec. 4)."""

    def __init__(self, mesh, physics, u_inf=None):
        super().__init__(mesh, physics, u_inf)
        n = self.n
        self.efr = self.kind == TRACE_FACE  # continuous trace at the GLL points
        self.bface = self.traced & self.bnd  # discontinuous boundary trace at the Gauss points
        self.xl, self.wl = gauss_lobatto(n)
        self.IGL = lagrange(self.ref.x, self.xl)  # (GLL point q, Gauss-aligned point m)
        self.ILG = lagrange(self.xl, self.ref.x)  # (Gauss-aligned point m, GLL point q)
        self._gll_geometry()
        self._number_nodes()

    def _gll_geometry(self):
        """Scaled normal, J_f and unit normal at the GLL points of every element face (the faces of
        a bilinear element are straight, so these equal their values at the flux points)."""
        verts = self.mesh.verts
        E, n = verts.shape[0], self.n
        NfL = np.zeros((E, 4, n, 2))
        for f, (r, sg) in enumerate(FACES_2D):
            fx, fe = (np.full(n, sg), self.xl) if r == 0 else (self.xl, np.full(n, sg))
            a, b = _bilinear_derivs(verts, fx, fe)
            _, Sf = _adjugate(a, b)
            NfL[:, f] = sg * Sf[:, :, r, :]
        self.JfL = np.sqrt(np.sum(NfL**2, axis=-1))
        self.normalL = NfL / self.JfL[..., None]

    def _number_nodes(self):
        """node_of (E, 4, n): the global trace node at each point of each element face (-1 without
        a trace).  Vertex nodes first (in increasing smallest element corner), then the p - 1
        interior GLL points of each interior trace face (in increasing global face id), then the
        n Gauss points of each boundary trace face (same order)."""
        m = self.mesh
        E, n = m.nelem, self.n
        parent = np.arange(4 * E)

        def find(i):
            while parent[i] != i:
                parent[i] = parent[parent[i]]
                i = parent[i]
            return i

        touched = set()
        for e in range(E):
            for f in range(4):
                if not self.efr[e, f]:
                    continue
                nb, nf = m.nbr[e, f], m.nbr_face[e, f]
                for end in range(2):
                    i, j = 4 * e + FACE_CORNERS[f][end], 4 * nb + FACE_CORNERS[nf][end]
                    touched.update((i, j))
                    ri, rj = find(i), find(j)
                    if ri != rj:
                        parent[max(ri, rj)] = min(ri, rj)
        roots = sorted({find(i) for i in touched})
        vid = {r: k for k, r in enumerate(roots)}
        self.nvert = len(roots)
        fid = m.face_of
        inner = {g: k for k, g in enumerate(np.unique(fid[self.efr]))}
        outer = {g: k for k, g in enumerate(np.unique(fid[self.bface]))}
        base = self.nvert + len(inner) * (n - 2)
        self.nnode = base + len(outer) * n
        node_of = -np.ones((E, 4, n), dtype=np.int64)
        for e in range(E):
            for f in range(4):
                if self.efr[e, f]:
                    node_of[e, f, 0] = vid[find(4 * e + FACE_CORNERS[f][0])]
                    node_of[e, f, n - 1] = vid[find(4 * e + FACE_CORNERS[f][1])]
                    node_of[e, f, 1:n - 1] = self.nvert + inner[fid[e, f]] * (n - 2) + np.arange(n - 2)
                elif self.bface[e, f]:
                    node_of[e, f] = base + outer[fid[e, f]] * n + np.arange(n)
        self.node_of = node_of

    # ----------------------------------------------------------------- residual
    def corrected_gradient(self, U, uhat_view):
        """Physical gradient q (E, Ns, 2, nv): the reference gradient of u^D plus the lifted jumps
        u_bar - u_f: on EFR faces taken at the GLL points (u_bar = u^) and interpolated to the
        Gauss-aligned points; on boundary trace faces u^ at the Gauss points; on the other faces
        as in the uniform operator (ghost u_inf on explicit far-field faces)."""
        geo = self.geo
        kind = self.kind[:, :, None, None]
        imp_e = self.imp[:, None, None, None]
        Uf = self.interp_faces(U)
        Uf_nb = self._other_state(Uf)
        UfL = np.einsum("qm,efm...->efq...", self.IGL, Uf)
        jump = np.where(self.bface[:, :, None, None], uhat_view - Uf, 0.5 * (Uf_nb - Uf))
        jump = np.where(self.efr[:, :, None, None],
                        np.einsum("mq,efq...->efm...", self.ILG, uhat_view - UfL), jump)
        jump = np.where(kind == IMEX_FACE, np.where(imp_e, Uf_nb - Uf, 0.0 * Uf), jump)
        dxi, deta = self.ref_derivative(U)
        cx, cy = self.lift(jump, signed=False)
        Qr = np.stack([dxi + cx, deta + cy], axis=2)
        return np.einsum("esrc,esrv->escv", geo.S, Qr) / geo.J[:, :, None, None]

    def residual(self, U, uhat_view):
        """R(u, u^) and J_f times each element face point's trace row: J_f F^.n at the GLL points
        of EFR faces, the boundary rows at the Gauss points of boundary trace faces, J_f F^.n at the
        flux points elsewhere.

        U (E, Ns, nv); uhat_view (E, 4, n, nv) the trace at each element face's trace points.
        Returns R (E, Ns, nv) and that array (E, 4, n, nv)."""
        ph = self.phys
        geo = self.geo
        kind = self.kind[:, :, None, None]
        efr = self.efr[:, :, None, None]
        bface = self.bface[:, :, None, None]
        imp_e = self.imp[:, None, None, None]
        Uf = self.interp_faces(U)
        Uf_nb = self._other_state(Uf)
        UfL = np.einsum("qm,efm...->efq...", self.IGL, Uf)
        if ph.viscous:
            q = self.corrected_gradient(U, uhat_view)
            qf = self.interp_faces(q)
            qf_nb = self.neighbour(qf)
            qfL = np.einsum("qm,efm...->efq...", self.IGL, qf)
            F = ph.conv(U) - ph.visc(U, q)
        else:
            F = ph.conv(U)
        Ft = np.einsum("esrc,escv->esrv", geo.S, F)
        Ftf = self.interp_faces(Ft)
        FDn = np.empty_like(Uf)
        for f, (r, sg) in enumerate(FACES_2D):
            FDn[:, f] = sg * Ftf[:, f, :, r, :]

        def dotn(Fx, nrm):
            return np.einsum("...cv,...c->...v", Fx, nrm)

        def one_sided(uf, uh, qfx, nrm):
            s = ph.stab(uh, nrm)[..., None]
            Fh = dotn(ph.conv(uh), nrm) + s * (uf - uh)
            if ph.viscous:
                Fh = Fh - dotn(ph.visc(uh, qfx), nrm)
            return Fh, s

        # FR and IMEX-interface faces at the flux points
        nrm = geo.normal
        lam = cmax(ph.wave_speed(Uf, nrm), ph.wave_speed(Uf_nb, nrm))
        Fr = 0.5 * dotn(ph.conv(Uf) + ph.conv(Uf_nb), nrm) + 0.5 * lam[..., None] * (Uf - Uf_nb)
        if ph.viscous:
            Fr_fr = Fr - 0.5 * dotn(ph.visc(Uf, qf) + ph.visc(Uf_nb, qf_nb), nrm)
            U_im = np.where(imp_e, Uf, Uf_nb)
            q_im = np.where(imp_e[..., None], qf, qf_nb)
            Fr_im = Fr - dotn(ph.visc(U_im, q_im), nrm)
        else:
            Fr_fr = Fr_im = Fr
        Jf = geo.Jf[..., None]
        FnG = Jf * np.where(kind == IMEX_FACE, Fr_im, Fr_fr)
        # boundary trace faces: one-sided flux and boundary rows at the flux points
        uhB = np.where(bface, uhat_view, Uf)
        FhB, sB = one_sided(Uf, uhB, qf if ph.viscous else None, nrm)
        rowB = Jf * FhB
        if self.u_inf is not None:
            rowB = np.where(kind == FARFIELD_FACE, Jf * sB * ((Uf - uhB) + (self.u_inf - uhB)), rowB)
        if self.nv == 4:
            wall = Jf * np.concatenate([FhB[..., :1], sB * uhB[..., 1:3], FhB[..., 3:]], axis=-1)
            rowB = np.where(kind == WALL_FACE, wall, rowB)
        # EFR faces: one-sided flux at the GLL points, interpolated to the flux points for the lift
        uhL = np.where(efr, uhat_view, UfL)
        FhL, _ = one_sided(UfL, uhL, qfL if ph.viscous else None, self.normalL)
        FnL = self.JfL[..., None] * FhL
        FnL_G = np.einsum("mq,efq...->efm...", self.ILG, FnL)
        Fn = np.where(efr, FnL_G, np.where(bface, Jf * FhB, FnG))
        dxi, deta = self.ref_derivative(Ft)
        cx, cy = self.lift(Fn - FDn, signed=True)
        R = -(dxi[:, :, 0] + deta[:, :, 1] + cx + cy) / geo.J[:, :, None]
        return R, np.where(efr, FnL, np.where(bface, rowB, FnG))

    # ------------------------------------------------------------ trace helpers
    def trace_view(self, uhat):
        """Global trace (nnode, nv) -> per element face point (E, 4, n, nv); zero off trace."""
        view = np.zeros(self.node_of.shape + (self.nv,), dtype=uhat.dtype)
        has = self.node_of >= 0
        view[has] = uhat[self.node_of[has]]
        return view

    def trace_weights(self, Fn):
        """Element contribution to the trace rows: w^GLL on EFR faces, the Gauss weights on
        boundary trace faces, zero elsewhere."""
        w = np.where(self.efr[:, :, None], self.wl[None, None, :], self.geo.wface[None, None, :])
        return np.where(self.traced[:, :, None, None], w[..., None] * Fn, 0.0)

    def assemble_trace(self, gview):
        """Sum element-face-point contributions (E, 4, n, nv) into the nodes (nnode, nv)."""
        g = np.zeros((self.nnode, self.nv), dtype=gview.dtype)
        has = self.node_of >= 0
        np.add.at(g, self.node_of[has], gview[has])
        return g

    def initial_trace(self, U):
        """EFR nodes: the average, over every element face carrying the node, of that side's state
        there; boundary trace faces as in ``oracle.boundary``."""
        UfL = np.einsum("qm,efm...->efq...", self.IGL, self.interp_faces(U))
        acc = np.zeros((self.nnode, self.nv))
        cnt = np.zeros(self.nnode)
        has = (self.node_of >= 0) & self.efr[:, :, None]
        np.add.at(acc, self.node_of[has], UfL[has])
        np.add.at(cnt, self.node_of[has], 1.0)
        out = acc / np.maximum(cnt, 1.0)[:, None]
        if np.any(self.bface):
            hfr = BoundaryDiscretisation.initial_trace(self, U)  # (ntrace, n, nv) by trace face
            for e, f in zip(*np.nonzero(self.bface)):
                out[self.node_of[e, f]] = hfr[self.tr_of[e, f]]
        return out

    def full_residual(self, U, uhat):
        """R (E, Ns, nv) and the trace residual g (nnode, nv)."""
        R, Fn = self.residual(U, self.trace_view(uhat))
        return R, self.assemble_trace(self.trace_weights(Fn))

    def trace_dof_map(self):
        """(E, 4 n nv) global trace unknown of each element trace unknown, -1 off trace."""
        nv = self.nv
        idx = self.node_of[..., None] * nv + np.arange(nv)
        idx = np.where(self.node_of[..., None] >= 0, idx, -1)
        return idx.reshape(self.mesh.nelem, -1)


def condensed_newton_step(d, U, uhat, Ustar, a_dt):
    """One Newton step of the EFR stage equations by static condensation (Sec. 3.2): per element
    S_k, t_k; L = sum_k P_k^T S_k P_k with P_k gathering the element's face points from the
    nodes (both copies of a corner node sum); direct solve; back-substitution.
    Returns (dU (E, Ns, nv) zero on explicit elements, duhat (nnode, nv))."""
    imp = d.imp_idx
    nA, nT = d.ns * d.nv, 4 * d.n * d.nv
    R, Fn = d.residual(U, d.trace_view(uhat))
    gv = d.trace_weights(Fn)
    h = U[imp] - Ustar[imp] - a_dt * R[imp]
    A, B, C, D = element_blocks(d, U, uhat, a_dt)
    XB, xr, S, t = condense(A[imp], B[imp], C[imp], D[imp], -h.reshape(-1, nA),
                            -gv[imp].reshape(-1, nT))
    idx = d.trace_dof_map()[imp]
    N = d.nnode * d.nv
    rows = np.repeat(idx[:, :, None], nT, axis=2)
    cols = np.repeat(idx[:, None, :], nT, axis=1)
    ok = (rows >= 0) & (cols >= 0)
    L = sp.coo_matrix((S[ok], (rows[ok], cols[ok])), shape=(N, N)).tocsc()
    rhs = np.zeros(N)
    np.add.at(rhs, idx[idx >= 0], t[idx >= 0])
    duh = spla.spsolve(L, rhs).reshape(d.nnode, d.nv)
    du = backsolve(XB, xr, d.trace_view(duh)[imp].reshape(len(imp), nT))
    dU = np.zeros_like(U)
    dU[imp] = du.reshape(len(imp), d.ns, d.nv)
    return dU, duh


def monolithic_newton_step(d, U, uhat, Ustar, a_dt):
    """The same Newton step from the dense Jacobian of [h; g] in [u_implicit; u^] (tiny meshes)."""
    imp = d.imp_idx
    nA = d.ns * d.nv
    nu, nh = len(imp) * nA, d.nnode * d.nv
    Jm = np.zeros((nu + nh, nu + nh))
    Uc, Hc = U.astype(np.complex128), uhat.astype(np.complex128)
    for col in range(nu + nh):
        Up, Hp = Uc.copy(), Hc.copy()
        if col < nu:
            k, j = divmod(col, nA)
            Up[imp[k]].reshape(-1)[j] += 1j * EPS
        else:
            Hp.reshape(-1)[col - nu] += 1j * EPS
        R, g = d.full_residual(Up, Hp)
        Jm[:nu, col] = (Up[imp] - a_dt * R[imp]).imag.reshape(-1) / EPS
        Jm[nu:, col] = g.imag.reshape(-1) / EPS
    R, g = d.full_residual(U, uhat)
    rhs = -np.concatenate([(U[imp] - Ustar[imp] - a_dt * R[imp]).reshape(-1), g.reshape(-1)])
    x = np.linalg.solve(Jm, rhs)
    dU = np.zeros_like(U)
    dU[imp] = x[:nu].reshape(len(imp), d.ns, d.nv)
    return dU, x[nu:].reshape(d.nnode, d.nv)


def newton_stage(d, U0, Ustar, uhat0, a_dt, tol=1e-8, maxit=25, linear="direct"):
    """Newton on the EFR stage equations with condensed steps and the stopping test of the
    uniform oracle, ||[h; g]||_2 <= tol ||[h; g]^0||_2.  Returns U, uhat, info."""
    U, uhat = U0.copy(), uhat0.copy()
    imp = d.imp_idx
    hist = []
    for it in range(maxit + 1):
        R, g = d.full_residual(U, uhat)
        h = U[imp] - Ustar[imp] - a_dt * R[imp]
        hist.append(float(np.sqrt(np.sum(h * h) + np.sum(g * g))))
        if hist[-1] <= tol * hist[0] or hist[-1] == 0.0 or it == maxit:
            break
        dU, duh = condensed_newton_step(d, U, uhat, Ustar, a_dt)
        U, uhat = U + dU, uhat + duh
    converged = hist[-1] <= tol * hist[0] or hist[-1] == 0.0
    return U, uhat, {"history": hist, "iterations": len(hist) - 1, "converged": converged}
