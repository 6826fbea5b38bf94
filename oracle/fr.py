"""FR and hybridized-FR residuals on a quadrilateral mesh (Secs. 2, 4).

Spatial operator (eqs. frfluxd, fluxcorrection, correctedflux, freq1, hfr1):

    du/dt = R(u) = -(1/J) [ sum_r d/dxi_r F~_r  +  sum_f sum_m (div g_f^m) H~_{f,m} ]

with F~ = S F (S the adjugate metric), H~ = J_f F^.n - F~^D . n~ the flux jump
at flux point m of face f and the DG-recovering correction functions, whose
divergence at the solution points along the face's axis is sigma * g_sigma'(xi).

Common fluxes:
* standard FR faces (Sec. 2.1): Rusanov, 1/2 (F(u-) + F(u+)).n + s/2 (u- - u+),
  s = max wave speed of the two states;
* hybridized faces (eq. hfrriemann): F(u^) + s (u_f - u^) n, one-sided;
* IMEX-interface faces (Sec. 4, eq. hfrimex): the standard FR flux of the
  implicit and explicit states; there is no trace there.

Trace residual (eqs. 5treerf, 53904jn, hfr2): per trace point q of a global face,
g_q = w_q J_{f,q} (F^_+ . n_+ + F^_- . n_-), i.e. the Gauss rule on the face
applied to the jump of the one-sided fluxes against the nodal trace basis.
Because the face mass matrix is diagonal on Gauss trace points, this is the
pointwise form the paper notes for discontinuous traces (end of Sec. 4).

Viscous terms are not written in the paper; the reading used here:
* corrected gradient q = J^{-T} [grad~ u^D + sum_f sum_m n~_f (div g_f^m)(u_bar - u_f)_m]
  with common solution u_bar = average of both sides on FR faces (BR1),
  u_bar = u^ (the element's own trace) on hybridized faces, and on IMEX-interface
  faces u_bar = the explicit side's value (so the explicit element's correction
  there vanishes and the implicit element's stays local);
* viscous common flux: average of both sides' F^v on FR faces; F^v(u^, q_f) on
  hybridized faces (inside the one-sided flux above); on IMEX-interface faces
  F^v of the implicit side's state and gradient, used identically from both
  sides so that the interface flux stays single-valued (conservative).
"""

from __future__ import annotations

import numpy as np

from .basis import RefElement1D
from .geometry import QuadGeometry, FACES_2D
from .physics import cmax

FR_FACE = 0
TRACE_FACE = 1
IMEX_FACE = 2


class Discretisation:
    """FR/HFR operators for a quad mesh with a single polynomial degree."""

    def __init__(self, mesh, physics):
        p = int(mesh.p[0])
        if np.any(mesh.p != p):
            raise NotImplementedError("oracle: uniform p only")
        if np.any(mesh.nbr < 0):
            raise NotImplementedError("oracle: boundary faces not implemented")
        self.mesh = mesh
        self.phys = physics
        self.p = p
        self.ref = RefElement1D(p)
        self.n = p + 1
        self.ns = self.n**2
        self.nv = physics.nv
        self.geo = QuadGeometry(mesh.verts, self.ref)
        E = mesh.nelem
        imp = mesh.implicit
        self.imp = imp
        kind = np.full((E, 4), FR_FACE, dtype=np.int32)
        for f in range(4):
            nb = mesh.nbr[:, f]
            both = imp & imp[nb]
            mixed = imp != imp[nb]
            kind[both, f] = TRACE_FACE
            kind[mixed, f] = IMEX_FACE
        self.kind = kind
        # trace numbering: trace faces in increasing global face id
        fid = mesh.face_of
        trace_fids = np.unique(fid[kind == TRACE_FACE])
        tr_of_fid = -np.ones(mesh.nface, dtype=np.int64)
        tr_of_fid[trace_fids] = np.arange(len(trace_fids))
        self.ntrace = len(trace_fids)
        self.tr_of = np.where(kind == TRACE_FACE, tr_of_fid[fid], -1)  # (E, 4)
        # element-face pairs of each trace face: owner side 0 = first appearance
        self.trace_sides = -np.ones((self.ntrace, 2, 2), dtype=np.int64)
        for e in range(E):
            for f in range(4):
                t = self.tr_of[e, f]
                if t >= 0:
                    s = 0 if self.trace_sides[t, 0, 0] < 0 else 1
                    self.trace_sides[t, s] = (e, f)
        self.imp_idx = np.nonzero(imp)[0]
        self.ex_idx = np.nonzero(~imp)[0]

    # ------------------------------------------------------------------ helpers
    def _grid(self, X):
        """(E, Ns, ...) -> (E, n_b, n_a, ...)"""
        return X.reshape((X.shape[0], self.n, self.n) + X.shape[2:])

    def _flat(self, X):
        return X.reshape((X.shape[0], self.ns) + X.shape[3:])

    def interp_faces(self, X):
        """Values at the flux points of every face: (E, Ns, *r) -> (E, 4, n, *r)."""
        G = self._grid(X)
        r = self.ref
        out = np.empty((X.shape[0], 4, self.n) + X.shape[2:], dtype=X.dtype)
        out[:, 0] = np.einsum("a,eba...->eb...", r.lm, G)
        out[:, 1] = np.einsum("a,eba...->eb...", r.lp, G)
        out[:, 2] = np.einsum("b,eba...->ea...", r.lm, G)
        out[:, 3] = np.einsum("b,eba...->ea...", r.lp, G)
        return out

    def ref_derivative(self, X):
        """(d/dxi X, d/deta X) at the solution points."""
        G = self._grid(X)
        D = self.ref.D
        dxi = np.einsum("ij,ebj...->ebi...", D, G)
        deta = np.einsum("ij,ej...->ei...", D, G)
        return self._flat(dxi), self._flat(deta)

    def lift(self, face_vals, signed):
        """sum_f c_f(xi) face_vals_f spread along each face's axis, where
        c_f = g_sigma' (signed=False, gradient correction n~_r div g) or
        sigma g_sigma' (signed=True, divergence of the correction flux).
        face_vals (E, 4, n, *r) -> two arrays (xi-part, eta-part) (E, Ns, *r)."""
        r = self.ref
        E = face_vals.shape[0]
        shp = (E, self.n, self.n) + face_vals.shape[3:]
        cx = np.zeros(shp, dtype=face_vals.dtype)
        cy = np.zeros(shp, dtype=face_vals.dtype)
        sl = -1.0 if signed else 1.0
        # xi faces: value indexed by b, spread along a
        cx += np.einsum("a,eb...->eba...", sl * r.dgL, face_vals[:, 0])
        cx += np.einsum("a,eb...->eba...", r.dgR, face_vals[:, 1])
        # eta faces: value indexed by a, spread along b
        cy += np.einsum("b,ea...->eba...", sl * r.dgL, face_vals[:, 2])
        cy += np.einsum("b,ea...->eba...", r.dgR, face_vals[:, 3])
        return self._flat(cx), self._flat(cy)

    def neighbour(self, Xf):
        """Face values seen from the other side of each face: (E, 4, ...)"""
        m = self.mesh
        return Xf[m.nbr, m.nbr_face]

    # ----------------------------------------------------------------- residual
    def residual(self, U, uhat_view):
        """R(u, u^) at every element and J_f F^.n at every element flux point.

        U (E, Ns, nv); uhat_view (E, 4, n, nv) the trace seen by each element
        face (read on hybridized faces only).  Returns R (E, Ns, nv) and
        Fn (E, 4, n, nv)."""
        ph = self.phys
        geo = self.geo
        kind = self.kind[:, :, None, None]
        imp_e = self.imp[:, None, None, None]
        Uf = self.interp_faces(U)
        Uf_nb = self.neighbour(Uf)
        # common solution for the gradient correction
        ubar = np.where(kind == TRACE_FACE, uhat_view, 0.5 * (Uf + Uf_nb))
        ubar = np.where(kind == IMEX_FACE, np.where(imp_e, Uf_nb, Uf), ubar)
        if ph.viscous:
            dxi, deta = self.ref_derivative(U)
            cx, cy = self.lift(ubar - Uf, signed=False)
            Qr = np.stack([dxi + cx, deta + cy], axis=2)  # (E, Ns, 2, nv) reference
            # physical gradient q_c = (1/J) sum_r S[r, c] Q~_r
            q = np.einsum("esrc,esrv->escv", geo.S, Qr) / geo.J[:, :, None, None]
            qf = self.interp_faces(q)  # (E, 4, n, 2, nv)
            qf_nb = self.neighbour(qf)
            F = ph.conv(U) - ph.visc(U, q)
        else:
            F = ph.conv(U)
        Ft = np.einsum("esrc,escv->esrv", geo.S, F)  # transformed flux
        Ftf = self.interp_faces(Ft)  # (E, 4, n, 2, nv)
        FDn = np.empty_like(Uf)
        for f, (r, sg) in enumerate(FACES_2D):
            FDn[:, f] = sg * Ftf[:, f, :, r, :]
        nrm = geo.normal  # (E, 4, n, 2)

        def dotn(Fx):
            return np.einsum("...cv,...c->...v", Fx, nrm)

        # hybridized one-sided flux (faces without a trace evaluate it at a
        # harmless state and discard it)
        uh = np.where(kind == TRACE_FACE, uhat_view, Uf)
        Fh = dotn(ph.conv(uh)) + ph.stab(uh, nrm)[..., None] * (Uf - uh)
        # standard FR Rusanov convective part
        lam = cmax(ph.wave_speed(Uf, nrm), ph.wave_speed(Uf_nb, nrm))
        Fr = 0.5 * dotn(ph.conv(Uf) + ph.conv(Uf_nb)) + 0.5 * lam[..., None] * (Uf - Uf_nb)
        if ph.viscous:
            Fh = Fh - dotn(ph.visc(uh, qf))
            Fvfr = 0.5 * dotn(ph.visc(Uf, qf) + ph.visc(Uf_nb, qf_nb))
            imp5 = imp_e[..., None]
            U_im = np.where(imp_e, Uf, Uf_nb)
            q_im = np.where(imp5, qf, qf_nb)
            Fvim = dotn(ph.visc(U_im, q_im))
            Fr_fr = Fr - Fvfr
            Fr_im = Fr - Fvim
        else:
            Fr_fr = Fr
            Fr_im = Fr
        Fhat = np.where(kind == TRACE_FACE, Fh, np.where(kind == IMEX_FACE, Fr_im, Fr_fr))
        Fn = geo.Jf[..., None] * Fhat
        H = Fn - FDn
        dxi, deta = self.ref_derivative(Ft)
        cx, cy = self.lift(H, signed=True)
        div = dxi[:, :, 0] + deta[:, :, 1] + cx + cy
        R = -div / geo.J[:, :, None]
        return R, Fn

    # ------------------------------------------------------------ trace helpers
    def trace_view(self, uhat):
        """Global trace (ntrace, n, nv) -> per element face (E, 4, n, nv); zero
        on faces without a trace."""
        E = self.mesh.nelem
        view = np.zeros((E, 4, self.n, self.nv), dtype=uhat.dtype)
        has = self.tr_of >= 0
        view[has] = uhat[self.tr_of[has]]
        return view

    def trace_weights(self, Fn):
        """Element contribution w_q Fn to the trace residual, zero off trace faces."""
        gv = self.geo.wface[None, None, :, None] * Fn
        return np.where((self.kind == TRACE_FACE)[:, :, None, None], gv, 0.0)

    def assemble_trace(self, gview):
        """Sum element-face contributions (E, 4, n, nv) into the global trace."""
        g = np.zeros((self.ntrace, self.n, self.nv), dtype=gview.dtype)
        for s in range(2):
            e = self.trace_sides[:, s, 0]
            f = self.trace_sides[:, s, 1]
            g += gview[e, f]
        return g

    def initial_trace(self, U):
        """Initial trace guess: average of both sides' interpolated states."""
        Uf = self.interp_faces(U)
        ts = self.trace_sides
        return 0.5 * (Uf[ts[:, 0, 0], ts[:, 0, 1]] + Uf[ts[:, 1, 0], ts[:, 1, 1]])

    def full_residual(self, U, uhat):
        """R (E, Ns, nv) and trace residual g (ntrace, n, nv)."""
        R, Fn = self.residual(U, self.trace_view(uhat))
        return R, self.assemble_trace(self.trace_weights(Fn))
