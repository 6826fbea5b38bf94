"""FR / HFR residual with boundary faces: no-slip adiabatic walls and far field (test
infrastructure: plain FP64, only ``tests/`` use it).

The paper's transmission conditions carry a boundary term, w_q J_f (F^.n - F^BC) on boundary faces,
with F^BC only called the normal boundary flux (Sec. 2.2, eq. hfr2); hybridized boundaries carry
a discontinuous trace (Sec. 2.2, EFR too).  Readings used here (uniform degree, quads):

* every boundary face of an implicit element carries a trace, numbered with the interior trace
  faces by increasing global face id; the element sees it as on any trace face (one-sided flux
  F^ = F(u^) + s (u_f - u^) n - F^v(u^, q_f), gradient jump u^ - u_f);
* far field: F^BC is the one-sided flux of a ghost element holding the free stream u_inf and the
  element's own gradient, seen with the opposite normal, so the boundary row is
  g_q = w_q J_f s(u^) ((u_f - u^) + (u_inf - u^)): the trace is the average of u_f and u_inf, the
  far-field counterpart of the interior condition;
* no-slip adiabatic wall (Navier-Stokes): the momentum rows set the trace velocity to zero,
  g_q = w_q J_f s(u^) (rho v)^; the mass and energy rows are the element's own normal fluxes,
  g_q = w_q J_f (F^.n)_rho, w_q J_f (F^.n)_E: no mass through the wall and no energy flux (heat flux
  balanced weakly by the stabilisation), which fixes rho^ = rho_f and the wall energy;
* explicit elements on a far-field face use the FR Rusanov flux against the ghost state u_inf
  (BR1 common solution the average of u_f and u_inf, viscous flux the average of both sides' with
  the element's own gradient); explicit elements on a wall are not supported.
"""

from __future__ import annotations

import numpy as np

from .basis import RefElement1D
from .fr import Discretisation, FR_FACE, IMEX_FACE, TRACE_FACE
from .geometry import FACES_2D, QuadGeometry
from .physics import NavierStokes2D, cmax
from workloads.mesh import BC_FARFIELD, BC_WALL

WALL_FACE = 3
FARFIELD_FACE = 4


class BoundaryDiscretisation(Discretisation):
    """FR/HFR operators for a quad mesh of uniform degree with wall and far-field faces."""

    def __init__(self, mesh, physics, u_inf=None):
        p = int(mesh.p[0])
        if np.any(mesh.p != p):
            raise NotImplementedError("oracle: uniform p only")
        self.mesh = mesh
        self.phys = physics
        self.p = p
        self.ref = RefElement1D(p)
        self.n = p + 1
        self.ns = self.n**2
        self.nv = physics.nv
        self.geo = QuadGeometry(mesh.verts, self.ref)
        self.u_inf = None if u_inf is None else np.asarray(u_inf, dtype=np.float64)
        E = mesh.nelem
        imp = np.asarray(mesh.implicit, dtype=bool)
        self.imp = imp
        bnd = mesh.nbr < 0
        nb = np.where(bnd, 0, mesh.nbr)
        kind = np.full((E, 4), FR_FACE, dtype=np.int32)
        kind[~bnd & imp[:, None] & imp[nb]] = TRACE_FACE
        kind[~bnd & (imp[:, None] != imp[nb])] = IMEX_FACE
        kind[bnd & (mesh.bc == BC_WALL)] = WALL_FACE
        kind[bnd & (mesh.bc == BC_FARFIELD)] = FARFIELD_FACE
        if np.any(bnd & ~np.isin(mesh.bc, (BC_WALL, BC_FARFIELD))):
            raise ValueError("boundary face without a wall or far-field tag")
        if np.any((kind == WALL_FACE) & ~imp[:, None]):
            raise NotImplementedError("oracle: walls on explicit elements")
        if np.any(kind == WALL_FACE) and not isinstance(physics, NavierStokes2D):
            raise NotImplementedError("oracle: walls for Navier-Stokes only")
        if np.any(kind == FARFIELD_FACE) and self.u_inf is None:
            raise ValueError("far-field faces need u_inf")
        self.kind = kind
        self.bnd = bnd
        # faces with a trace: interior trace faces and the boundary faces of implicit elements
        self.traced = (kind == TRACE_FACE) | (bnd & imp[:, None])
        fid = mesh.face_of
        trace_fids = np.unique(fid[self.traced])
        tr_of_fid = -np.ones(mesh.nface, dtype=np.int64)
        tr_of_fid[trace_fids] = np.arange(len(trace_fids))
        self.ntrace = len(trace_fids)
        self.tr_of = np.where(self.traced, tr_of_fid[fid], -1)
        self.trace_sides = -np.ones((self.ntrace, 2, 2), dtype=np.int64)
        for e in range(E):
            for f in range(4):
                t = self.tr_of[e, f]
                if t >= 0:
                    s = 0 if self.trace_sides[t, 0, 0] < 0 else 1
                    self.trace_sides[t, s] = (e, f)
        self.imp_idx = np.nonzero(imp)[0]
        self.ex_idx = np.nonzero(~imp)[0]

    def neighbour(self, Xf):
        """Other side's face values; the boundary faces get the element's own values (callers
        replace them where a ghost state applies)."""
        m = self.mesh
        out = Xf[np.where(self.bnd, 0, m.nbr), np.where(self.bnd, 0, m.nbr_face)]
        bnd = self.bnd.reshape(self.bnd.shape + (1,) * (Xf.ndim - 2))
        return np.where(bnd, Xf, out)

    def _other_state(self, Uf):
        """The other side's face state: the neighbour's, u_inf on far-field faces (the ghost
        state; wall faces always carry a trace)."""
        far = (self.kind == FARFIELD_FACE)[:, :, None, None]
        if self.u_inf is None:
            return self.neighbour(Uf)
        return np.where(far, np.broadcast_to(self.u_inf, Uf.shape), self.neighbour(Uf))

    def corrected_gradient(self, U, uhat_view):
        """Physical gradient q (E, Ns, 2, nv) with the lifted jumps u_bar - u_f: u_bar = u^ on every
        face with a trace (boundary faces of implicit elements included), the average with the
        other side (the ghost u_inf on far-field faces) on FR faces, the explicit side's state on
        IMEX-interface faces."""
        geo = self.geo
        kind = self.kind[:, :, None, None]
        imp_e = self.imp[:, None, None, None]
        Uf = self.interp_faces(U)
        Uf_nb = self._other_state(Uf)
        jump = np.where(self.traced[:, :, None, None], uhat_view - Uf, 0.5 * (Uf_nb - Uf))
        jump = np.where(kind == IMEX_FACE, np.where(imp_e, Uf_nb - Uf, 0.0 * Uf), jump)
        dxi, deta = self.ref_derivative(U)
        cx, cy = self.lift(jump, signed=False)
        Qr = np.stack([dxi + cx, deta + cy], axis=2)
        return np.einsum("esrc,esrv->escv", geo.S, Qr) / geo.J[:, :, None, None]

    # ----------------------------------------------------------------- residual
    def residual(self, U, uhat_view):
        """R(u, u^) (E, Ns, nv) and J_f times the element's trace row at every face point
        (E, 4, n, nv): its normal flux on interior trace faces, the boundary rows above on
        boundary faces of implicit elements, unused elsewhere."""
        ph, geo = self.phys, self.geo
        kind = self.kind[:, :, None, None]
        traced = self.traced[:, :, None, None]
        far = kind == FARFIELD_FACE
        imp_e = self.imp[:, None, None, None]
        Uf = self.interp_faces(U)
        Uf_nb = self._other_state(Uf)
        if ph.viscous:
            q = self.corrected_gradient(U, uhat_view)
            qf = self.interp_faces(q)
            qf_nb = self.neighbour(qf)  # the element's own gradient on boundary faces
            F = ph.conv(U) - ph.visc(U, q)
        else:
            F = ph.conv(U)
        Ft = np.einsum("esrc,escv->esrv", geo.S, F)
        Ftf = self.interp_faces(Ft)
        FDn = np.empty_like(Uf)
        for f, (r, sg) in enumerate(FACES_2D):
            FDn[:, f] = sg * Ftf[:, f, :, r, :]
        nrm = geo.normal

        def dotn(Fx):
            return np.einsum("...cv,...c->...v", Fx, nrm)

        lam = cmax(ph.wave_speed(Uf, nrm), ph.wave_speed(Uf_nb, nrm))
        Fr = 0.5 * dotn(ph.conv(Uf) + ph.conv(Uf_nb)) + 0.5 * lam[..., None] * (Uf - Uf_nb)
        if ph.viscous:
            Fr_fr = Fr - 0.5 * dotn(ph.visc(Uf, qf) + ph.visc(Uf_nb, qf_nb))
            U_im = np.where(imp_e, Uf, Uf_nb)
            q_im = np.where(imp_e[..., None], qf, qf_nb)
            Fr_im = Fr - dotn(ph.visc(U_im, q_im))
        else:
            Fr_fr = Fr_im = Fr
        uh = np.where(traced, uhat_view, Uf)
        s = ph.stab(uh, nrm)[..., None]
        Fh = dotn(ph.conv(uh)) + s * (Uf - uh)
        if ph.viscous:
            Fh = Fh - dotn(ph.visc(uh, qf))
        Fhat = np.where(traced, Fh, np.where(kind == IMEX_FACE, Fr_im, Fr_fr))
        Jf = geo.Jf[..., None]
        Fn = Jf * Fhat
        dxi, deta = self.ref_derivative(Ft)
        cx, cy = self.lift(Fn - FDn, signed=True)
        R = -(dxi[:, :, 0] + deta[:, :, 1] + cx + cy) / geo.J[:, :, None]
        # trace rows
        G = Fn if self.u_inf is None else np.where(far, Jf * s * ((Uf - uh) + (self.u_inf - uh)), Fn)
        if self.nv == 4:
            wall = Jf * np.concatenate([Fh[..., :1], s * uh[..., 1:3], Fh[..., 3:]], axis=-1)
            G = np.where(kind == WALL_FACE, wall, G)
        return R, G

    def assemble_trace(self, gview):
        """Sum the element-face contributions into the global trace (one side on boundaries)."""
        g = np.zeros((self.ntrace, self.n, self.nv), dtype=gview.dtype)
        for s in range(2):
            ok = self.trace_sides[:, s, 0] >= 0
            e, f = self.trace_sides[ok, s, 0], self.trace_sides[ok, s, 1]
            g[ok] += gview[e, f]
        return g

    def trace_weights(self, Fn):
        gv = self.geo.wface[None, None, :, None] * Fn
        return np.where(self.traced[:, :, None, None], gv, 0.0)

    def initial_trace(self, U):
        """Average of both sides' states on interior faces; on far-field faces the average with
        u_inf; on walls the element's density and energy with zero momentum."""
        Uf = self.interp_faces(U)
        out = np.zeros((self.ntrace, self.n, self.nv))
        for t in range(self.ntrace):
            (e0, f0), (e1, f1) = self.trace_sides[t]
            if e1 >= 0:
                out[t] = 0.5 * (Uf[e0, f0] + Uf[e1, f1])
            elif self.kind[e0, f0] == FARFIELD_FACE:
                out[t] = 0.5 * (Uf[e0, f0] + self.u_inf)
            else:
                out[t] = Uf[e0, f0]
                out[t, :, 1:3] = 0.0
        return out
