"""FR and hybridized-FR residuals on a quadrilateral mesh whose elements carry different
polynomial degrees (test infrastructure: plain FP64, element by element; only ``tests/`` use it).

The paper's element blocks accommodate faces with different numbers of trace points (Sec. 3.2,
p-adaptive meshes) but it writes no operator for them.  Reading used here, which reduces to the
uniform-degree operator of ``oracle.fr`` when all degrees agree:

* every face carries the Gauss points of the higher of its two elements' degrees,
  n_f = max(p-, p+) + 1; both sides evaluate their interpolated state, discontinuous flux and
  gradient at those points, and the common fluxes, the trace unknowns (hybridized faces) and the
  trace residual g_q = w_q J_f (F^_+ . n_+ + F^_- . n_-) live there;
* an element lifts a face jump h (flux jump H, or solution jump for the gradient) from the face
  points onto its own face nodes by the L2 projection with the face Gauss rule,
  (P h)_b = sum_q w_q l_b(s_q) h_q / w_b, exact for face polynomials of the element's degree, and
  spreads it with its DG-recovering correction derivatives along the face normal: the nodal-DG
  lift of the jump, the identity projection when n_f equals the element's point count;
* the discontinuous flux at a face point is the element's flux polynomial there (interpolation of
  the transformed flux from its solution points), as in the uniform operator.

Face kinds, common fluxes and viscous readings are those of ``oracle.fr``; boundary faces (walls,
far field) follow ``oracle.boundary``: a boundary face carries the element's own point count, a
trace when its element is implicit, and the wall / far-field trace rows there.
"""

from __future__ import annotations

import numpy as np

from .basis import RefElement1D, gauss_legendre, lagrange
from .boundary import FARFIELD_FACE, WALL_FACE
from .fr import FR_FACE, IMEX_FACE, TRACE_FACE
from .geometry import FACES_2D, _adjugate, _bilinear_derivs
from .physics import NavierStokes2D, cmax
from workloads.mesh import BC_FARFIELD, BC_WALL


class MixedDiscretisation:
    """FR/HFR operators element by element for a quad mesh with per-element degrees."""

    def __init__(self, mesh, physics, u_inf=None):
        self.mesh = mesh
        self.phys = physics
        self.nv = physics.nv
        self.u_inf = None if u_inf is None else np.asarray(u_inf, dtype=np.float64)
        E = mesh.nelem
        self.E = E
        self.p = np.asarray(mesh.p, dtype=np.int64)
        self.n = self.p + 1
        self.refs = {int(p): RefElement1D(int(p)) for p in np.unique(self.p)}
        imp = np.asarray(mesh.implicit, dtype=bool)
        self.imp = imp
        bnd = mesh.nbr < 0
        self.bnd = bnd
        nbr = np.where(bnd, np.arange(E)[:, None], mesh.nbr)  # boundary faces point at themselves
        kind = np.full((E, 4), FR_FACE, dtype=np.int32)
        kind[~bnd & imp[:, None] & imp[nbr]] = TRACE_FACE
        kind[~bnd & (imp[:, None] != imp[nbr])] = IMEX_FACE
        kind[bnd & (mesh.bc == BC_WALL)] = WALL_FACE
        kind[bnd & (mesh.bc == BC_FARFIELD)] = FARFIELD_FACE
        if np.any(bnd & ~np.isin(mesh.bc, (BC_WALL, BC_FARFIELD))):
            raise ValueError("boundary face without a wall or far-field tag")
        if np.any(kind == WALL_FACE) and (np.any((kind == WALL_FACE) & ~imp[:, None])
                                          or not isinstance(physics, NavierStokes2D)):
            raise NotImplementedError("oracle: walls on implicit Navier-Stokes elements only")
        if np.any(kind == FARFIELD_FACE) and self.u_inf is None:
            raise ValueError("far-field faces need u_inf")
        self.kind = kind
        self.traced = (kind == TRACE_FACE) | (bnd & imp[:, None])
        # face point count: the higher degree of the two sides (the own one on boundaries)
        self.nf = np.maximum(self.n[:, None], self.n[nbr])  # (E, 4)
        self.rule = {int(m): gauss_legendre(int(m)) for m in np.unique(self.nf)}
        # trace numbering as in oracle.fr: faces with a trace in increasing global face id
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
        self.trace_npts = np.array([self.nf[e, f] for e, f in self.trace_sides[:, 0]], dtype=np.int64)
        self._geometry()
        self._face_operators()

    # ------------------------------------------------------------------ set-up
    def _geometry(self):
        """Metrics at each element's solution points and at the points of each of its faces
        (the bilinear map of oracle.geometry evaluated element by element)."""
        verts = self.mesh.verts
        self.J, self.S = [], []
        self.Jf, self.normal = {}, {}
        for e in range(self.E):
            r = self.refs[int(self.p[e])]
            xi, eta = np.tile(r.x, r.n), np.repeat(r.x, r.n)
            a, b = _bilinear_derivs(verts[e:e + 1], xi, eta)
            J, S = _adjugate(a, b)
            self.J.append(J[0])
            self.S.append(S[0])
            for f, (ax, sg) in enumerate(FACES_2D):
                s = self.rule[int(self.nf[e, f])][0]
                fx, fe = (np.full(len(s), sg), s) if ax == 0 else (s, np.full(len(s), sg))
                a, b = _bilinear_derivs(verts[e:e + 1], fx, fe)
                _, Sf = _adjugate(a, b)
                N = sg * Sf[0, :, ax, :]
                Jf = np.sqrt(np.sum(N**2, axis=-1))
                self.Jf[e, f] = Jf
                self.normal[e, f] = N / Jf[:, None]

    def _face_operators(self):
        """T[n, m]: element nodes (n) -> face points (m), T[q, b] = l_b(s_q);
        P[n, m]: face points -> element nodes, the L2 projection with the face Gauss rule."""
        self.T, self.P = {}, {}
        for e in range(self.E):
            r = self.refs[int(self.p[e])]
            for f in range(4):
                m = int(self.nf[e, f])
                if (r.n, m) in self.T:
                    continue
                s, w = self.rule[m]
                T = lagrange(r.x, s)
                self.T[r.n, m] = T
                self.P[r.n, m] = (w[:, None] * T).T / r.w[:, None]

    # ------------------------------------------------------------------ element operators
    def _grid(self, e, X):
        n = int(self.n[e])
        return X.reshape((n, n) + X.shape[1:])

    def to_face(self, e, f, X):
        """Element field at its solution points (Ns, ...) -> values at the points of face f."""
        r = self.refs[int(self.p[e])]
        G = self._grid(e, X)
        ax, sg = FACES_2D[f]
        c = r.lp if sg > 0 else r.lm
        line = np.einsum("a,ba...->b...", c, G) if ax == 0 else np.einsum("b,ba...->a...", c, G)
        return np.einsum("qb,b...->q...", self.T[r.n, int(self.nf[e, f])], line)

    def ref_derivative(self, e, X):
        r = self.refs[int(self.p[e])]
        G = self._grid(e, X)
        dxi = np.einsum("ij,bj...->bi...", r.D, G)
        deta = np.einsum("ij,j...->i...", r.D, G)
        ns = r.n * r.n
        return dxi.reshape((ns,) + X.shape[1:]), deta.reshape((ns,) + X.shape[1:])

    def lift(self, e, face_vals, signed):
        """The four faces' jumps (each at its face points) projected onto the element's face
        nodes and spread along the face normals with the correction derivatives: the xi-part and
        eta-part (Ns, ...), as oracle.fr.Discretisation.lift."""
        r = self.refs[int(self.p[e])]
        rest = face_vals[0].shape[1:]
        cx = np.zeros((r.n, r.n) + rest, dtype=np.result_type(*face_vals))
        cy = np.zeros_like(cx)
        sl = -1.0 if signed else 1.0
        for f, (ax, sg) in enumerate(FACES_2D):
            hp = np.einsum("bq,q...->b...", self.P[r.n, int(self.nf[e, f])], face_vals[f])
            coef = r.dgR if sg > 0 else sl * r.dgL
            if ax == 0:
                cx += np.einsum("a,b...->ba...", coef, hp)
            else:
                cy += np.einsum("b,a...->ba...", coef, hp)
        ns = r.n * r.n
        return cx.reshape((ns,) + rest), cy.reshape((ns,) + rest)

    # ------------------------------------------------------------------ residual
    def residual(self, U, uhat):
        """R(u, u^) and J_f times the element's trace row at every element face point: its normal
        flux J_f F^.n on interior faces, the wall / far-field rows of ``oracle.boundary`` on
        boundary faces of implicit elements.

        U: list of (Ns_e, nv) arrays; uhat: list over trace faces of (n_f, nv) arrays.
        Returns R (list of (Ns_e, nv)) and Fn (list over elements of 4 arrays (n_f, nv))."""
        ph = self.phys
        m = self.mesh
        E = self.E
        Uf = [[self.to_face(e, f, U[e]) for f in range(4)] for e in range(E)]

        def other_state(e, f):
            """The other side's state at the face points: the neighbour's, u_inf on far field."""
            if self.kind[e, f] == FARFIELD_FACE:
                return np.broadcast_to(self.u_inf, Uf[e][f].shape)
            return Uf[m.nbr[e, f]][m.nbr_face[e, f]]

        def face_trace(e, f):
            return uhat[self.tr_of[e, f]]

        if ph.viscous:
            q, qf = [], []
            for e in range(E):
                jumps = []
                for f in range(4):
                    k = self.kind[e, f]
                    if self.traced[e, f]:
                        ubar = face_trace(e, f)
                    elif k == IMEX_FACE:
                        ubar = other_state(e, f) if self.imp[e] else Uf[e][f]
                    else:
                        ubar = 0.5 * (Uf[e][f] + other_state(e, f))
                    jumps.append(ubar - Uf[e][f])
                dxi, deta = self.ref_derivative(e, U[e])
                cx, cy = self.lift(e, jumps, signed=False)
                Qr = np.stack([dxi + cx, deta + cy], axis=1)  # (Ns, 2, nv) reference gradient
                qe = np.einsum("src,srv->scv", self.S[e], Qr) / self.J[e][:, None, None]
                q.append(qe)
                qf.append([self.to_face(e, f, qe) for f in range(4)])

        def other_grad(e, f):
            """The other side's gradient: the neighbour's, the element's own on boundary faces."""
            return qf[e][f] if self.bnd[e, f] else qf[m.nbr[e, f]][m.nbr_face[e, f]]

        R, Fn = [], []
        for e in range(E):
            F = ph.conv(U[e]) - ph.visc(U[e], q[e]) if ph.viscous else ph.conv(U[e])
            Ft = np.einsum("src,scv->srv", self.S[e], F)  # transformed flux
            Fn_e, H = [], []
            for f, (ax, sg) in enumerate(FACES_2D):
                nrm = self.normal[e, f]
                Jf = self.Jf[e, f][:, None]

                def dotn(Fx):
                    return np.einsum("qcv,qc->qv", Fx, nrm)

                uf = Uf[e][f]
                k = self.kind[e, f]
                if self.traced[e, f]:
                    uh = face_trace(e, f)
                    s = ph.stab(uh, nrm)[:, None]
                    Fhat = dotn(ph.conv(uh)) + s * (uf - uh)
                    if ph.viscous:
                        Fhat = Fhat - dotn(ph.visc(uh, qf[e][f]))
                    if k == FARFIELD_FACE:
                        row = Jf * s * ((uf - uh) + (self.u_inf - uh))
                    elif k == WALL_FACE:
                        row = Jf * np.concatenate([Fhat[:, :1], s * uh[:, 1:3], Fhat[:, 3:]], axis=1)
                    else:
                        row = Jf * Fhat
                else:
                    un = other_state(e, f)
                    lam = cmax(ph.wave_speed(uf, nrm), ph.wave_speed(un, nrm))
                    Fhat = 0.5 * dotn(ph.conv(uf) + ph.conv(un)) + 0.5 * lam[:, None] * (uf - un)
                    if ph.viscous:
                        qn = other_grad(e, f)
                        if k == IMEX_FACE:
                            u_im, q_im = (uf, qf[e][f]) if self.imp[e] else (un, qn)
                            Fhat = Fhat - dotn(ph.visc(u_im, q_im))
                        else:
                            Fhat = Fhat - 0.5 * dotn(ph.visc(uf, qf[e][f]) + ph.visc(un, qn))
                    row = Jf * Fhat
                FDn = sg * self.to_face(e, f, Ft)[:, ax, :]
                Fn_e.append(row)
                H.append(Jf * Fhat - FDn)
            dxi, _ = self.ref_derivative(e, Ft[:, 0])
            _, deta = self.ref_derivative(e, Ft[:, 1])
            cx, cy = self.lift(e, H, signed=True)
            R.append(-(dxi + deta + cx + cy) / self.J[e][:, None])
            Fn.append(Fn_e)
        return R, Fn

    # ------------------------------------------------------------------ trace
    def trace_residual(self, Fn):
        """g_q = w_q (J_f F^.n)_+ + w_q (J_f F^.n)_- at the points of every trace face."""
        g = []
        for t in range(self.ntrace):
            w = self.rule[int(self.trace_npts[t])][1]
            acc = 0.0
            for s in range(2):
                e, f = self.trace_sides[t, s]
                if e >= 0:
                    acc = acc + w[:, None] * Fn[e][f]
            g.append(acc)
        return g

    def initial_trace(self, U):
        """Average of both sides' interpolated states at each trace face's points (boundary faces as
        in ``oracle.boundary``)."""
        out = []
        for t in range(self.ntrace):
            (e0, f0), (e1, f1) = self.trace_sides[t]
            u0 = self.to_face(e0, f0, U[e0])
            if e1 >= 0:
                out.append(0.5 * (u0 + self.to_face(e1, f1, U[e1])))
            elif self.kind[e0, f0] == FARFIELD_FACE:
                out.append(0.5 * (u0 + self.u_inf))
            else:  # wall: the element's density and energy, no momentum
                u0 = u0.copy()
                u0[:, 1:3] = 0.0
                out.append(u0)
        return out

    def full_residual(self, U, uhat):
        R, Fn = self.residual(U, uhat)
        return R, self.trace_residual(Fn)
