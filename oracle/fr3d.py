"""FR and hybridized-FR residuals on hexahedra (test infrastructure: plain FP64, only ``tests/``
use it).  The operators of ``oracle.fr`` in three dimensions (Secs. 2, 4; the paper's 3D cases run
the same scheme on hexahedra, Sec. 5.3):

* Gauss solution points in tensor product, pt = a + n b + n^2 c; trilinear map, adjugate metric
  S[r, :] = x_{xi_s} x x_{xi_t} over the cyclic pairs (s, t) of r, F~_r = S[r, :] . F;
* faces 0/1: xi = -1/+1, 2/3: eta, 4/5: zeta; face point m = (first tangential index) + n (second),
  scaled normal N = sigma S[r, :], J_f = |N|, face weights w_s w_t;
* correction functions: the DG-recovering pair spread along each face's normal axis;
* common fluxes, viscous readings, face kinds, trace residual g_q = w_q J_f (F^_+ . n_+ + F^_- . n_-)
  and trace numbering by increasing global face id exactly as in two dimensions.

Boundary faces (walls, far field) follow the readings of ``oracle.boundary`` with the momentum
rows over the three velocity components.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .basis import RefElement1D
from .blocks import EPS
from .boundary import FARFIELD_FACE, WALL_FACE
from .fr import FR_FACE, IMEX_FACE, TRACE_FACE
from .physics import NavierStokes3D, cmax
from .solve import backsolve, condense
from workloads.mesh import BC_FARFIELD, BC_WALL

# (axis, sign) of each local face
FACES_3D = ((0, -1.0), (0, 1.0), (1, -1.0), (1, 1.0), (2, -1.0), (2, 1.0))
_SA = np.array([-1.0, 1, -1, 1, -1, 1, -1, 1])
_SB = np.array([-1.0, -1, 1, 1, -1, -1, 1, 1])
_SC = np.array([-1.0, -1, -1, -1, 1, 1, 1, 1])


def trilinear_derivs(verts, xi, eta, zeta):
    """dx/dxi, dx/deta, dx/dzeta at reference points for every element: (E, P, 3) each."""
    d = [0.125 * _SA[None] * (1 + _SB[None] * eta[:, None]) * (1 + _SC[None] * zeta[:, None]),
         0.125 * _SB[None] * (1 + _SA[None] * xi[:, None]) * (1 + _SC[None] * zeta[:, None]),
         0.125 * _SC[None] * (1 + _SA[None] * xi[:, None]) * (1 + _SB[None] * eta[:, None])]
    return [np.einsum("pk,ekc->epc", dk, verts) for dk in d]


def adjugate3(x_xi, x_eta, x_zeta):
    """Determinant and adjugate S[r, c] = J d xi_r / d x_c of the map's Jacobian."""
    S = np.stack([np.cross(x_eta, x_zeta), np.cross(x_zeta, x_xi), np.cross(x_xi, x_eta)], axis=-2)
    J = np.einsum("...c,...c->...", x_xi, S[..., 0, :])
    return J, S


class Discretisation3D:
    """FR/HFR operators for a hex mesh with a single polynomial degree (periodic, walls, far field)."""

    def __init__(self, mesh, physics, u_inf=None):
        p = int(mesh.p[0])
        if np.any(mesh.p != p):
            raise NotImplementedError("oracle: uniform p only")
        self.mesh, self.phys, self.p = mesh, physics, p
        self.u_inf = None if u_inf is None else np.asarray(u_inf, dtype=np.float64)
        self.ref = RefElement1D(p)
        n = self.n = p + 1
        self.ns, self.nfp = n**3, n**2
        self.nv = physics.nv
        x = self.ref.x
        a, b, c = np.meshgrid(x, x, x, indexing="ij")  # index [a, b, c] -> flatten c-fastest
        xi, eta, zeta = (np.transpose(v, (2, 1, 0)).reshape(-1) for v in (a, b, c))  # pt = a + n b + n^2 c
        self.J, self.S = adjugate3(*trilinear_derivs(mesh.verts, xi, eta, zeta))
        N = 0.125 * (1 + _SA[None] * xi[:, None]) * (1 + _SB[None] * eta[:, None]) * (1 + _SC[None] * zeta[:, None])
        self.xyz = np.einsum("pk,ekc->epc", N, mesh.verts)
        E = mesh.nelem
        s1, s2 = np.tile(x, n), np.repeat(x, n)  # face point m = i + n j
        self.Nf = np.zeros((E, 6, self.nfp, 3))
        for f, (r, sg) in enumerate(FACES_3D):
            ref = [None, None, None]
            ref[r] = np.full(self.nfp, sg)
            t = [ax for ax in range(3) if ax != r]
            ref[t[0]], ref[t[1]] = s1, s2
            _, Sf = adjugate3(*trilinear_derivs(mesh.verts, *ref))
            self.Nf[:, f] = sg * Sf[:, :, r, :]
        self.Jf = np.sqrt(np.sum(self.Nf**2, axis=-1))
        self.normal = self.Nf / self.Jf[..., None]
        self.wface = np.outer(self.ref.w, self.ref.w).reshape(-1)  # [j, i] -> m = i + n j
        self.wvol = np.einsum("c,b,a->cba", *(self.ref.w,) * 3).reshape(-1)
        imp = np.asarray(mesh.implicit, dtype=bool)
        self.imp = imp
        bnd = mesh.nbr < 0
        self.bnd = bnd
        nb = np.where(bnd, 0, mesh.nbr)
        kind = np.full((E, 6), FR_FACE, dtype=np.int32)
        kind[~bnd & imp[:, None] & imp[nb]] = TRACE_FACE
        kind[~bnd & (imp[:, None] != imp[nb])] = IMEX_FACE
        kind[bnd & (mesh.bc == BC_WALL)] = WALL_FACE
        kind[bnd & (mesh.bc == BC_FARFIELD)] = FARFIELD_FACE
        if np.any(bnd & ~np.isin(mesh.bc, (BC_WALL, BC_FARFIELD))):
            raise ValueError("boundary face without a wall or far-field tag")
        if np.any(kind == WALL_FACE) and (np.any((kind == WALL_FACE) & ~imp[:, None])
                                          or not isinstance(physics, NavierStokes3D)):
            raise NotImplementedError("oracle: walls on implicit Navier-Stokes elements only")
        if np.any(kind == FARFIELD_FACE) and self.u_inf is None:
            raise ValueError("far-field faces need u_inf")
        self.kind = kind
        self.traced = (kind == TRACE_FACE) | (bnd & imp[:, None])
        fid = mesh.face_of
        trace_fids = np.unique(fid[self.traced])
        tr_of_fid = -np.ones(mesh.nface, dtype=np.int64)
        tr_of_fid[trace_fids] = np.arange(len(trace_fids))
        self.ntrace = len(trace_fids)
        self.tr_of = np.where(self.traced, tr_of_fid[fid], -1)
        self.trace_sides = -np.ones((self.ntrace, 2, 2), dtype=np.int64)
        for e in range(E):
            for f in range(6):
                t = self.tr_of[e, f]
                if t >= 0:
                    self.trace_sides[t, 0 if self.trace_sides[t, 0, 0] < 0 else 1] = (e, f)
        self.imp_idx = np.nonzero(imp)[0]
        self.ex_idx = np.nonzero(~imp)[0]

    # ------------------------------------------------------------------ helpers
    def _grid(self, X):
        n = self.n
        return X.reshape((X.shape[0], n, n, n) + X.shape[2:])  # [e, c, b, a, ...]

    def interp_faces(self, X):
        """Values at the flux points of every face: (E, Ns, *r) -> (E, 6, n^2, *r)."""
        G = self._grid(X)
        r = self.ref
        E, nfp = X.shape[0], self.nfp
        out = np.empty((E, 6, nfp) + X.shape[2:], dtype=X.dtype)
        for f, (ax, sg) in enumerate(FACES_3D):
            l = r.lp if sg > 0 else r.lm
            if ax == 0:
                v = np.einsum("a,ecba...->ecb...", l, G)
            elif ax == 1:
                v = np.einsum("b,ecba...->eca...", l, G)
            else:
                v = np.einsum("c,ecba...->eba...", l, G)
            out[:, f] = v.reshape((E, nfp) + X.shape[2:])
        return out

    def ref_derivative(self, X):
        """(d/dxi, d/deta, d/dzeta) of X at the solution points."""
        G = self._grid(X)
        D = self.ref.D
        E = X.shape[0]
        shp = (E, self.ns) + X.shape[2:]
        return (np.einsum("ij,ecbj...->ecbi...", D, G).reshape(shp),
                np.einsum("ij,ecja...->ecia...", D, G).reshape(shp),
                np.einsum("ij,ejba...->eiba...", D, G).reshape(shp))

    def lift(self, face_vals, signed):
        """Each face's values spread along its normal axis with the correction derivatives
        (sigma g' when signed, g' otherwise): three arrays (E, Ns, *r), one per axis."""
        r, n = self.ref, self.n
        E = face_vals.shape[0]
        rest = face_vals.shape[3:]
        out = [np.zeros((E, n, n, n) + rest, dtype=face_vals.dtype) for _ in range(3)]
        sl = -1.0 if signed else 1.0
        for f, (ax, sg) in enumerate(FACES_3D):
            coef = r.dgR if sg > 0 else sl * r.dgL
            V = face_vals[:, f].reshape((E, n, n) + rest)  # [e, j, i]
            if ax == 0:
                out[0] += np.einsum("a,ecb...->ecba...", coef, V)
            elif ax == 1:
                out[1] += np.einsum("b,eca...->ecba...", coef, V)
            else:
                out[2] += np.einsum("c,eba...->ecba...", coef, V)
        return [o.reshape((E, self.ns) + rest) for o in out]

    def neighbour(self, Xf):
        """Other side's face values; boundary faces get the element's own values."""
        m = self.mesh
        out = Xf[np.where(self.bnd, 0, m.nbr), np.where(self.bnd, 0, m.nbr_face)]
        return np.where(self.bnd.reshape(self.bnd.shape + (1,) * (Xf.ndim - 2)), Xf, out)

    def _other_state(self, Uf):
        """The neighbour's face state, the ghost u_inf on far-field faces."""
        far = (self.kind == FARFIELD_FACE)[:, :, None, None]
        if not np.any(far):
            return self.neighbour(Uf)
        return np.where(far, np.broadcast_to(self.u_inf, Uf.shape), self.neighbour(Uf))

    # ----------------------------------------------------------------- residual
    def corrected_gradient(self, U, uhat_view):
        """Physical gradient q (E, Ns, 3, nv): reference gradient plus the lifted jumps u_bar - u_f
        (u^ on trace faces, the average on FR faces, the explicit side's state on IMEX faces)."""
        kind = self.kind[:, :, None, None]
        imp_e = self.imp[:, None, None, None]
        Uf = self.interp_faces(U)
        Uf_nb = self._other_state(Uf)
        jump = np.where(self.traced[:, :, None, None], uhat_view - Uf, 0.5 * (Uf_nb - Uf))
        jump = np.where(kind == IMEX_FACE, np.where(imp_e, Uf_nb - Uf, 0.0 * Uf), jump)
        d = self.ref_derivative(U)
        c = self.lift(jump, signed=False)
        Qr = np.stack([d[k] + c[k] for k in range(3)], axis=2)
        return np.einsum("esrc,esrv->escv", self.S, Qr) / self.J[:, :, None, None]

    def residual(self, U, uhat_view):
        """R (E, Ns, nv) and J_f times the element's trace row at every flux point (E, 6, n^2, nv):
        J_f F^.n on interior faces, the wall / far-field rows on boundary faces of implicit
        elements."""
        ph = self.phys
        kind = self.kind[:, :, None, None]
        traced = self.traced[:, :, None, None]
        imp_e = self.imp[:, None, None, None]
        Uf = self.interp_faces(U)
        Uf_nb = self._other_state(Uf)
        if ph.viscous:
            q = self.corrected_gradient(U, uhat_view)
            qf = self.interp_faces(q)
            qf_nb = self.neighbour(qf)
            F = ph.conv(U) - ph.visc(U, q)
        else:
            F = ph.conv(U)
        Ft = np.einsum("esrc,escv->esrv", self.S, F)
        Ftf = self.interp_faces(Ft)
        FDn = np.empty_like(Uf)
        for f, (r, sg) in enumerate(FACES_3D):
            FDn[:, f] = sg * Ftf[:, f, :, r, :]
        nrm = self.normal

        def dotn(Fx):
            return np.einsum("...cv,...c->...v", Fx, nrm)

        uh = np.where(traced, uhat_view, Uf)
        stab = ph.stab(uh, nrm)[..., None]
        Fh = dotn(ph.conv(uh)) + stab * (Uf - uh)
        lam = cmax(ph.wave_speed(Uf, nrm), ph.wave_speed(Uf_nb, nrm))
        Fr = 0.5 * dotn(ph.conv(Uf) + ph.conv(Uf_nb)) + 0.5 * lam[..., None] * (Uf - Uf_nb)
        if ph.viscous:
            Fh = Fh - dotn(ph.visc(uh, qf))
            Fr_fr = Fr - 0.5 * dotn(ph.visc(Uf, qf) + ph.visc(Uf_nb, qf_nb))
            Fr_im = Fr - dotn(ph.visc(np.where(imp_e, Uf, Uf_nb), np.where(imp_e[..., None], qf, qf_nb)))
        else:
            Fr_fr = Fr_im = Fr
        Fhat = np.where(traced, Fh, np.where(kind == IMEX_FACE, Fr_im, Fr_fr))
        Jf = self.Jf[..., None]
        Fn = Jf * Fhat
        d = self.ref_derivative(Ft)
        c = self.lift(Fn - FDn, signed=True)
        div = d[0][:, :, 0] + d[1][:, :, 1] + d[2][:, :, 2] + c[0] + c[1] + c[2]
        G = Fn
        if np.any(kind == FARFIELD_FACE):
            G = np.where(kind == FARFIELD_FACE, Jf * stab * ((Uf - uh) + (self.u_inf - uh)), G)
        if np.any(kind == WALL_FACE):
            wall = Jf * np.concatenate([Fh[..., :1], stab * uh[..., 1:4], Fh[..., 4:]], axis=-1)
            G = np.where(kind == WALL_FACE, wall, G)
        return -div / self.J[:, :, None], G

    # ------------------------------------------------------------ trace helpers
    def trace_view(self, uhat):
        view = np.zeros((self.mesh.nelem, 6, self.nfp, self.nv), dtype=uhat.dtype)
        has = self.tr_of >= 0
        view[has] = uhat[self.tr_of[has]]
        return view

    def trace_weights(self, Fn):
        gv = self.wface[None, None, :, None] * Fn
        return np.where(self.traced[:, :, None, None], gv, 0.0)

    def assemble_trace(self, gview):
        g = np.zeros((self.ntrace, self.nfp, self.nv), dtype=gview.dtype)
        for s in range(2):
            ok = self.trace_sides[:, s, 0] >= 0
            g[ok] += gview[self.trace_sides[ok, s, 0], self.trace_sides[ok, s, 1]]
        return g

    def initial_trace(self, U):
        """Average of both sides' states; with u_inf on far-field faces; on walls the element's
        density and energy with zero momentum."""
        Uf = self.interp_faces(U)
        out = np.zeros((self.ntrace, self.nfp, self.nv))
        for t in range(self.ntrace):
            (e0, f0), (e1, f1) = self.trace_sides[t]
            if e1 >= 0:
                out[t] = 0.5 * (Uf[e0, f0] + Uf[e1, f1])
            elif self.kind[e0, f0] == FARFIELD_FACE:
                out[t] = 0.5 * (Uf[e0, f0] + self.u_inf)
            else:
                out[t] = Uf[e0, f0]
                out[t, :, 1:4] = 0.0
        return out

    def full_residual(self, U, uhat):
        R, Fn = self.residual(U, self.trace_view(uhat))
        return R, self.assemble_trace(self.trace_weights(Fn))


def element_blocks_3d(d, U, uhat, a_dt):
    """A, B, C, D of every element by complex-step differentiation (as ``oracle.blocks``): element
    unknown i = pt nv + v, element trace unknown l = (f n^2 + m) nv + v over the six faces."""
    E, nv = d.mesh.nelem, d.nv
    nA, nT = d.ns * nv, 6 * d.nfp * nv
    Uc = U.astype(np.complex128)
    Vc = d.trace_view(uhat).astype(np.complex128)
    imp = d.imp
    A, B = np.zeros((E, nA, nA)), np.zeros((E, nA, nT))
    C, D = np.zeros((E, nT, nA)), np.zeros((E, nT, nT))
    for j in range(nA):
        Up = Uc.copy()
        Up.reshape(E, nA)[imp, j] += 1j * EPS
        R, Fn = d.residual(Up, Vc)
        A[:, :, j] = -a_dt * R.imag.reshape(E, nA) / EPS
        C[:, :, j] = d.trace_weights(Fn).imag.reshape(E, nT) / EPS
    for l in range(nT):
        Vp = Vc.copy()
        Vp.reshape(E, nT)[imp, l] += 1j * EPS
        R, Fn = d.residual(Uc, Vp)
        B[:, :, l] = -a_dt * R.imag.reshape(E, nA) / EPS
        D[:, :, l] = d.trace_weights(Fn).imag.reshape(E, nT) / EPS
    A += np.eye(nA)[None]
    return A, B, C, D


def condensed_newton_step(d, U, uhat, Ustar, a_dt):
    """One Newton step of the stage equations by static condensation (Sec. 3.2) with a direct
    sparse trace solve: (dU (E, Ns, nv), duhat (ntrace, n^2, nv))."""
    imp = d.imp_idx
    nv, nfp = d.nv, d.nfp
    nA, nT = d.ns * nv, 6 * nfp * nv
    R, Fn = d.residual(U, d.trace_view(uhat))
    gv = d.trace_weights(Fn)
    h = U[imp] - Ustar[imp] - a_dt * R[imp]
    A, B, C, D = element_blocks_3d(d, U, uhat, a_dt)
    XB, xr, S, t = condense(A[imp], B[imp], C[imp], D[imp], -h.reshape(-1, nA), -gv[imp].reshape(-1, nT))
    tr = d.tr_of[imp]  # (Ei, 6)
    idx = (tr[:, :, None, None] * nfp + np.arange(nfp)[:, None]) * nv + np.arange(nv)
    idx = np.where(tr[:, :, None, None] >= 0, idx, -1).reshape(len(imp), nT)
    N = d.ntrace * nfp * nv
    rows = np.repeat(idx[:, :, None], nT, axis=2)
    cols = np.repeat(idx[:, None, :], nT, axis=1)
    ok = (rows >= 0) & (cols >= 0)
    L = sp.coo_matrix((S[ok], (rows[ok], cols[ok])), shape=(N, N)).tocsc()
    rhs = np.zeros(N)
    np.add.at(rhs, idx[idx >= 0], t[idx >= 0])
    duh = spla.spsolve(L, rhs).reshape(d.ntrace, nfp, nv)
    du = backsolve(XB, xr, d.trace_view(duh)[imp].reshape(len(imp), nT))
    dU = np.zeros_like(U)
    dU[imp] = du.reshape(len(imp), d.ns, nv)
    return dU, duh


def monolithic_newton_step(d, U, uhat, Ustar, a_dt):
    """The same step from the dense Jacobian of [h; g] in [u_implicit; u^] (tiny meshes)."""
    imp = d.imp_idx
    nA = d.ns * d.nv
    nu, nh = len(imp) * nA, uhat.size
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
    x = np.linalg.solve(Jm, -np.concatenate([(U[imp] - Ustar[imp] - a_dt * R[imp]).reshape(-1), g.reshape(-1)]))
    dU = np.zeros_like(U)
    dU[imp] = x[:nu].reshape(len(imp), d.ns, d.nv)
    return dU, x[nu:].reshape(uhat.shape)
