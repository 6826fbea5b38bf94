"""Element blocks and the hybridized Newton step on meshes of mixed degrees (test infrastructure).

Blocks as in ``oracle.blocks`` (Sec. 3.2, eqs. elemA, elemsystem, elemsystemB), by complex-step
differentiation of ``oracle.fr_mixed``: for implicit element k with nA_k = (p_k + 1)^2 nv unknowns
and nT_k = sum_f n_f nv trace unknowns (face f's n_f points, faces in local order, then point,
then variable; rows and columns of faces without a trace are zero),

    A_k = I - a dt dR_k/du_k,  B_k = -a dt dR_k/du^_k,  C_k = dg^k/du_k,  D_k = dg^k/du^_k.

The hybridized step (Sec. 3.2, eqs. assembly, assembly2, localproblems) condenses each element,
S_k = D_k - C_k A_k^{-1} B_k and t_k = s_k - C_k A_k^{-1} r_k, assembles the trace system from the
element-face blocks, solves it directly and back-substitutes; on tiny meshes it is compared with
the monolithic Newton step on [u; u^].
"""

from __future__ import annotations

import numpy as np

EPS = 1.0e-30


def trace_offsets(m):
    """Offset of each trace face's unknowns (points x variables) in the global trace vector."""
    sizes = [int(k) * m.nv for k in m.trace_npts]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def trace_unflatten(m, vec):
    off = trace_offsets(m)
    return [vec[off[t]:off[t + 1]].reshape(int(m.trace_npts[t]), m.nv) for t in range(m.ntrace)]


def trace_flatten(gs):
    return np.concatenate([g.reshape(-1) for g in gs]) if gs else np.zeros(0)


def _elem_trace_layout(m, e):
    """(face, trace face or -1, points, offset) of element e's trace unknowns."""
    out, o = [], 0
    for f in range(4):
        k = int(m.nf[e, f])
        t = int(m.tr_of[e, f])
        out.append((f, t, k, o))
        o += k * m.nv
    return out, o


def _elem_g(m, e, Fn):
    """Element e's contribution w_q J_f F^.n to the trace residual, its own layout."""
    layout, nT = _elem_trace_layout(m, e)
    g = np.zeros(nT, dtype=Fn[e][0].dtype)
    for f, t, k, o in layout:
        if t >= 0:
            w = m.rule[k][1]
            g[o:o + k * m.nv] = (w[:, None] * Fn[e][f]).reshape(-1)
    return g


def element_blocks_mixed(m, U, uhat, a_dt: float):
    """{k: (A, B, C, D)} for every implicit element k."""
    Uc = [u.astype(np.complex128) for u in U]
    Hc = [h.astype(np.complex128) for h in uhat]
    out = {}
    for e in np.nonzero(m.imp)[0]:
        nA = U[e].size
        layout, nT = _elem_trace_layout(m, e)
        A = np.zeros((nA, nA))
        B = np.zeros((nA, nT))
        C = np.zeros((nT, nA))
        D = np.zeros((nT, nT))
        for j in range(nA):
            Up = list(Uc)
            Up[e] = Uc[e].copy()
            Up[e].reshape(-1)[j] += 1j * EPS
            R, Fn = m.residual(Up, Hc)
            A[:, j] = -a_dt * R[e].imag.reshape(-1) / EPS
            C[:, j] = _elem_g(m, e, Fn).imag / EPS
        A += np.eye(nA)
        for f, t, k, o in layout:
            if t < 0:
                continue
            for l in range(k * m.nv):
                Hp = list(Hc)
                Hp[t] = Hc[t].copy()
                Hp[t].reshape(-1)[l] += 1j * EPS
                R, Fn = m.residual(Uc, Hp)
                B[:, o + l] = -a_dt * R[e].imag.reshape(-1) / EPS
                D[:, o + l] = _elem_g(m, e, Fn).imag / EPS
        out[int(e)] = (A, B, C, D)
    return out


def stage_residual(m, U, uhat, Ustar, a_dt: float):
    """h_k = u_k - u*_k - a dt R_k (implicit elements) and the trace residual g."""
    R, g = m.full_residual(U, uhat)
    h = {int(e): (U[e] - Ustar[e] - a_dt * R[e]).reshape(-1) for e in np.nonzero(m.imp)[0]}
    return h, trace_flatten(g)


def hybridized_step(m, U, uhat, Ustar, a_dt: float):
    """One Newton step by static condensation: (du per implicit element, du^ flat)."""
    blocks = element_blocks_mixed(m, U, uhat, a_dt)
    h, g = stage_residual(m, U, uhat, Ustar, a_dt)
    off = trace_offsets(m)
    L = np.zeros((off[-1], off[-1]))
    t_glob = -g.copy()  # s = -g: the global trace right-hand side
    X = {}
    for e, (A, B, C, D) in blocks.items():
        r = -h[e]
        XB = np.linalg.solve(A, B)
        xr = np.linalg.solve(A, r)
        S = D - C @ XB
        X[e] = (XB, xr)
        layout, _ = _elem_trace_layout(m, e)
        # t_k = s_k - C_k x_r; s_k is already in t_glob through -g (the sum of the elements' g^k)
        tk = -(C @ xr)
        for f, t, k, o in layout:
            if t < 0:
                continue
            rows = slice(off[t], off[t + 1])
            t_glob[rows] += tk[o:o + k * m.nv]
            for f2, t2, k2, o2 in layout:
                if t2 < 0:
                    continue
                L[rows, off[t2]:off[t2 + 1]] += S[o:o + k * m.nv, o2:o2 + k2 * m.nv]
    duh = np.linalg.solve(L, t_glob)
    du = {}
    for e, (XB, xr) in X.items():
        layout, nT = _elem_trace_layout(m, e)
        de = np.zeros(nT)
        for f, t, k, o in layout:
            if t >= 0:
                de[o:o + k * m.nv] = duh[off[t]:off[t + 1]]
        du[e] = xr - XB @ de
    return du, duh


def monolithic_step(m, U, uhat, Ustar, a_dt: float):
    """The same Newton step from the dense Jacobian of [h; g] in [u_implicit; u^] (tiny meshes)."""
    imp = [int(e) for e in np.nonzero(m.imp)[0]]
    sizes = [U[e].size for e in imp]
    uoff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    nh = int(trace_offsets(m)[-1])
    N = int(uoff[-1]) + nh
    Jm = np.zeros((N, N))
    Uc = [u.astype(np.complex128) for u in U]
    Hc = trace_flatten(uhat).astype(np.complex128)
    for col in range(N):
        Up = list(Uc)
        Hp = Hc.copy()
        if col < uoff[-1]:
            k = int(np.searchsorted(uoff, col, side="right") - 1)
            e = imp[k]
            Up[e] = Uc[e].copy()
            Up[e].reshape(-1)[col - uoff[k]] += 1j * EPS
        else:
            Hp[col - uoff[-1]] += 1j * EPS
        h, g = stage_residual(m, Up, trace_unflatten(m, Hp), Ustar, a_dt)
        Jm[:uoff[-1], col] = np.concatenate([h[e].imag for e in imp]) / EPS
        Jm[uoff[-1]:, col] = g.imag / EPS
    h, g = stage_residual(m, U, uhat, Ustar, a_dt)
    rhs = -np.concatenate([np.concatenate([h[e] for e in imp]), g])
    d = np.linalg.solve(Jm, rhs)
    du = {e: d[uoff[k]:uoff[k + 1]] for k, e in enumerate(imp)}
    return du, d[uoff[-1]:]
