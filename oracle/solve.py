"""Static condensation, trace assembly, trace solve and back-substitution
(Sec. 3.2: L = D - C A^{-1} B, t = s - C A^{-1} r, eqs. assembly, assembly2,
localproblems).

Per implicit element k with Newton right-hand sides r_k = -h_k and
s_k = -g^k (its own contribution to the trace residual):

    X_k = A_k^{-1} [B_k | r_k]                 (LAPACK LU solve, a library step)
    S_k = D_k - C_k X_B,   t_k = s_k - C_k x_r   (elemental L^k, t^k)
    L = sum_k scatter(S_k),  t = sum_k scatter(t_k)  (surjective element-face-point
                                                     to global-trace-point map)
    solve L du^ = t
    du_k = x_r - X_B du^_k                      (= A_k^{-1}(r_k - B_k du^_k))

The trace solve is either a direct sparse LU (scipy) or restarted GMRES(m)
with modified Gram-Schmidt and right face-block-Jacobi preconditioning
P_f = sum of the (f, f) diagonal blocks of the S_k touching face f (the paper
does not name its linear solver; this is the reading used).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def condense(A, B, C, D, r, s):
    """Per element: X_B, x_r, S, t (the condensed blocks)."""
    nT = B.shape[2]
    X = np.linalg.solve(A, np.concatenate([B, r[:, :, None]], axis=2))
    XB = X[:, :, :nT]
    xr = X[:, :, nT]
    S = D - C @ XB
    t = s - np.einsum("eij,ej->ei", C, xr)
    return XB, xr, S, t


def trace_dof_map(disc):
    """(E, nT) global trace unknown of each element trace unknown, -1 off trace."""
    E = disc.mesh.nelem
    n, nv = disc.n, disc.nv
    nT = 4 * n * nv
    idx = -np.ones((E, nT), dtype=np.int64)
    for f in range(4):
        t = disc.tr_of[:, f]
        has = t >= 0
        for m in range(n):
            for v in range(nv):
                l = (f * n + m) * nv + v
                idx[has, l] = (t[has] * n + m) * nv + v
    return idx


def assemble_L(disc, S, elems):
    """Sparse global trace matrix sum_k scatter(S_k) over elements ``elems``."""
    idx = trace_dof_map(disc)[elems]
    N = disc.ntrace * disc.n * disc.nv
    rows = np.repeat(idx[:, :, None], idx.shape[1], axis=2)
    cols = np.repeat(idx[:, None, :], idx.shape[1], axis=1)
    ok = (rows >= 0) & (cols >= 0)
    L = sp.coo_matrix((S[ok], (rows[ok], cols[ok])), shape=(N, N)).tocsr()
    return L


def assemble_t(disc, t, elems):
    idx = trace_dof_map(disc)[elems]
    N = disc.ntrace * disc.n * disc.nv
    out = np.zeros(N)
    ok = idx >= 0
    np.add.at(out, idx[ok], t[ok])
    return out


def face_block_jacobi(disc, S, elems):
    """Inverse of P_f = sum over the two sides of S_k's diagonal face block."""
    n, nv = disc.n, disc.nv
    bs = n * nv
    P = np.zeros((disc.ntrace, bs, bs))
    tr = disc.tr_of[elems]
    for f in range(4):
        has = tr[:, f] >= 0
        blk = S[:, f * bs:(f + 1) * bs, f * bs:(f + 1) * bs]
        np.add.at(P, tr[has, f], blk[has])
    return np.linalg.inv(P)


def gmres(matvec, b, precond, rtol=1e-10, restart=30, maxit=2000):
    """Right-preconditioned restarted GMRES with modified Gram-Schmidt.
    Solves A x = b from x0 = 0; stops when ||b - A x|| <= rtol ||b||.
    Returns x, total inner iterations, final relative residual."""
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    if nb == 0.0:
        return x, 0, 0.0
    it = 0
    rel = 1.0
    while it < maxit:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        rel = beta / nb
        if rel <= rtol:
            break
        m = restart
        V = np.zeros((m + 1, len(b)))
        Z = np.zeros((m, len(b)))
        H = np.zeros((m + 1, m))
        V[0] = r / beta
        k_done = 0
        for k in range(m):
            Z[k] = precond(V[k])
            w = matvec(Z[k])
            for i in range(k + 1):
                H[i, k] = w @ V[i]
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            k_done = k + 1
            it += 1
            e1 = np.zeros(k + 2)
            e1[0] = beta
            y, *_ = np.linalg.lstsq(H[: k + 2, : k + 1], e1, rcond=None)
            res = np.linalg.norm(e1 - H[: k + 2, : k + 1] @ y)
            if H[k + 1, k] != 0.0:
                V[k + 1] = w / H[k + 1, k]
            if res / nb <= rtol or H[k + 1, k] == 0.0 or it >= maxit:
                break
        x = x + Z[:k_done].T @ y
        rel = np.linalg.norm(b - matvec(x)) / nb
        if rel <= rtol:
            break
    return x, it, rel


def solve_trace(disc, S, t, elems, method="direct", rtol=1e-12, restart=30, maxit=5000):
    """Solve L du^ = t; returns du^ (ntrace*n*nv,), iterations, relative residual."""
    L = assemble_L(disc, S, elems)
    tg = assemble_t(disc, t, elems)
    if method == "direct":
        x = spla.spsolve(L.tocsc(), tg)
        nb = np.linalg.norm(tg)
        rel = np.linalg.norm(tg - L @ x) / nb if nb > 0 else 0.0
        return x, 0, rel
    Pinv = face_block_jacobi(disc, S, elems)
    bs = disc.n * disc.nv

    def precond(v):
        return np.einsum("fij,fj->fi", Pinv, v.reshape(-1, bs)).reshape(-1)

    return gmres(lambda v: L @ v, tg, precond, rtol=rtol, restart=restart, maxit=maxit)


def backsolve(XB, xr, duhat_view):
    """du_k = x_r - X_B du^_k for every element (duhat_view (E, nT))."""
    return xr - np.einsum("eij,ej->ei", XB, duhat_view)
