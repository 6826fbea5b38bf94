"""Newton on the DIRK stage equations and the IMEX time step (Secs. 3.1, 4).

Stage equations (eqs. 9oind, 23nffsd):  u - u* - a_ii dt R(u, u^) = 0,
g(u, u^) = 0, with u* = u^n + dt sum_{j<i} a_ij R_j.

Newton stops when ||[h; g]||_2 <= tol ||[h; g]^0||_2 (the paper quotes implicit
tolerances without naming a norm; this relative 2-norm is the reading used),
starting from u = u*, u^ = the trace carried in.

IMEX step (Algorithm 1 with the domain split of Sec. 4): explicit elements
take u_i^ex = u_n^ex + dt sum_{j<=i} ahat_{i+1,j} R^ex_j (eq. explicitimex),
implicit elements solve the hybridized stage, R^ex_{i+1} = R(u_i) and finally
u_{n+1} = u_n + dt sum b_j R^im_j + dt sum bhat_j R^ex_j.

Tableaux.  SDIRK2 is printed in Sec. 3.1 (gamma = 1 - sqrt(2)/2, c = (gamma, 1),
A = [[gamma, 0], [1 - gamma, gamma]], b = (1 - gamma, gamma)); its explicit
partner IMEX_{3,2} is cited to Ascher-Ruuth-Spiteri but its tableau is not in
the paper's text: the ARS(2,3,2) explicit tableau with delta = -2 sqrt(2)/3,
c_hat = (0, gamma, 1), rows [0], [gamma], [delta, 1 - delta], b_hat =
(0, 1 - gamma, gamma) is used.  The one-stage pair is backward Euler with the
explicit partner c_hat = (0, 1), ahat_21 = 1, b_hat = (0, 1) (ARS(1,2,1)).
Both pairs satisfy b_hat_{j+1} = b_j, which makes the interface flux
contributions cancel in the step update.
"""

from __future__ import annotations

import math

import numpy as np

from .blocks import element_blocks
from .solve import condense, solve_trace, backsolve

_G = 1.0 - math.sqrt(2.0) / 2.0
_DELTA = -2.0 * math.sqrt(2.0) / 3.0

TABLEAUX = {
    "be": {
        "a": np.array([[1.0]]),
        "b": np.array([1.0]),
        "ahat": np.array([[0.0, 0.0], [1.0, 0.0]]),
        "bhat": np.array([0.0, 1.0]),
    },
    "sdirk2": {
        "a": np.array([[_G, 0.0], [1.0 - _G, _G]]),
        "b": np.array([1.0 - _G, _G]),
        "ahat": np.array([[0.0, 0.0, 0.0], [_G, 0.0, 0.0], [_DELTA, 1.0 - _DELTA, 0.0]]),
        "bhat": np.array([0.0, 1.0 - _G, _G]),
    },
}


def newton_stage(disc, U0, Ustar, uhat0, a_dt, tol=1e-8, maxit=25, linear="direct",
                 gmres_rtol=1e-12):
    """Solve the hybridized stage for the implicit elements of ``U0`` (explicit
    elements are held fixed).  Returns U, uhat, info dict."""
    U = U0.copy()
    uhat = uhat0.copy()
    imp = disc.imp_idx
    nA = disc.ns * disc.nv
    nT = 4 * disc.n * disc.nv
    hist = []
    lin_its = []
    for it in range(maxit + 1):
        R, Fn = disc.residual(U, disc.trace_view(uhat))
        gview = disc.trace_weights(Fn)
        g = disc.assemble_trace(gview)
        h = U[imp] - Ustar[imp] - a_dt * R[imp]
        nrm = math.sqrt(float(np.sum(h * h) + np.sum(g * g)))
        hist.append(nrm)
        if nrm <= tol * hist[0] or nrm == 0.0 or it == maxit:
            break
        A, B, C, D = element_blocks(disc, U, uhat, a_dt)
        r = -h.reshape(len(imp), nA)
        s = -gview[imp].reshape(len(imp), nT)
        XB, xr, S, t = condense(A[imp], B[imp], C[imp], D[imp], r, s)
        x, its, _ = solve_trace(disc, S, t, imp, method=linear, rtol=gmres_rtol)
        lin_its.append(its)
        duh = x.reshape(disc.ntrace, disc.n, disc.nv)
        dview = disc.trace_view(duh)[imp].reshape(len(imp), nT)
        du = backsolve(XB, xr, dview)
        U[imp] += du.reshape(len(imp), disc.ns, disc.nv)
        uhat = uhat + duh
    converged = hist[-1] <= tol * hist[0] or hist[-1] == 0.0
    return U, uhat, {"history": hist, "iterations": len(hist) - 1,
                     "linear_iterations": lin_its, "converged": converged}


def imex_step(disc, Un, uhat, dt, tableau="sdirk2", tol=1e-10, linear="direct", maxit=25, stage=None):
    """One IMEX step; returns U_{n+1}, trace, per-stage info.  ``stage`` replaces
    ``newton_stage`` (same signature) for discretisations with another trace space."""
    stage = newton_stage if stage is None else stage
    tab = TABLEAUX[tableau] if isinstance(tableau, str) else tableau
    a, b, ahat, bhat = tab["a"], tab["b"], tab["ahat"], tab["bhat"]
    s = len(b)
    imp, ex = disc.imp_idx, disc.ex_idx
    R1, _ = disc.full_residual(Un, uhat)
    Rex = [R1]
    Rim = []
    infos = []
    for i in range(1, s + 1):
        Ui = Un.copy()
        for j in range(1, i + 1):
            Ui[ex] += dt * ahat[i, j - 1] * Rex[j - 1][ex]
        Ustar = Un.copy()
        for j in range(1, i):
            Ustar[imp] += dt * a[i - 1, j - 1] * Rim[j - 1][imp]
        Ui[imp] = Ustar[imp]
        Ui, uhat, info = stage(disc, Ui, Ustar, uhat, a[i - 1, i - 1] * dt, tol=tol,
                               linear=linear, maxit=maxit)
        infos.append(info)
        R, _ = disc.full_residual(Ui, uhat)
        Rim.append(R)
        Rex.append(R)
    Unew = Un.copy()
    for j in range(s):
        Unew[imp] += dt * b[j] * Rim[j][imp]
    for j in range(s + 1):
        Unew[ex] += dt * bhat[j] * Rex[j][ex]
    return Unew, uhat, infos
