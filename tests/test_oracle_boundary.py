"""Pins of the boundary-face oracle (no-slip adiabatic walls and far field on hybridized elements,
FR ghost state on explicit far-field faces; Sec. 2.2, eq. hfr2) against facts fixed by physics and
mathematics: rest and free-stream states are steady, walls pass no mass and no energy once the
trace is solved, the far-field trace is the average of the two states, the condensed Newton step
equals the monolithic one, and Newton converges quadratically."""

import numpy as np
import pytest

from oracle.blocks import EPS, element_blocks, global_jacobian
from oracle.boundary import FARFIELD_FACE, WALL_FACE, BoundaryDiscretisation
from oracle.physics import make_physics
from oracle.solve import backsolve, condense, solve_trace
from oracle.stepping import newton_stage
from workloads.mesh import BC_FARFIELD, BC_WALL, structured_quads, uniform_nodes
from workloads.states import freestream

NS = make_physics({"kind": "ns", "gamma": 1.4, "mu": 2e-2, "Pr": 0.72, "lref": 1.0})
REST = np.array([1.2, 0.0, 0.0, 2.0])
U_INF = freestream((1,), mach=0.4, angle=0.3)[0]


def _mesh(nx, ny, p, imp_rows, bc_y, jitter=0.1, seed=0):
    imp = np.zeros((ny, nx), bool)
    imp[imp_rows, :] = True
    return structured_quads(uniform_nodes(nx, 0, 1), uniform_nodes(ny, 0, 1), periodic=(True, False),
                            jitter=jitter, seed=seed, p=p, implicit=imp.reshape(-1), bc_y=bc_y)


def _solve_trace_equations(d, U, uh, tol=1e-13):
    """Newton on g(u, u^) = 0 for u^ alone (dense complex-step Jacobian; tiny meshes)."""
    for _ in range(30):
        _, g = d.full_residual(U, uh)
        if np.abs(g).max() < tol:
            return uh
        N = uh.size
        Jg = np.zeros((N, N))
        Hc = uh.astype(np.complex128)
        for k in range(N):
            Hp = Hc.copy()
            Hp.reshape(-1)[k] += 1j * EPS
            Jg[:, k] = d.full_residual(U.astype(np.complex128), Hp)[1].imag.reshape(-1) / EPS
        uh = uh - np.linalg.solve(Jg, g.reshape(-1)).reshape(uh.shape)
    raise AssertionError("trace equations did not converge")


def _boundary_traces(d, kind):
    return [t for t in range(d.ntrace)
            if d.trace_sides[t, 1, 0] < 0 and d.kind[tuple(d.trace_sides[t, 0])] == kind]


def test_face_kinds_and_trace_count():
    m = _mesh(4, 5, 2, [0, 1, 3, 4], (BC_WALL, BC_FARFIELD))
    d = BoundaryDiscretisation(m, NS, U_INF)
    walls, fars = _boundary_traces(d, WALL_FACE), _boundary_traces(d, FARFIELD_FACE)
    assert len(walls) == 4 and len(fars) == 4
    # 2 x 4 vertical faces per implicit row, 1 x 4 horizontal inside each implicit pair, 8 boundary
    assert d.ntrace == 4 * 4 * 1 + 2 * 4 + 8
    with pytest.raises(NotImplementedError):
        BoundaryDiscretisation(_mesh(4, 5, 2, [1, 2], (BC_WALL, BC_WALL)), NS, REST)  # explicit wall
    with pytest.raises(NotImplementedError):
        BoundaryDiscretisation(m, make_physics({"kind": "advdiff", "beta": (1.0, 0.5), "nu": 0.01}), [0.0])


def test_rest_state_between_walls_and_free_stream_under_far_field_are_steady():
    m = _mesh(4, 5, 2, [0, 1, 3, 4], (BC_WALL, BC_WALL), jitter=0.15, seed=3)
    d = BoundaryDiscretisation(m, NS, REST)
    U = np.tile(REST, (m.nelem, d.ns, 1))
    R, g = d.full_residual(U, d.initial_trace(U))
    assert np.abs(R).max() < 1e-12 and np.abs(g).max() < 1e-12
    m = _mesh(4, 5, 3, [0, 1], (BC_FARFIELD, BC_FARFIELD), jitter=0.15, seed=3)  # explicit far field on top
    d = BoundaryDiscretisation(m, NS, U_INF)
    U = np.tile(U_INF, (m.nelem, d.ns, 1))
    R, g = d.full_residual(U, d.initial_trace(U))
    assert np.abs(R).max() < 1e-12 and np.abs(g).max() < 1e-12


def test_walls_pass_no_mass_and_no_energy_with_the_solved_trace():
    """Channel with implicit rows on both walls and an explicit core: with g = 0 the element
    integrals of R sum to zero for mass and energy; momentum is not conserved (wall stress)."""
    m = _mesh(3, 4, 2, [0, 3], (BC_WALL, BC_WALL), seed=4)
    d = BoundaryDiscretisation(m, NS, REST)
    xy = d.geo.xy
    U = np.tile(REST, (m.nelem, d.ns, 1))
    U[..., 1] = 0.2 * np.sin(2 * np.pi * xy[..., 0]) * np.sin(np.pi * xy[..., 1])
    U[..., 2] = 0.1 * np.cos(2 * np.pi * xy[..., 0]) * xy[..., 1]
    U[..., 3] += 0.1 * np.cos(2 * np.pi * xy[..., 0])
    uh = _solve_trace_equations(d, U, d.initial_trace(U))
    R, _ = d.full_residual(U, uh)
    W = np.outer(d.ref.w, d.ref.w).reshape(-1)
    total = np.einsum("s,es,esv->v", W, d.geo.J, R)
    scale = np.einsum("s,es,esv->v", W, d.geo.J, np.abs(R))
    assert abs(total[0]) < 1e-14 * scale[0] and abs(total[3]) < 1e-14 * scale[3]
    assert abs(total[1]) > 1e-6 * scale[1]
    for t in _boundary_traces(d, WALL_FACE):
        assert np.abs(uh[t, :, 1:3]).max() < 1e-14  # no-slip
    R0, _ = d.full_residual(U, d.initial_trace(U))  # without the solve energy leaks
    assert abs(np.einsum("s,es,es->", W, d.geo.J, R0[..., 3])) > 1e-6 * scale[3]


def test_far_field_trace_is_the_average_of_the_two_states():
    m = _mesh(3, 4, 2, [0, 1, 2, 3], (BC_WALL, BC_FARFIELD), seed=4)
    d = BoundaryDiscretisation(m, NS, U_INF)
    xy = d.geo.xy
    U = np.tile(U_INF, (m.nelem, d.ns, 1)) * (1 + 0.01 * np.sin(7 * xy[..., :1]))
    U[..., 1:3] *= xy[..., 1:2]
    uh = _solve_trace_equations(d, U, d.initial_trace(U))
    Uf = d.interp_faces(U)
    fars = _boundary_traces(d, FARFIELD_FACE)
    assert len(fars) == 3
    for t in fars:
        e, f = d.trace_sides[t, 0]
        assert np.abs(uh[t] - 0.5 * (Uf[e, f] + U_INF)).max() < 1e-14


def test_condensed_step_equals_the_monolithic_step_with_walls_and_far_field():
    m = _mesh(3, 3, 2, [0, 1], (BC_WALL, BC_FARFIELD), seed=5)
    d = BoundaryDiscretisation(m, NS, U_INF)
    rng = np.random.default_rng(1)
    U = np.tile(U_INF, (m.nelem, d.ns, 1)) * (1 + 1e-2 * rng.standard_normal((m.nelem, d.ns, 4)))
    uh = d.initial_trace(U)
    a_dt, imp = 0.03, d.imp_idx
    Jm = global_jacobian(d, U, uh, a_dt)
    R, Fn = d.residual(U, d.trace_view(uh))
    h = -a_dt * R[imp]
    gv = d.trace_weights(Fn)
    x = np.linalg.solve(Jm, -np.concatenate([h.reshape(-1), d.assemble_trace(gv).reshape(-1)]))
    A, B, C, D = element_blocks(d, U, uh, a_dt)
    nA, nT = A.shape[1], B.shape[2]
    XB, xr, S, t = condense(A[imp], B[imp], C[imp], D[imp], -h.reshape(-1, nA), -gv[imp].reshape(-1, nT))
    duh, _, _ = solve_trace(d, S, t, imp, method="direct")
    du = backsolve(XB, xr, d.trace_view(duh.reshape(d.ntrace, d.n, d.nv))[imp].reshape(-1, nT))
    xc = np.concatenate([du.reshape(-1), duh])
    assert np.abs(xc - x).max() < 1e-12 * np.abs(x).max()


def test_newton_converges_quadratically_with_walls():
    m = _mesh(3, 3, 2, [0, 1], (BC_WALL, BC_FARFIELD), seed=5)
    d = BoundaryDiscretisation(m, NS, U_INF)
    rng = np.random.default_rng(1)
    U = np.tile(U_INF, (m.nelem, d.ns, 1)) * (1 + 1e-2 * rng.standard_normal((m.nelem, d.ns, 4)))
    _, _, info = newton_stage(d, U, U, d.initial_trace(U), 0.05, tol=1e-12)
    hist = np.array(info["history"]) / info["history"][0]
    assert info["converged"] and len(hist) <= 6
    # quadratic: each contraction at least squares the previous one (up to a constant)
    for k in range(1, len(hist) - 1):
        if hist[k] > 1e-10:
            assert hist[k + 1] < 50 * hist[k] ** 2, hist


def _euler_flux_n(u, n, gamma=1.4):
    """Inviscid flux of the conserved state (rho, rho v, E) through unit normal n (textbook)."""
    rho, mx, my, E = u
    vx, vy = mx / rho, my / rho
    p = (gamma - 1.0) * (E - 0.5 * rho * (vx * vx + vy * vy))
    vn = vx * n[0] + vy * n[1]
    return np.array([rho * vn, mx * vn + p * n[0], my * vn + p * n[1], (E + p) * vn]), abs(vn) + np.sqrt(gamma * p / rho)


def test_explicit_far_field_faces_take_the_rusanov_flux_against_the_free_stream():
    """All-explicit inviscid channel with far field top and bottom, uniform u0 != u_inf: interior
    fluxes cancel, so the domain integral of R is minus the Rusanov flux of (u0, u_inf) through both
    boundaries (unit length each)."""
    m = _mesh(3, 3, 2, [], (BC_FARFIELD, BC_FARFIELD), jitter=0.0)
    d = BoundaryDiscretisation(m, make_physics({"kind": "ns", "gamma": 1.4, "mu": 0.0, "Pr": 0.72}), U_INF)
    u0 = np.array([1.1, 0.2, -0.1, 2.1])
    U = np.tile(u0, (m.nelem, d.ns, 1))
    R, _ = d.full_residual(U, np.zeros((0, d.n, d.nv)))
    W = np.outer(d.ref.w, d.ref.w).reshape(-1)
    total = np.einsum("s,es,esv->v", W, d.geo.J, R)
    expected = np.zeros(4)
    for n in ((0.0, 1.0), (0.0, -1.0)):
        f0, a0 = _euler_flux_n(u0, n)
        f1, a1 = _euler_flux_n(U_INF, n)
        expected -= 0.5 * (f0 + f1) + 0.5 * max(a0, a1) * (u0 - U_INF)
    assert np.abs(total - expected).max() < 1e-12 * np.abs(expected).max()


def test_mean_corrected_gradient_includes_the_boundary_jumps():
    """Per element, sum_i W_i J_i q_i = sum_i W_i S_i^T grad~ u_i + sum_f sum_q w_q J_f n (u_bar - u_f)_q
    (the DG lifting tested against the constant and the metric terms), with u_bar = u^ on every
    traced face, boundary faces included."""
    m = _mesh(3, 4, 2, [0, 1, 3], (BC_WALL, BC_FARFIELD), jitter=0.2, seed=6)
    d = BoundaryDiscretisation(m, NS, U_INF)
    rng = np.random.default_rng(5)
    U = np.tile(U_INF, (m.nelem, d.ns, 1)) + 0.1 * rng.standard_normal((m.nelem, d.ns, 4))
    uh = np.tile(U_INF, (d.ntrace, d.n, 1)) + 0.1 * rng.standard_normal((d.ntrace, d.n, 4))
    view = d.trace_view(uh)
    q = d.corrected_gradient(U, view)
    W = np.outer(d.ref.w, d.ref.w).reshape(-1)
    lhs = np.einsum("s,es,escv->ecv", W, d.geo.J, q)
    dxi, deta = d.ref_derivative(U)
    vol = np.einsum("s,esrc,esrv->ecv", W, d.geo.S, np.stack([dxi, deta], axis=2))
    Uf = d.interp_faces(U)
    nb = np.where(d.bnd[:, :, None, None], U_INF, Uf[np.where(d.bnd, 0, m.nbr), np.where(d.bnd, 0, m.nbr_face)])
    imp = d.imp[:, None, None, None]
    kind = d.kind[:, :, None, None]
    ubar = np.where(kind == 2, np.where(imp, nb, Uf), 0.5 * (Uf + nb))  # IMEX faces: explicit side
    ubar = np.where(d.traced[:, :, None, None], view, ubar)
    face = np.einsum("q,efq,efqc,efqv->ecv", d.geo.wface, d.geo.Jf, d.geo.normal, ubar - Uf)
    assert np.abs(lhs - vol - face).max() < 1e-12 * np.abs(lhs).max()
    assert np.any(d.bnd & d.imp[:, None])  # the boundary faces of implicit elements are exercised
