"""Pins of the EFR oracle (trace continuous on the implicit skeleton at GLL face points, Sec. 2.2)
against facts fixed by mathematics and by the paper's statements about EFR: the GLL rule, closed
counts of trace unknowns, free-stream preservation, polynomial exactness, conservation of the
implicit region as a whole (Sec. 4), the condensed Newton step against the monolithic one, and
design-order convergence."""

import math

import numpy as np
import pytest

from oracle.basis import gauss_lobatto
from oracle.efr import EmbeddedDiscretisation, condensed_newton_step, monolithic_newton_step
from oracle.fr import Discretisation
from oracle.physics import AdvectionDiffusion, make_physics
from oracle.stepping import newton_stage
from workloads.mesh import structured_quads, uniform_nodes
from workloads.states import freestream, isentropic_vortex

NS = {"kind": "ns", "gamma": 1.4, "mu": 5e-3, "Pr": 0.72, "lref": 1.0}


def _mesh(n, hi, p, implicit=None, jitter=0.0, seed=0):
    return structured_quads(uniform_nodes(n, 0, hi), uniform_nodes(n, 0, hi), jitter=jitter,
                            seed=seed, p=p, implicit=implicit)


def _band(n, rows):
    imp = np.zeros((n, n), bool)
    imp[rows, :] = True
    return imp.reshape(-1)


def test_gauss_lobatto_closed_forms_and_exactness():
    x, w = gauss_lobatto(3)
    assert np.allclose(x, [-1, 0, 1], atol=1e-15) and np.allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    x, w = gauss_lobatto(4)
    assert np.allclose(x, [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], atol=1e-15)
    assert np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    x, w = gauss_lobatto(5)
    assert np.allclose(x, [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], atol=1e-15)
    assert np.allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)
    for n in range(2, 9):
        x, w = gauss_lobatto(n)
        for k in range(2 * n - 2):  # exact to degree 2n - 3
            assert abs(np.sum(w * x**k) - (0.0 if k % 2 else 2.0 / (k + 1))) < 1e-14
        # interior nodes: the roots of P'_{n-1} (independent library routine)
        roots = np.sort(np.polynomial.legendre.Legendre.basis(n - 1).deriv().roots().real)
        assert np.allclose(x[1:-1], roots, atol=1e-14)


def test_trace_node_counts_and_shared_coordinates():
    ad = AdvectionDiffusion((1.0, 0.5), 0.01)
    for n, p in ((4, 1), (4, 2), (5, 3)):
        d = EmbeddedDiscretisation(_mesh(n, 1.0, p), ad)
        # all implicit, periodic: every vertex once, p - 1 interior points on each of 2 n^2 faces
        assert d.nvert == n * n and d.nnode == n * n + 2 * n * n * (p - 1)
        assert d.nnode < d.ntrace * d.n  # fewer unknowns than HFR's (p + 1) per face
    n, p = 6, 3
    d = EmbeddedDiscretisation(_mesh(n, 10.0, p, _band(n, [2, 3]), jitter=0.2, seed=3), ad)
    # band of two full rows: 2n vertical and n horizontal trace faces touching 3n vertices
    assert d.ntrace == 3 * n and d.nvert == 3 * n and d.nnode == 3 * n + 3 * n * (p - 1)
    d = EmbeddedDiscretisation(_mesh(4, 1.0, 2, np.arange(16) == 5), ad)
    assert d.ntrace == 0 and d.nnode == 0  # an isolated implicit element has no trace
    # every copy of a node sits at the same physical point (modulo the period)
    d = EmbeddedDiscretisation(_mesh(6, 10.0, 3, _band(6, [2, 3]), jitter=0.2, seed=3), ad)
    sa, sb = np.array([-1.0, 1, -1, 1]), np.array([-1.0, -1, 1, 1])
    where = {}
    for e, f, q in zip(*np.nonzero(d.node_of >= 0)):
        xi, eta = ((-1.0, 1.0)[f], d.xl[q]) if f < 2 else (d.xl[q], (-1.0, 1.0)[f - 2])
        xy = (0.25 * (1 + sa * xi) * (1 + sb * eta)) @ d.mesh.verts[e]
        k = d.node_of[e, f, q]
        if k in where:
            assert np.abs((xy - where[k] + 5.0) % 10.0 - 5.0).max() < 1e-12
        where[k] = xy
    assert len(where) == d.nnode


def test_free_stream_is_preserved_on_skewed_imex_meshes():
    for p in (2, 3):
        mesh = _mesh(6, 10.0, p, _band(6, [2, 3]), jitter=0.2, seed=3)
        d = EmbeddedDiscretisation(mesh, make_physics(NS))
        U = freestream((mesh.nelem, d.ns), mach=0.4, angle=0.3)
        R, g = d.full_residual(U, d.initial_trace(U))
        assert np.abs(R).max() < 1e-12 and np.abs(g).max() < 1e-12


def test_advection_residual_is_exact_for_a_continuous_quadratic():
    """u = x^2 + xy - y is in every element's space and continuous, the averaged trace is exact at
    every node off the periodic seam, so every jump vanishes and R = -beta . grad u on elements
    away from the seam."""
    n = 5
    for p in (2, 3):
        d = EmbeddedDiscretisation(_mesh(n, 1.0, p), AdvectionDiffusion((1.0, 0.5), 0.0))
        x, y = d.geo.xy[..., 0], d.geo.xy[..., 1]
        U = (x**2 + x * y - y)[..., None]
        R, _ = d.full_residual(U, d.initial_trace(U))
        exact = -(1.0 * (2 * x + y) + 0.5 * (x - 1))
        inner = [i + n * j for j in range(1, n - 1) for i in range(1, n - 1)]
        assert np.abs(R[inner, :, 0] - exact[inner]).max() < 1e-12


def test_solved_trace_conserves_the_domain_and_cancels_fluxes_at_face_interior_nodes():
    """With h = 0 and g = 0: the total of int J R over all elements vanishes (implicit region
    conservative as a whole, FR flux on the interface); at interior GLL points of a trace face the
    two sides' fluxes cancel pointwise, at vertex nodes only summed over the faces meeting there."""
    imp = np.array([1, 1, 1, 0, 1, 1, 1, 0, 0, 1, 1, 0, 0, 0, 0, 0], bool)
    mesh = _mesh(4, 1.0, 3, imp, jitter=0.15, seed=5)
    d = EmbeddedDiscretisation(mesh, AdvectionDiffusion((1.0, 0.5), 0.02))
    rng = np.random.default_rng(0)
    U = rng.standard_normal((mesh.nelem, d.ns, 1))
    uh0 = d.initial_trace(U)
    dU, duh = condensed_newton_step(d, U, uh0, U, 0.05)  # affine problem: one step solves it
    U1, uh1 = U + dU, uh0 + duh
    R, Fn = d.residual(U1, d.trace_view(uh1))
    g = d.assemble_trace(d.trace_weights(Fn))
    assert np.abs(U1[d.imp_idx] - U[d.imp_idx] - 0.05 * R[d.imp_idx]).max() < 1e-12
    assert np.abs(g).max() < 1e-13
    W = np.outer(d.ref.w, d.ref.w).reshape(-1)
    scale = np.sum(W * d.geo.J * np.abs(R[..., 0]))
    assert abs(np.sum(W * d.geo.J * R[..., 0])) < 1e-14 * scale
    R0, _ = d.full_residual(U1, d.initial_trace(U1))
    assert abs(np.sum(W * d.geo.J * R0[..., 0])) > 1e-3 * scale
    # per face: sum of both sides' w J F^.n at each GLL point
    jump = np.zeros((d.ntrace, d.n))
    for t in range(d.ntrace):
        for s in range(2):
            e, f = d.trace_sides[t, s]
            jump[t] += d.wl * Fn[e, f, :, 0]
    assert np.abs(jump[:, 1:-1]).max() < 1e-13
    assert np.abs(jump[:, [0, -1]]).max() > 1e-6  # vertex nodes: not face by face


def test_condensed_newton_step_equals_the_monolithic_step():
    imp = np.array([1, 1, 1, 1, 1, 0, 0, 0, 0], bool)
    mesh = _mesh(3, 10.0, 2, imp, jitter=0.1, seed=2)
    d = EmbeddedDiscretisation(mesh, make_physics(dict(NS, mu=2e-2)))
    U = isentropic_vortex(d.geo.xy)
    rng = np.random.default_rng(4)
    Ustar = U + 1e-3 * rng.standard_normal(U.shape)
    uh = d.initial_trace(U) * (1 + 1e-3 * rng.standard_normal((d.nnode, d.nv)))
    a = condensed_newton_step(d, U, uh, Ustar, 0.04)
    b = monolithic_newton_step(d, U, uh, Ustar, 0.04)
    scale = max(np.abs(b[0]).max(), np.abs(b[1]).max())
    assert scale > 1e-3
    assert max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max()) < 1e-12 * scale


def test_residual_converges_at_design_order_on_smooth_field():
    errs = []
    for n in (8, 16, 32):
        d = EmbeddedDiscretisation(_mesh(n, 1.0, 3), AdvectionDiffusion((1.0, 0.5), 0.0))
        xy = d.geo.xy
        k = 2 * np.pi
        U = np.sin(k * xy[..., 0]) * np.cos(k * xy[..., 1])
        exact = -(1.0 * k * np.cos(k * xy[..., 0]) * np.cos(k * xy[..., 1])
                  - 0.5 * k * np.sin(k * xy[..., 0]) * np.sin(k * xy[..., 1]))
        R, _ = d.full_residual(U[..., None], d.initial_trace(U[..., None]))
        errs.append(np.abs(R[..., 0] - exact).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.8), rates


@pytest.mark.parametrize("p", [2, 3])
def test_backward_euler_spatial_convergence_p_plus_one(p):
    """One backward-Euler step of a Fourier mode (advection-diffusion, affine: one condensed
    Newton step solves it) against the continuous-in-space BE solution converges at p + 1."""
    beta, nu, dt = (1.0, 0.5), 0.01, 0.05
    kx, ky = 1, 2
    errs = []
    for n in (8, 16, 32):
        d = EmbeddedDiscretisation(_mesh(n, 1.0, p), AdvectionDiffusion(beta, nu))
        xy = d.geo.xy
        phase = 2 * np.pi * (kx * xy[..., 0] + ky * xy[..., 1])
        U0 = np.cos(phase)[..., None]
        lam = 2j * np.pi * (beta[0] * kx + beta[1] * ky) + 4 * np.pi**2 * nu * (kx * kx + ky * ky)
        exact = np.real(np.exp(1j * phase) / (1 + dt * lam))
        dU, _ = condensed_newton_step(d, U0, d.initial_trace(U0), U0, dt)
        W = np.outer(d.ref.w, d.ref.w).reshape(-1)
        errs.append(math.sqrt(np.sum(W * d.geo.J * ((U0 + dU)[..., 0] - exact) ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > p + 0.8), (errs, rates)


def test_efr_and_hfr_agree_to_discretisation_error():
    """Both are consistent discretisations of the same stage: their BE solutions differ by far
    less than the step changes the state, and the difference shrinks under refinement."""
    diffs = []
    for n in (8, 16):
        mesh = _mesh(n, 1.0, 2)
        ad = AdvectionDiffusion((1.0, 0.5), 0.01)
        de, dh = EmbeddedDiscretisation(mesh, ad), Discretisation(mesh, ad)
        xy = de.geo.xy
        U0 = np.cos(2 * np.pi * (xy[..., 0] + 2 * xy[..., 1]))[..., None]
        dUe, _ = condensed_newton_step(de, U0, de.initial_trace(U0), U0, 0.05)
        Uh, _, _ = newton_stage(dh, U0, U0, dh.initial_trace(U0), 0.05, tol=1e-13)
        diffs.append(np.abs(U0 + dUe - Uh).max() / np.abs(Uh - U0).max())
    assert diffs[0] < 0.05 and diffs[1] < diffs[0] / 4, diffs


def test_transmission_residuals_sum_to_the_net_element_flux():
    """For any state and trace on a fully implicit periodic mesh, sum_i g_i = -sum_k int J R_k:
    the DG-recovering lift integrates the GLL interpolant of each face's flux exactly, and the
    transmission conditions weight it by the GLL rule."""
    mesh = _mesh(4, 1.0, 3, jitter=0.15, seed=8)
    for phys in (AdvectionDiffusion((1.0, 0.5), 0.02), make_physics(NS)):
        d = EmbeddedDiscretisation(mesh, phys)
        rng = np.random.default_rng(3)
        if d.nv == 1:
            U = rng.standard_normal((mesh.nelem, d.ns, 1))
        else:
            U = isentropic_vortex(d.geo.xy) * (1 + 1e-2 * rng.standard_normal((mesh.nelem, d.ns, d.nv)))
        uh = d.initial_trace(U) * (1 + 1e-2 * rng.standard_normal((d.nnode, d.nv)))
        R, g = d.full_residual(U, uh)
        W = np.outer(d.ref.w, d.ref.w).reshape(-1)
        total = np.einsum("s,es,esv->v", W, d.geo.J, R)
        assert np.abs(g.sum(axis=0) + total).max() < 1e-12 * np.abs(g).sum()


def test_mean_corrected_gradient_equals_the_gll_face_integral_of_the_jump():
    """Per element, sum_i W_i J_i q_i = sum_i W_i S_i^T grad~ u_i + sum_f sum_q w^GLL_q J_f n (u^ - u_f)_q:
    the gradient correction is the DG lifting of the GLL jump polynomial, tested against the
    constant and the metric terms (in the element's space for p >= 1)."""
    mesh = _mesh(4, 1.0, 3, jitter=0.2, seed=6)
    d = EmbeddedDiscretisation(mesh, AdvectionDiffusion((1.0, 0.5), 0.02))
    rng = np.random.default_rng(5)
    U = rng.standard_normal((mesh.nelem, d.ns, 1))
    uh = rng.standard_normal((d.nnode, 1))
    view = d.trace_view(uh)
    q = d.corrected_gradient(U, view)
    W = np.outer(d.ref.w, d.ref.w).reshape(-1)
    lhs = np.einsum("s,es,escv->ecv", W, d.geo.J, q)
    dxi, deta = d.ref_derivative(U)
    vol = np.einsum("s,esrc,esrv->ecv", W, d.geo.S, np.stack([dxi, deta], axis=2))
    UfL = np.einsum("qm,efmv->efqv", d.IGL, d.interp_faces(U))
    face = np.einsum("q,efq,efqc,efqv->ecv", d.wl, d.JfL, d.normalL, view - UfL)
    assert np.abs(lhs - vol - face).max() < 1e-12 * np.abs(lhs).max()


def test_efr_imex_step_conserves_across_the_interface():
    """Algorithm 1 with EFR on the implicit band and FR elsewhere (Sec. 4): the FR flux on the
    interface and b^_{j+1} = b_j make the step conservative for the whole domain, the implicit
    region being conservative as a whole (the paper's statement for EFR)."""
    from oracle import efr
    from oracle.stepping import imex_step
    n = 6
    mesh = _mesh(n, 10.0, 2, _band(n, [2, 3]), jitter=0.15, seed=4)
    d = EmbeddedDiscretisation(mesh, make_physics(dict(NS, mu=1e-2)))
    U0 = isentropic_vortex(d.geo.xy)
    W = np.outer(d.ref.w, d.ref.w).reshape(-1)
    mass0 = np.einsum("s,es,esv->v", W, d.geo.J, U0)
    U1, _, infos = imex_step(d, U0, d.initial_trace(U0), 0.05, "sdirk2", tol=1e-12, stage=efr.newton_stage)
    assert all(i["converged"] for i in infos)
    mass1 = np.einsum("s,es,esv->v", W, d.geo.J, U1)
    assert np.abs(mass1 - mass0).max() < 1e-12 * np.abs(mass0).max()
    assert np.abs(U1 - U0).max() > 1e-4  # the step moves the state


# ------------------------------------------------------- EFR with walls and far field
from oracle.blocks import EPS  # noqa: E402
from oracle.boundary import FARFIELD_FACE, WALL_FACE  # noqa: E402
from workloads.mesh import BC_FARFIELD, BC_WALL  # noqa: E402

NS_B = make_physics(dict(NS, mu=2e-2))
REST = np.array([1.2, 0.0, 0.0, 2.0])
U_INF = np.array([1.0, 0.3, 0.05, 2.6])


def _wall_mesh(nx, ny, p, rows, bc_y, jitter=0.1, seed=0):
    imp = np.zeros((ny, nx), bool)
    imp[rows, :] = True
    return structured_quads(uniform_nodes(nx, 0, 1), uniform_nodes(ny, 0, 1), periodic=(True, False),
                            jitter=jitter, seed=seed, p=p, implicit=imp.reshape(-1), bc_y=bc_y)


def _solve_g(d, U, uh):
    for _ in range(30):
        _, g = d.full_residual(U, uh)
        if np.abs(g).max() < 1e-13:
            return uh
        Jg = np.empty((uh.size, uh.size))
        for k in range(uh.size):
            hp = uh.astype(np.complex128)
            hp.reshape(-1)[k] += 1j * EPS
            Jg[:, k] = d.full_residual(U.astype(np.complex128), hp)[1].imag.reshape(-1) / EPS
        uh = uh - np.linalg.solve(Jg, g.reshape(-1)).reshape(uh.shape)
    raise AssertionError("trace equations did not converge")


def test_boundary_faces_keep_their_own_gauss_point_nodes():
    m = _wall_mesh(4, 4, 3, [0, 1, 2, 3], (BC_WALL, BC_FARFIELD))
    d = EmbeddedDiscretisation(m, NS_B, U_INF)
    nb = int(d.bface.sum())
    assert nb == 8 and d.efr.sum() == 2 * (4 * 4 + 4 * 3)
    # vertices of the interior skeleton: 5 rows of 4 (boundary vertex rows met by x-faces only)
    assert d.nvert == 5 * 4 and d.nnode == d.nvert + (d.efr.sum() // 2) * (d.n - 2) + nb * d.n
    own = d.node_of[d.bface]
    assert len(np.unique(own)) == own.size and own.min() >= d.nnode - nb * d.n


def test_rest_state_between_walls_is_steady():
    m = _wall_mesh(4, 5, 2, [0, 1, 3, 4], (BC_WALL, BC_WALL), jitter=0.15, seed=3)
    d = EmbeddedDiscretisation(m, NS_B)
    U = np.tile(REST, (m.nelem, d.ns, 1))
    R, g = d.full_residual(U, d.initial_trace(U))
    assert np.abs(R).max() < 1e-12 and np.abs(g).max() < 1e-12


def test_walls_conserve_mass_and_energy_with_the_solved_efr_trace():
    m = _wall_mesh(3, 4, 2, [0, 3], (BC_WALL, BC_WALL), seed=4)
    d = EmbeddedDiscretisation(m, NS_B)
    rng = np.random.default_rng(4)
    U = REST + 0.05 * rng.standard_normal((m.nelem, d.ns, 4))
    uh = _solve_g(d, U, d.initial_trace(U))
    R, _ = d.full_residual(U, uh)
    W = np.outer(d.ref.w, d.ref.w).reshape(-1)
    total = np.einsum("s,es,esv->v", W, d.geo.J, R)
    scale = np.einsum("s,es,esv->v", W, d.geo.J, np.abs(R))
    assert abs(total[0]) < 1e-13 * scale[0] and abs(total[3]) < 1e-13 * scale[3]
    assert np.abs(uh[d.node_of[d.bface]][..., 1:3]).max() < 1e-14  # no-slip at the wall nodes


def test_far_field_nodes_hold_the_average_and_condensed_equals_monolithic():
    m = _wall_mesh(3, 3, 2, [0, 1, 2], (BC_WALL, BC_FARFIELD), seed=5)
    d = EmbeddedDiscretisation(m, NS_B, U_INF)
    rng = np.random.default_rng(6)
    U = U_INF * (1 + 1e-2 * rng.standard_normal((m.nelem, d.ns, 4)))
    uh = _solve_g(d, U, d.initial_trace(U))
    Uf = d.interp_faces(U)
    far = d.bface & (d.kind == FARFIELD_FACE)
    assert far.sum() == 3
    assert np.abs(uh[d.node_of[far]] - 0.5 * (Uf[far] + U_INF)).max() < 1e-14
    Ustar = U + 1e-3 * rng.standard_normal(U.shape)
    a = condensed_newton_step(d, U, d.initial_trace(U), Ustar, 0.03)
    b = monolithic_newton_step(d, U, d.initial_trace(U), Ustar, 0.03)
    scale = max(np.abs(b[0]).max(), np.abs(b[1]).max())
    assert scale > 1e-3 and max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max()) < 1e-12 * scale


def test_mean_corrected_gradient_with_boundary_traces():
    """Per element of an all-implicit wall / far-field mesh: sum_i W_i J_i q_i = volume term + the
    GLL face sums of u^ - u_f on EFR faces + the Gauss face sums of u^ - u_f on boundary faces."""
    m = _wall_mesh(3, 4, 2, [0, 1, 2, 3], (BC_WALL, BC_FARFIELD), jitter=0.2, seed=7)
    d = EmbeddedDiscretisation(m, NS_B, U_INF)
    rng = np.random.default_rng(8)
    U = U_INF + 0.1 * rng.standard_normal((m.nelem, d.ns, 4))
    view = d.trace_view(U_INF + 0.1 * rng.standard_normal((d.nnode, 4)))
    q = d.corrected_gradient(U, view)
    W = np.outer(d.ref.w, d.ref.w).reshape(-1)
    lhs = np.einsum("s,es,escv->ecv", W, d.geo.J, q)
    dxi, deta = d.ref_derivative(U)
    vol = np.einsum("s,esrc,esrv->ecv", W, d.geo.S, np.stack([dxi, deta], axis=2))
    Uf = d.interp_faces(U)
    UfL = np.einsum("qm,efmv->efqv", d.IGL, Uf)
    efr = d.efr[:, :, None, None]
    bf = d.bface[:, :, None, None]
    face = np.einsum("q,efq,efqc,efqv->ecv", d.wl, d.JfL, d.normalL, np.where(efr, view - UfL, 0.0))
    face += np.einsum("q,efq,efqc,efqv->ecv", d.geo.wface, d.geo.Jf, d.geo.normal, np.where(bf, view - Uf, 0.0))
    assert np.all(d.efr | d.bface)  # every face carries a trace here
    assert np.abs(lhs - vol - face).max() < 1e-12 * np.abs(lhs).max()
