"""Pins of the mixed-degree FP64 oracle (p-adaptive meshes, Sec. 3.2) against facts fixed by the
uniform operator and by mathematics: reduction to the uniform-degree residual when all degrees
agree, exactness of the face projection, free-stream preservation across faces of unequal degree,
polynomial exactness of the advection residual, discrete conservation with the solved trace, and
the condensed Newton step against the monolithic one."""

import numpy as np
import pytest

from oracle.basis import RefElement1D, gauss_legendre, lagrange
from oracle.blocks_mixed import hybridized_step, monolithic_step, trace_flatten
from oracle.fr import Discretisation
from oracle.fr_mixed import MixedDiscretisation
from oracle.physics import make_physics
from workloads import make_config
from workloads.mesh import structured_quads, uniform_nodes
from workloads.states import isentropic_vortex, sample_points

NS = {"kind": "ns", "gamma": 1.4, "mu": 5e-3, "Pr": 0.72, "lref": 1.0}
ADV = {"kind": "advdiff", "beta": (1.0, 0.5), "nu": 0.0, "lref": 1.0}
ADVDIFF = {"kind": "advdiff", "beta": (1.0, 0.5), "nu": 0.01, "lref": 1.0}


def _mesh(n, lo, hi, degrees, seed, implicit=None, jitter=0.0):
    rng = np.random.default_rng(seed)
    p = rng.choice(degrees, size=n * n).astype(np.int32)
    imp = np.ones(n * n, bool) if implicit is None else implicit
    return structured_quads(uniform_nodes(n, lo, hi), uniform_nodes(n, lo, hi), jitter=jitter,
                            seed=seed, p=p, implicit=imp)


def _points(mesh, e):
    """Element e's solution points through the bilinear map of its corner vertices."""
    r = RefElement1D(int(mesh.p[e]))
    xi, eta = np.tile(r.x, r.n), np.repeat(r.x, r.n)
    sa = np.array([-1.0, 1.0, -1.0, 1.0])
    sb = np.array([-1.0, -1.0, 1.0, 1.0])
    N = 0.25 * (1 + sa[None, :] * xi[:, None]) * (1 + sb[None, :] * eta[:, None])
    return N @ mesh.verts[e]


def _quad_weights(m, e):
    r = m.refs[int(m.p[e])]
    return np.outer(r.w, r.w).reshape(-1) * m.J[e]


def _compare_uniform(mesh, u0, phys, seed=0):
    d = Discretisation(mesh, make_physics(phys))
    m = MixedDiscretisation(mesh, make_physics(phys))
    rng = np.random.default_rng(seed)
    uh = d.initial_trace(u0)
    uh = uh * (1 + 1e-3 * rng.standard_normal(uh.shape))
    R, g = d.full_residual(u0, uh)
    Rm, gm = m.full_residual([u0[e] for e in range(mesh.nelem)], [uh[t] for t in range(d.ntrace)])
    assert np.abs(np.stack(Rm) - R).max() <= 1e-13 * np.abs(R).max()
    if d.ntrace:
        assert np.abs(np.stack(gm) - g).max() <= 1e-13 * np.abs(g).max()


def test_uniform_degree_reduces_to_the_uniform_operator():
    w = make_config("vortex", n=4, p=3, jitter=0.15, seed=9, re=200.0)  # skewed, all implicit
    _compare_uniform(w.mesh, w.u0, w.physics)
    n = 6
    band = np.repeat([False, False, True, True, False, False], n)  # IMEX band of two rows
    mesh = structured_quads(uniform_nodes(n, 0, 10), uniform_nodes(n, 0, 10), p=3, implicit=band)
    _compare_uniform(mesh, isentropic_vortex(sample_points(mesh, 3)), NS)


def test_face_projection_inverts_interpolation_and_is_exact_to_the_element_degree():
    for p in range(1, 6):
        r = RefElement1D(p)
        for nf in range(p + 1, p + 4):
            s, w = gauss_legendre(nf)
            T = lagrange(r.x, s)  # element nodes -> face points
            P = (w[:, None] * T).T / r.w[:, None]  # the projection the oracle builds
            assert np.allclose(P @ T, np.eye(r.n), atol=1e-13)
            # any polynomial of degree <= p at the face points returns its nodal values
            for k in range(p + 1):
                assert np.allclose(P @ s**k, r.x**k, atol=1e-13)
    mesh = _mesh(4, 0.0, 1.0, [1, 2, 3, 4], 3)
    m = MixedDiscretisation(mesh, make_physics(ADV))
    for (n, k), T in m.T.items():
        assert k >= n and np.allclose(m.P[n, k] @ T, np.eye(n), atol=1e-13)
    # faces carry the higher degree of the two sides, and both sides agree on the point count
    for t in range(m.ntrace):
        (e0, f0), (e1, f1) = m.trace_sides[t]
        assert m.nf[e0, f0] == m.nf[e1, f1] == max(m.n[e0], m.n[e1]) == m.trace_npts[t]


def test_free_stream_is_preserved_across_faces_of_unequal_degree():
    n = 6
    band = np.zeros((n, n), bool)
    band[2:4, :] = True
    mesh = _mesh(n, 0.0, 10.0, [2, 3, 4], 3, implicit=band.reshape(-1), jitter=0.2)
    assert len(set(mesh.p.tolist())) == 3
    m = MixedDiscretisation(mesh, make_physics(NS))
    c = np.array([1.2, 0.3, -0.2, 2.5])
    U = [np.tile(c, (int(mesh.p[e] + 1) ** 2, 1)) for e in range(mesh.nelem)]
    uh = [np.tile(c, (int(k), 1)) for k in m.trace_npts]
    R, g = m.full_residual(U, uh)
    assert max(np.abs(r).max() for r in R) < 1e-12
    assert max(np.abs(x).max() for x in g) < 1e-12


def test_advection_residual_is_exact_for_a_quadratic_on_interior_elements():
    """u = x^2 + xy - y lies in every element's space (p >= 2) and is continuous, so every jump
    vanishes with the exact trace and R = -beta . grad u at the points of elements away from the
    periodic seam (where u is discontinuous)."""
    n = 5
    mesh = _mesh(n, 0.0, 1.0, [2, 3, 4], 5)
    m = MixedDiscretisation(mesh, make_physics(ADV))
    U = []
    for e in range(mesh.nelem):
        x, y = _points(mesh, e).T
        U.append((x**2 + x * y - y)[:, None])
    uh = [m.to_face(*m.trace_sides[t, 0], U[m.trace_sides[t, 0, 0]]) for t in range(m.ntrace)]
    R, _ = m.full_residual(U, uh)
    for j in range(1, n - 1):
        for i in range(1, n - 1):
            e = i + n * j
            x, y = _points(mesh, e).T
            exact = -(1.0 * (2 * x + y) + 0.5 * (x - 1))
            assert np.abs(R[e][:, 0] - exact).max() < 1e-12


def test_conservation_with_the_solved_trace():
    """With g(u^) = 0 the common fluxes of both sides of every face cancel: sum_k int J R = 0."""
    mesh = _mesh(3, 0.0, 1.0, [2, 3, 4], 11, jitter=0.15)
    m = MixedDiscretisation(mesh, make_physics(ADVDIFF))
    rng = np.random.default_rng(1)
    U = [rng.standard_normal(((int(mesh.p[e]) + 1) ** 2, 1)) for e in range(mesh.nelem)]
    off = np.concatenate([[0], np.cumsum(m.trace_npts)])

    def unflat(v):
        return [v[off[t]:off[t + 1]][:, None] for t in range(m.ntrace)]

    g0 = trace_flatten(m.full_residual(U, unflat(np.zeros(off[-1])))[1])
    G = np.empty((off[-1], off[-1]))
    for k in range(off[-1]):  # g is affine in u^ for advection-diffusion
        ek = np.zeros(off[-1])
        ek[k] = 1.0
        G[:, k] = trace_flatten(m.full_residual(U, unflat(ek))[1]) - g0
    R, g = m.full_residual(U, unflat(np.linalg.solve(G, -g0)))
    assert np.abs(trace_flatten(g)).max() < 1e-12
    total = sum(np.sum(_quad_weights(m, e) * R[e][:, 0]) for e in range(mesh.nelem))
    scale = max(np.sum(_quad_weights(m, e) * np.abs(R[e][:, 0])) for e in range(mesh.nelem))
    assert abs(total) < 1e-13 * scale
    # without the trace solve the sum is not zero: the pin sees a wrong g
    R0, _ = m.full_residual(U, unflat(np.zeros(off[-1])))
    assert abs(sum(np.sum(_quad_weights(m, e) * R0[e][:, 0]) for e in range(mesh.nelem))) > 1e-6 * scale


@pytest.mark.parametrize("phys", [NS, ADVDIFF], ids=["ns", "advdiff"])
def test_condensed_newton_step_equals_the_monolithic_step(phys):
    """Static condensation, trace assembly over faces of unequal point counts and
    back-substitution give the Newton step of the dense system on [u; u^]."""
    n = 3
    band = np.zeros((n, n), bool)
    band[0:2, :] = True
    mesh = _mesh(n, 0.0, 1.0, [1, 2, 3], 7, implicit=band.reshape(-1))
    ph = dict(phys, mu=2e-2) if phys["kind"] == "ns" else phys
    m = MixedDiscretisation(mesh, make_physics(ph))
    rng = np.random.default_rng(2)
    base = np.array([1.0, 0.3, -0.2, 2.5])[: m.nv]
    U = [base + 0.05 * rng.standard_normal(((int(mesh.p[e]) + 1) ** 2, m.nv)) for e in range(mesh.nelem)]
    Ustar = [u + 0.01 * rng.standard_normal(u.shape) for u in U]
    uh = m.initial_trace(U)
    du1, dh1 = hybridized_step(m, U, uh, Ustar, 0.05)
    du2, dh2 = monolithic_step(m, U, uh, Ustar, 0.05)
    scale = max(np.abs(dh2).max(), max(np.abs(v).max() for v in du2.values()))
    assert scale > 1e-3
    assert np.abs(dh1 - dh2).max() < 1e-12 * scale
    assert max(np.abs(du1[e] - du2[e]).max() for e in du1) < 1e-12 * scale


# ------------------------------------ wall and far-field faces on a stretched mixed-degree wall band
from oracle.blocks import EPS  # noqa: E402
from oracle.boundary import BoundaryDiscretisation  # noqa: E402
from workloads.mesh import BC_FARFIELD, BC_WALL, geometric_nodes  # noqa: E402

NS_WALL = {"kind": "ns", "gamma": 1.4, "mu": 2e-2, "Pr": 0.72, "lref": 1.0}
REST = np.array([1.2, 0.0, 0.0, 2.0])
U_INF = np.array([1.0, 0.3, 0.05, 2.6])


def _bl_mesh(nx, degrees, imp_rows, bc_y, seed, h0=0.02, ratio=1.6, jitter=0.0):
    """Wall-normal geometric growth from h0 (a stretched boundary-layer band), periodic in x."""
    yn = geometric_nodes(h0, ratio, 0.25, 1.0)
    ny = len(yn) - 1
    imp = np.zeros((ny, nx), bool)
    imp[imp_rows, :] = True
    p = np.random.default_rng(seed).choice(degrees, size=nx * ny).astype(np.int32)
    return structured_quads(uniform_nodes(nx, 0.0, 1.0), yn, periodic=(True, False), jitter=jitter,
                            seed=seed, p=p, implicit=imp.reshape(-1), bc_y=bc_y)


def _trace_solve(m, U, uh):
    """Newton on g(u, u^) = 0 for u^ alone (dense complex-step Jacobian; tiny meshes)."""
    off = np.concatenate([[0], np.cumsum(m.trace_npts * m.nv)])

    def unflat(v):
        return [v[off[t]:off[t + 1]].reshape(-1, m.nv) for t in range(m.ntrace)]

    x = trace_flatten(uh)
    Uc = [u.astype(np.complex128) for u in U]
    for _ in range(30):
        g = trace_flatten(m.full_residual(U, unflat(x))[1])
        if np.abs(g).max() < 1e-13:
            return unflat(x)
        Jg = np.empty((x.size, x.size))
        for k in range(x.size):
            xp = x.astype(np.complex128)
            xp[k] += 1j * EPS
            Jg[:, k] = trace_flatten(m.full_residual(Uc, unflat(xp))[1]).imag / EPS
        x = x - np.linalg.solve(Jg, g)
    raise AssertionError("trace equations did not converge")


@pytest.mark.parametrize("rows", [[0, 1], list(range(8))], ids=["explicit_far_field", "implicit_far_field"])
def test_uniform_degree_with_walls_and_far_field_reduces_to_the_boundary_operator(rows):
    mesh = _bl_mesh(3, [3], rows, (BC_WALL, BC_FARFIELD), seed=1, jitter=0.1)
    assert mesh.ny == 8
    ph = make_physics(NS_WALL)
    d = BoundaryDiscretisation(mesh, ph, U_INF)
    m = MixedDiscretisation(mesh, ph, U_INF)
    rng = np.random.default_rng(0)
    U = np.tile(U_INF, (mesh.nelem, d.ns, 1)) * (1 + 1e-2 * rng.standard_normal((mesh.nelem, d.ns, 4)))
    uh = d.initial_trace(U) * (1 + 1e-2 * rng.standard_normal((d.ntrace, d.n, 4)))
    R, g = d.full_residual(U, uh)
    Rm, gm = m.full_residual(list(U), list(uh))
    assert np.abs(np.stack(Rm) - R).max() <= 1e-13 * np.abs(R).max()
    assert np.abs(np.stack(gm) - g).max() <= 1e-13 * np.abs(g).max()
    assert np.abs(np.stack(m.initial_trace(list(U))) - d.initial_trace(U)).max() < 1e-15


def test_rest_state_is_steady_on_a_stretched_mixed_degree_wall_band():
    mesh = _bl_mesh(4, [2, 3, 4, 5], [0, 1, 2], (BC_WALL, BC_FARFIELD), seed=2)
    assert len(set(mesh.p.tolist())) > 2
    m = MixedDiscretisation(mesh, make_physics(NS_WALL), REST)
    # boundary faces carry the element's own points; interior faces the higher degree's
    e_b, f_b = np.nonzero(m.bnd)
    assert len(e_b) == 2 * mesh.nx and np.all(m.nf[e_b, f_b] == m.n[e_b])
    e_i, f_i = np.nonzero(~m.bnd)
    assert np.all(m.nf[e_i, f_i] == np.maximum(m.n[e_i], m.n[mesh.nbr[e_i, f_i]]))
    U = [np.tile(REST, ((int(mesh.p[e]) + 1) ** 2, 1)) for e in range(mesh.nelem)]
    R, g = m.full_residual(U, m.initial_trace(U))
    # R carries 1/h: rounding of O(1) fluxes over the thinnest cells (h0 = 0.02)
    assert max(np.abs(r).max() for r in R) < 1e-12 / 0.02 and max(np.abs(x).max() for x in g) < 1e-12


def test_walls_conserve_mass_and_energy_across_unequal_degrees():
    mesh = _bl_mesh(3, [2, 3], [0, 4], (BC_WALL, BC_WALL), seed=3, ratio=1.0, h0=0.2)
    m = MixedDiscretisation(mesh, make_physics(NS_WALL))
    rng = np.random.default_rng(4)
    U = [REST + 0.05 * rng.standard_normal(((int(mesh.p[e]) + 1) ** 2, 4)) for e in range(mesh.nelem)]
    uh = _trace_solve(m, U, m.initial_trace(U))
    R, _ = m.full_residual(U, uh)
    total = sum(np.einsum("s,sv->v", _quad_weights(m, e), R[e]) for e in range(mesh.nelem))
    scale = sum(np.einsum("s,sv->v", _quad_weights(m, e), np.abs(R[e])) for e in range(mesh.nelem))
    assert abs(total[0]) < 1e-13 * scale[0] and abs(total[3]) < 1e-13 * scale[3]
    for t in range(m.ntrace):
        e, f = m.trace_sides[t, 0]
        if m.kind[e, f] == 3:  # wall: no-slip
            assert np.abs(uh[t][:, 1:3]).max() < 1e-14


def test_condensed_step_equals_the_monolithic_step_on_a_boundary_layer_band():
    mesh = _bl_mesh(3, [1, 2, 3], [0, 1], (BC_WALL, BC_FARFIELD), seed=5, ratio=2.0, h0=0.05)
    m = MixedDiscretisation(mesh, make_physics(NS_WALL), U_INF)
    rng = np.random.default_rng(6)
    U = [U_INF * (1 + 1e-2 * rng.standard_normal(((int(mesh.p[e]) + 1) ** 2, 4))) for e in range(mesh.nelem)]
    Ustar = [u + 1e-3 * rng.standard_normal(u.shape) for u in U]
    uh = m.initial_trace(U)
    du1, dh1 = hybridized_step(m, U, uh, Ustar, 0.03)
    du2, dh2 = monolithic_step(m, U, uh, Ustar, 0.03)
    scale = max(np.abs(dh2).max(), max(np.abs(v).max() for v in du2.values()))
    assert scale > 1e-3
    assert np.abs(dh1 - dh2).max() < 1e-12 * scale
    assert max(np.abs(du1[e] - du2[e]).max() for e in du1) < 1e-12 * scale
