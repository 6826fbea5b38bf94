"""Pins of the hexahedral FP64 oracle (the scheme of Secs. 2-4 on hexahedra, Sec. 5.3) against facts
fixed by geometry and mathematics: the trilinear map's volume and closed element surfaces,
free-stream preservation on skewed hexes, design-order convergence of the residual and of a
backward-Euler step, HFR reproducing upwind FR for linear advection, and the condensed Newton step
against the monolithic one."""

import math

import numpy as np
import pytest

from oracle.fr3d import Discretisation3D, condensed_newton_step, monolithic_newton_step
from oracle.physics import AdvectionDiffusion, NavierStokes2D, NavierStokes3D, make_physics
from workloads.mesh import structured_hexes, uniform_nodes

NS3 = make_physics({"kind": "ns3d", "gamma": 1.4, "mu": 2e-2, "Pr": 0.72})
U_INF = np.array([1.0, 0.3, -0.2, 0.1, 2.5])
BETA = (1.0, 0.5, 0.25)


def _hexes(n, p, imp=None, jitter=0.0, seed=0):
    nodes = [uniform_nodes(k, 0.0, 1.0) for k in n]
    return structured_hexes(*nodes, periodic=(True, True, True), jitter=jitter, seed=seed, p=p, implicit=imp)


def test_navier_stokes_3d_reduces_to_2d_for_planar_states():
    rng = np.random.default_rng(0)
    u2, q2 = np.array([1.1, 0.3, -0.2, 2.4]), rng.standard_normal((2, 4))
    u3 = np.array([1.1, 0.3, -0.2, 0.0, 2.4])
    q3 = np.zeros((3, 5))
    q3[:2, [0, 1, 2, 4]] = q2
    a, b = NavierStokes2D(mu=0.1), NavierStokes3D(mu=0.1)
    assert np.abs(b.conv(u3)[:2][:, [0, 1, 2, 4]] - a.conv(u2)).max() < 1e-15
    assert np.abs(b.visc(u3, q3)[:2][:, [0, 1, 2, 4]] - a.visc(u2, q2)).max() < 1e-15
    p = (1.4 - 1) * (2.4 - 0.5 * (0.3**2 + 0.2**2) / 1.1)
    assert np.allclose(b.conv(u3)[2], [0, 0, 0, p, 0])  # z-flux of a planar state: pressure only


def test_trilinear_volume_and_closed_element_surfaces():
    m = _hexes((3, 3, 3), 2, jitter=0.15, seed=1)
    d = Discretisation3D(m, NS3)
    assert abs(np.sum(d.wvol * d.J) - 1.0) < 1e-13  # periodic jitter tiles the unit box
    surf = np.einsum("q,efq,efqc->ec", d.wface, d.Jf, d.normal)
    assert np.abs(surf.sum(axis=1)).max() < 1e-14
    # an undisturbed cube of side h: J = h^3 / 8, face J_f = h^2 / 4, outward axis normals
    d = Discretisation3D(_hexes((2, 2, 2), 1), NS3)
    assert np.allclose(d.J, 0.5**3 / 8) and np.allclose(d.Jf, 0.25**2)
    assert np.allclose(d.normal[0, 5], [0, 0, 1]) and np.allclose(d.normal[0, 0], [-1, 0, 0])


def test_free_stream_is_preserved_on_skewed_hexes():
    imp = np.arange(27) % 3 != 0  # implicit and explicit elements mixed: all three face kinds
    for p in (2, 3):
        d = Discretisation3D(_hexes((3, 3, 3), p, imp=imp, jitter=0.15, seed=1), NS3)
        U = np.tile(U_INF, (27, d.ns, 1))
        R, g = d.full_residual(U, d.initial_trace(U))
        assert np.abs(R).max() < 1e-12 and np.abs(g).max() < 1e-12


def test_residual_converges_at_design_order_on_smooth_field():
    errs = []
    for n in (4, 8, 16):
        d = Discretisation3D(_hexes((n, n, n), 2), AdvectionDiffusion(BETA, 0.0))
        x, y, z = (d.xyz[..., c] for c in range(3))
        k = 2 * np.pi
        U = np.sin(k * x) * np.cos(k * y) * np.sin(k * z)
        exact = -(BETA[0] * k * np.cos(k * x) * np.cos(k * y) * np.sin(k * z)
                  - BETA[1] * k * np.sin(k * x) * np.sin(k * y) * np.sin(k * z)
                  + BETA[2] * k * np.sin(k * x) * np.cos(k * y) * np.cos(k * z))
        R, _ = d.full_residual(U[..., None], d.initial_trace(U[..., None]))
        errs.append(np.abs(R[..., 0] - exact).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.9), rates  # >= p


def test_backward_euler_spatial_convergence_p_plus_one():
    """One hybridized BE step of a Fourier mode (advection-diffusion: one Newton step solves it)
    against the continuous-in-space BE solution converges at p + 1 = 3."""
    nu, dt = 0.01, 0.05
    kv = np.array([1, 1, 1])
    errs, hs = [], []
    for n in (4, 8):
        d = Discretisation3D(_hexes((n, n, n), 2), AdvectionDiffusion(BETA, nu))
        phase = 2 * np.pi * (d.xyz @ kv)
        U0 = np.cos(phase)[..., None]
        lam = 2j * np.pi * np.dot(BETA, kv) + 4 * np.pi**2 * nu * np.dot(kv, kv)
        exact = np.real(np.exp(1j * phase) / (1 + dt * lam))
        dU, _ = condensed_newton_step(d, U0, d.initial_trace(U0), U0, dt)
        errs.append(math.sqrt(np.sum(d.wvol * d.J * ((U0 + dU)[..., 0] - exact) ** 2)))
        hs.append(1.0 / n)
    rate = math.log(errs[0] / errs[1]) / math.log(hs[0] / hs[1])
    # 2.69 measured on this pre-asymptotic pair (the 2D oracle's first pair gives 2.87, then 3.24);
    # an order-losing slip (inconsistent lift or flux) drops it to 2 or below
    assert rate > 2.6, (errs, rate)


def test_hfr_backward_euler_equals_upwind_fr_for_linear_advection():
    """With nu = 0 and s = |beta . n| the pointwise transmission condition makes the trace the
    upwind state, so the all-hybridized BE step equals the implicit BE step of upwind FR."""
    m = _hexes((2, 3, 2), 2, jitter=0.1, seed=3)
    ad = AdvectionDiffusion(BETA, 0.0)
    dh = Discretisation3D(m, ad)
    rng = np.random.default_rng(2)
    U0 = rng.standard_normal((m.nelem, dh.ns, 1))
    dt = 0.07
    dU, _ = condensed_newton_step(dh, U0, dh.initial_trace(U0), U0, dt)
    m.implicit = np.zeros(m.nelem, bool)  # the same mesh with FR faces everywhere
    df = Discretisation3D(m, ad)
    N = U0.size
    R0, _ = df.full_residual(np.zeros_like(U0), np.zeros((0, df.nfp, 1)))
    M = np.zeros((N, N))  # R is linear: R(U) = M U
    for j in range(N):
        ej = np.zeros(N)
        ej[j] = 1.0
        M[:, j] = df.full_residual(ej.reshape(U0.shape), np.zeros((0, df.nfp, 1)))[0].reshape(-1) - R0.reshape(-1)
    U_fr = np.linalg.solve(np.eye(N) - dt * M, U0.reshape(-1))
    assert np.abs(U0.reshape(-1) + dU.reshape(-1) - U_fr).max() < 1e-12 * np.abs(U_fr).max()


def test_condensed_step_equals_the_monolithic_step_navier_stokes():
    imp = np.array([1, 1, 0, 1, 1, 1, 0, 1, 1, 1, 0, 1], bool)
    m = _hexes((3, 2, 2), 1, imp=imp, jitter=0.1, seed=2)
    d = Discretisation3D(m, NS3)
    rng = np.random.default_rng(0)
    U = np.tile(U_INF, (m.nelem, d.ns, 1)) * (1 + 1e-2 * rng.standard_normal((m.nelem, d.ns, 5)))
    Ustar = U + 1e-3 * rng.standard_normal(U.shape)
    uh = d.initial_trace(U)
    a = condensed_newton_step(d, U, uh, Ustar, 0.03)
    b = monolithic_newton_step(d, U, uh, Ustar, 0.03)
    scale = max(np.abs(b[0]).max(), np.abs(b[1]).max())
    assert scale > 1e-3
    assert max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max()) < 1e-12 * scale


def test_lift_is_the_dg_lifting_of_each_face():
    """DG-recovering corrections on Gauss points: for every polynomial phi of the element's tensor
    space and face values V on face f, sum_i W_i phi_i lift(V)_i = s sum_m w_m phi(x_m) V_m with
    s = 1 in the divergence (signed) form and s = sigma_f, the face's outward sign, in the gradient
    form; checked with random phi and V on every face."""
    d = Discretisation3D(_hexes((2, 2, 2), 3), NS3)
    rng = np.random.default_rng(7)
    phi = rng.standard_normal((1, d.ns))
    phif = d.interp_faces(phi)[0]  # (6, n^2): phi at each face's points
    for f in range(6):
        V = np.zeros((1, 6, d.nfp))
        V[0, f] = rng.standard_normal(d.nfp)
        sg = (-1.0, 1.0)[f % 2]
        for signed in (False, True):
            L = d.lift(V, signed)
            lhs = sum(np.sum(d.wvol * phi[0] * L[k][0]) for k in range(3))
            rhs = (1.0 if signed else sg) * np.sum(d.wface * phif[f] * V[0, f])
            assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(rhs))
            assert np.abs(L[(f // 2 + 1) % 3][0]).max() == 0.0  # nothing along the other axes


def test_trace_residuals_sum_to_the_net_element_flux():
    """For any state and trace on a fully implicit mesh, sum of g = -sum_k int J R_k: the lift
    integrates each face's J_f F^.n with the face rule, and g weights it with the same rule."""
    m = _hexes((2, 3, 2), 2, jitter=0.15, seed=5)
    for phys in (AdvectionDiffusion(BETA, 0.02), NS3):
        d = Discretisation3D(m, phys)
        rng = np.random.default_rng(3)
        base = np.zeros(1) if d.nv == 1 else U_INF
        U = base + 0.1 * rng.standard_normal((m.nelem, d.ns, d.nv))
        uh = d.initial_trace(U) + 0.05 * rng.standard_normal((d.ntrace, d.nfp, d.nv))
        R, g = d.full_residual(U, uh)
        total = np.einsum("s,es,esv->v", d.wvol, d.J, R)
        assert np.abs(g.sum(axis=(0, 1)) + total).max() < 1e-12 * np.abs(g).sum()


# ------------------------------------------------- walls in a tanh-clustered hexahedral channel
from oracle.blocks import EPS  # noqa: E402
from oracle.boundary import WALL_FACE, BoundaryDiscretisation  # noqa: E402
from workloads.mesh import BC_FARFIELD, BC_WALL, structured_quads, tanh_nodes  # noqa: E402

REST3 = np.array([1.2, 0.0, 0.0, 0.0, 2.0])


def _channel(nx, ny, nz, p, imp_layers, bc_y=(BC_WALL, BC_WALL), yn=None):
    """Box periodic in x and z, walls at y = -1, 1 with tanh clustering (beta = 2.5)."""
    yn = tanh_nodes(ny, 2.5) if yn is None else yn
    imp = np.zeros((nz, ny, nx), bool)
    imp[:, imp_layers, :] = True
    return structured_hexes(uniform_nodes(nx, 0, 2 * np.pi), yn, uniform_nodes(nz, 0, np.pi),
                            periodic=(True, False, True), p=p, implicit=imp.reshape(-1), bc_y=bc_y)


@pytest.mark.parametrize("rows", [[True, True, True, False], [True] * 4], ids=["explicit_top", "all_implicit"])
def test_planar_states_reduce_to_the_2d_boundary_operator(rows):
    """One periodic element in z, a z-invariant state with w = 0: every z-slice of the 3D residual is
    the 2D residual with walls below and far field above (explicit or implicit far-field elements)."""
    nx, p = 3, 2
    yn = np.array([0.0, 0.05, 0.2, 0.5, 1.0])
    imp = np.repeat(rows, nx)
    ns2 = structured_quads(uniform_nodes(nx, 0, 1), yn, periodic=(True, False), p=p,
                           implicit=imp, bc_y=(BC_WALL, BC_FARFIELD))
    m3 = structured_hexes(uniform_nodes(nx, 0, 1), yn, uniform_nodes(1, 0, 0.3), periodic=(True, False, True),
                          p=p, implicit=imp, bc_y=(BC_WALL, BC_FARFIELD))
    u2inf = np.array([1.0, 0.3, 0.05, 2.6])
    u3inf = np.array([1.0, 0.3, 0.05, 0.0, 2.6])
    ph2 = NavierStokes2D(mu=2e-2)
    d2 = BoundaryDiscretisation(ns2, ph2, u2inf)
    d3 = Discretisation3D(m3, NavierStokes3D(mu=2e-2), u3inf)
    rng = np.random.default_rng(0)
    U2 = np.tile(u2inf, (ns2.nelem, d2.ns, 1)) * (1 + 1e-2 * rng.standard_normal((ns2.nelem, d2.ns, 4)))
    uh2 = d2.initial_trace(U2) * (1 + 1e-2 * rng.standard_normal((d2.ntrace, d2.n, 4)))
    n = p + 1
    U3 = np.zeros((m3.nelem, d3.ns, 5))
    for c in range(n):
        U3[:, c * n * n:(c + 1) * n * n][..., [0, 1, 2, 4]] = U2
    uh3 = d3.initial_trace(U3)
    for t in range(d3.ntrace):
        e, f = d3.trace_sides[t, 0]
        if f < 4:  # x and y faces: 2D face point i, repeated along z
            uh3[t][:, [0, 1, 2, 4]] = np.tile(uh2[d2.tr_of[e, f]], (n, 1))
    R2, g2 = d2.full_residual(U2, uh2)
    R3, g3 = d3.full_residual(U3, uh3)
    for c in range(n):
        sl = R3[:, c * n * n:(c + 1) * n * n]
        assert np.abs(sl[..., [0, 1, 2, 4]] - R2).max() < 1e-12 * np.abs(R2).max()
        assert np.abs(sl[..., 3]).max() < 1e-12 * np.abs(R2).max()
    # trace rows of x and y faces: the 2D rows times the z weight and the z half-length
    wz = d3.ref.w * 0.3 / 2
    for t in range(d3.ntrace):
        e, f = d3.trace_sides[t, 0]
        if f < 4:
            exp = np.kron(wz[:, None], np.ones((n, 1))) * np.tile(g2[d2.tr_of[e, f]], (n, 1))
            assert np.abs(g3[t][:, [0, 1, 2, 4]] - exp).max() < 1e-12 * np.abs(g2).max()


def test_rest_state_is_steady_in_a_wall_clustered_channel():
    m = _channel(2, 6, 2, 3, [0, 5])
    d = Discretisation3D(m, NavierStokes3D(mu=2e-2))
    assert np.sum(d.kind == WALL_FACE) == 2 * 2 * 2
    U = np.tile(REST3, (m.nelem, d.ns, 1))
    R, g = d.full_residual(U, d.initial_trace(U))
    hmin = np.diff(tanh_nodes(6, 2.5)).min()
    assert np.abs(R).max() < 1e-12 / hmin and np.abs(g).max() < 1e-12


def test_walls_conserve_mass_and_energy_in_3d():
    m = _channel(2, 4, 2, 1, [0, 3])
    d = Discretisation3D(m, NavierStokes3D(mu=2e-2))
    rng = np.random.default_rng(1)
    U = REST3 + 0.05 * rng.standard_normal((m.nelem, d.ns, 5))
    uh = d.initial_trace(U)
    for _ in range(20):  # Newton on g(u, u^) = 0 for u^ alone
        _, g = d.full_residual(U, uh)
        if np.abs(g).max() < 1e-13:
            break
        Jg = np.empty((uh.size, uh.size))
        for k in range(uh.size):
            hp = uh.astype(np.complex128)
            hp.reshape(-1)[k] += 1j * EPS
            Jg[:, k] = d.full_residual(U.astype(np.complex128), hp)[1].imag.reshape(-1) / EPS
        uh = uh - np.linalg.solve(Jg, g.reshape(-1)).reshape(uh.shape)
    R, g = d.full_residual(U, uh)
    assert np.abs(g).max() < 1e-13
    total = np.einsum("s,es,esv->v", d.wvol, d.J, R)
    scale = np.einsum("s,es,esv->v", d.wvol, d.J, np.abs(R))
    assert abs(total[0]) < 1e-13 * scale[0] and abs(total[4]) < 1e-13 * scale[4]
    assert abs(total[1]) > 1e-6 * scale[1]  # wall shear: momentum is not conserved
    walls = [t for t in range(d.ntrace) if d.trace_sides[t, 1, 0] < 0]
    assert len(walls) == 8 and np.abs(uh[walls][..., 1:4]).max() < 1e-14


def test_condensed_step_equals_the_monolithic_step_with_walls_3d():
    m = _channel(2, 3, 2, 1, [0, 2])
    d = Discretisation3D(m, NavierStokes3D(mu=2e-2))
    rng = np.random.default_rng(2)
    U = REST3 + np.array([0, 0.1, 0.05, 0.02, 0]) + 0.02 * rng.standard_normal((m.nelem, d.ns, 5))
    Ustar = U + 1e-3 * rng.standard_normal(U.shape)
    uh = d.initial_trace(U)
    a = condensed_newton_step(d, U, uh, Ustar, 0.02)
    b = monolithic_newton_step(d, U, uh, Ustar, 0.02)
    scale = max(np.abs(b[0]).max(), np.abs(b[1]).max())
    assert scale > 1e-4
    assert max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max()) < 1e-12 * scale
