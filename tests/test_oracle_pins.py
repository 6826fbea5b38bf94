"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand) fails at least one of them.
"""

import math
import os

import numpy as np
import pytest

from oracle.basis import RefElement1D, gauss_legendre, lagrange, lagrange_derivative, radau_corrections
from oracle.blocks import element_blocks, global_jacobian, EPS
from oracle.fr import Discretisation
from oracle.geometry import QuadGeometry
from oracle.physics import AdvectionDiffusion, NavierStokes2D
from oracle.solve import condense, solve_trace, backsolve
from oracle.stepping import TABLEAUX, imex_step, newton_stage
from workloads.mesh import structured_quads, uniform_nodes
from workloads.states import sample_points, isentropic_vortex, freestream

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- reference element
def test_gauss_legendre_closed_forms_and_exactness():
    x, w = gauss_legendre(2)
    assert np.allclose(x, [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-15)
    assert np.allclose(w, [1.0, 1.0], atol=1e-15)
    x, w = gauss_legendre(3)
    assert np.allclose(x, [-math.sqrt(0.6), 0.0, math.sqrt(0.6)], atol=1e-15)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)
    for n in range(1, 8):
        x, w = gauss_legendre(n)
        for k in range(2 * n):  # exact to degree 2n-1
            exact = 0.0 if k % 2 else 2.0 / (k + 1)
            assert abs(np.sum(w * x**k) - exact) < 1e-14
        xr, wr = np.polynomial.legendre.leggauss(n)  # independent library rule
        assert np.allclose(x, xr, atol=1e-15) and np.allclose(w, wr, atol=1e-14)


def test_lagrange_interpolates_and_differentiates_polynomials():
    for p in range(1, 6):
        x, _ = gauss_legendre(p + 1)
        t = np.linspace(-1, 1, 11)
        L = lagrange(x, t)
        D = lagrange_derivative(x, x)
        for k in range(p + 1):
            assert np.allclose(L @ x**k, t**k, atol=1e-13)
            dk = k * x ** max(k - 1, 0) if k else 0 * x
            assert np.allclose(D @ x**k, dk, atol=1e-12)


def test_radau_corrections_end_values_and_dg_identity():
    for p in range(1, 7):
        gL, _, gR, _ = radau_corrections(p, np.array([-1.0, 1.0]))
        assert np.allclose(gL, [1.0, 0.0], atol=1e-14)
        assert np.allclose(gR, [0.0, 1.0], atol=1e-14)
        ref = RefElement1D(p)
        # DG-recovering FR on Gauss points is nodal DG: g_R'(x_i) = l_i(1)/w_i
        assert np.allclose(ref.dgR, ref.lp / ref.w, atol=1e-12)
        assert np.allclose(ref.dgL, -ref.lm / ref.w, atol=1e-12)


# ------------------------------------------------------------------------ geometry
def test_geometry_area_and_normals():
    mesh = structured_quads(uniform_nodes(4, 0, 2), uniform_nodes(3, 0, 1), jitter=0.2, seed=5, p=3)
    ref = RefElement1D(3)
    geo = QuadGeometry(mesh.verts, ref)
    W = np.outer(ref.w, ref.w).reshape(-1)  # pt = a + n b -> w_a w_b
    area = np.einsum("s,es->e", W, geo.J)
    v = mesh.verts
    quad = v[:, [0, 1, 3, 2]]  # counter-clockwise corner order
    shoelace = 0.5 * np.sum(quad[:, :, 0] * np.roll(quad[:, :, 1], -1, 1) - np.roll(quad[:, :, 0], -1, 1) * quad[:, :, 1], axis=1)
    assert np.allclose(area, shoelace, atol=1e-13)
    assert np.allclose(np.linalg.norm(geo.normal, axis=-1), 1.0)
    # shared faces: equal J_f, opposite normals
    nb, nf = mesh.nbr, mesh.nbr_face
    assert np.allclose(geo.Nf, -geo.Nf[nb, nf], atol=1e-13)
    # outward: normal of face 1 (xi=+1) of an undistorted cell is +x
    mesh0 = structured_quads(uniform_nodes(2, 0, 1), uniform_nodes(2, 0, 1), p=2)
    g0 = QuadGeometry(mesh0.verts, RefElement1D(2))
    assert np.allclose(g0.normal[:, 1], [1.0, 0.0]) and np.allclose(g0.normal[:, 2], [0.0, -1.0])
    assert np.allclose(g0.Jf[:, 0], 0.25)  # half the edge length 0.5


# ------------------------------------------------------------------------- physics
def test_euler_flux_values_and_rotation_invariance():
    ns = NavierStokes2D(gamma=1.4, mu=0.0)
    rho, u, v, p = 1.3, 0.7, -0.4, 2.1
    E = p / 0.4 + 0.5 * rho * (u * u + v * v)
    U = np.array([rho, rho * u, rho * v, E])
    F = ns.conv(U)
    assert np.allclose(F[0], [rho * u, rho * u * u + p, rho * u * v, (E + p) * u])
    assert np.allclose(F[1], [rho * v, rho * u * v, rho * v * v + p, (E + p) * v])
    th = 0.37
    n = np.array([math.cos(th), math.sin(th)])
    T = np.array([[1, 0, 0, 0], [0, n[0], n[1], 0], [0, -n[1], n[0], 0], [0, 0, 0, 1]])
    Fn = np.einsum("cv,c->v", F, n)
    assert np.allclose(T.T @ ns.conv(T @ U)[0], Fn)
    c = math.sqrt(1.4 * p / rho)
    assert np.isclose(ns.wave_speed(U, n), abs(u * n[0] + v * n[1]) + c)


def test_navier_stokes_viscous_flux_shear_and_conduction():
    mu, Pr, g = 0.01, 0.72, 1.4
    ns = NavierStokes2D(gamma=g, mu=mu, Pr=Pr)
    rho, u, v, p = 1.0, 0.3, 0.0, 1.0
    E = p / (g - 1) + 0.5 * rho * u * u
    U = np.array([rho, rho * u, 0.0, E])
    # simple shear du/dy = 2 at constant rho, p: tau_xy = mu * 2
    q = np.zeros((2, 4))
    q[1, 1] = rho * 2.0
    q[1, 3] = rho * u * 2.0  # dE/dy = rho u du/dy keeps p constant
    F = ns.visc(U, q)
    assert np.allclose(F[1, 1], 2 * mu) and np.allclose(F[0, 2], 2 * mu)
    assert np.allclose(F[0, 1], 0.0) and np.allclose(F[1, 2], 0.0)
    assert np.isclose(F[1, 3], u * 2 * mu)  # work of the shear stress, no heat flux
    # pure conduction: dT/dx = 1 at rest with rho fixed: dE/dx = rho / (g - 1)
    U = np.array([1.0, 0.0, 0.0, 1.0 / (g - 1)])
    q = np.zeros((2, 4))
    q[0, 3] = 1.0 / (g - 1)
    F = ns.visc(U, q)
    kappa = mu * g / ((g - 1) * Pr)
    assert np.isclose(F[0, 3], kappa) and np.allclose(F[:, :3], 0.0)


# ------------------------------------------------------------- residual properties
def _ns_disc(n=4, p=3, jitter=0.0, seed=0, mu=5e-5, implicit=None):
    mesh = structured_quads(uniform_nodes(n, 0, 10), uniform_nodes(n, 0, 10), jitter=jitter,
                            seed=seed, p=p, implicit=implicit)
    return Discretisation(mesh, NavierStokes2D(1.4, mu, 0.72)), mesh


def test_free_stream_preservation_on_skewed_quads():
    for implicit in (None, np.arange(16) % 3 == 0):
        d, mesh = _ns_disc(jitter=0.2, seed=7, implicit=implicit)
        U = freestream((mesh.nelem, d.ns), mach=0.4, angle=0.3)
        R, g = d.full_residual(U, d.initial_trace(U))
        assert np.abs(R).max() < 1e-12 and np.abs(g).max() < 1e-12


def test_residual_converges_at_design_order_on_smooth_field():
    # linear advection, nu=0: R(u) -> -beta.grad u at the solution points
    errs = []
    for n in (4, 8, 16):
        mesh = structured_quads(uniform_nodes(n, 0, 1), uniform_nodes(n, 0, 1), p=3)
        d = Discretisation(mesh, AdvectionDiffusion((1.0, 0.5), 0.0))
        xy = d.geo.xy
        k = 2 * np.pi
        U = np.sin(k * xy[..., 0]) * np.cos(k * xy[..., 1])
        exact = -(1.0 * k * np.cos(k * xy[..., 0]) * np.cos(k * xy[..., 1])
                  - 0.5 * k * np.sin(k * xy[..., 0]) * np.sin(k * xy[..., 1]))
        R, _ = d.full_residual(U[..., None], d.initial_trace(U[..., None]))
        errs.append(np.abs(R[..., 0] - exact).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.7), rates  # >= p for the residual of a p=3 scheme


def test_backward_euler_spatial_convergence_p_plus_one():
    """C1 physics: error of one hybridized BE step against the continuous-in-space
    BE solution of a Fourier mode converges at p+1 = 3."""
    beta, nu, dt = (1.0, 0.5), 0.01, 0.05
    kx, ky = 1, 2
    errs = []
    for n in (8, 16, 32):
        mesh = structured_quads(uniform_nodes(n, 0, 1), uniform_nodes(n, 0, 1), p=2)
        d = Discretisation(mesh, AdvectionDiffusion(beta, nu))
        xy = d.geo.xy
        phase = 2 * np.pi * (kx * xy[..., 0] + ky * xy[..., 1])
        U0 = np.cos(phase)[..., None]
        lam = 2j * np.pi * (beta[0] * kx + beta[1] * ky) + 4 * np.pi**2 * nu * (kx * kx + ky * ky)
        exact = np.real(np.exp(1j * phase) / (1 + dt * lam))
        U1, _, info = newton_stage(d, U0, U0, d.initial_trace(U0), dt, tol=1e-13)
        W = np.outer(d.ref.w, d.ref.w).reshape(-1)
        errs.append(math.sqrt(np.sum(W * d.geo.J * (U1[..., 0] - exact) ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.8), (errs, rates)


# ---------------------------------------------------------------- Jacobian blocks
def test_blocks_match_central_differences_and_vanish_off_trace():
    d, mesh = _ns_disc(n=3, p=2, jitter=0.1, seed=2, mu=1e-2)
    U = isentropic_vortex(d.geo.xy)
    uh = d.initial_trace(U) * (1 + 1e-3 * np.sin(np.arange(d.ntrace))[:, None, None])
    a_dt = 0.03
    A, B, C, D = element_blocks(d, U, uh, a_dt)
    rng = np.random.default_rng(0)
    view = d.trace_view(uh)
    eps = 1e-6
    for _ in range(6):
        j = rng.integers(A.shape[1])
        pt, v = divmod(j, d.nv)
        Up, Um = U.copy(), U.copy()
        Up[:, pt, v] += eps
        Um[:, pt, v] -= eps
        Rp, Fp = d.residual(Up, view)
        Rm, Fm = d.residual(Um, view)
        fdA = -a_dt * (Rp - Rm).reshape(len(U), -1) / (2 * eps)
        fdA[:, j] += 1.0
        assert np.abs(fdA - A[:, :, j]).max() < 1e-7 * max(1.0, np.abs(A).max())
        fdC = (d.trace_weights(Fp) - d.trace_weights(Fm)).reshape(len(U), -1) / (2 * eps)
        assert np.abs(fdC - C[:, :, j]).max() < 1e-6 * np.abs(C).max()
        l = rng.integers(B.shape[2])
        fm, v = divmod(l, d.nv)
        f, m = divmod(fm, d.n)
        Vp, Vm = view.copy(), view.copy()
        Vp[:, f, m, v] += eps
        Vm[:, f, m, v] -= eps
        Rp, Fp = d.residual(U, Vp)
        Rm, Fm = d.residual(U, Vm)
        fdB = -a_dt * (Rp - Rm).reshape(len(U), -1) / (2 * eps)
        assert np.abs(fdB - B[:, :, l]).max() < 1e-6 * np.abs(B).max()
        fdD = (d.trace_weights(Fp) - d.trace_weights(Fm)).reshape(len(U), -1) / (2 * eps)
        assert np.abs(fdD - D[:, :, l]).max() < 1e-6 * np.abs(D).max()
    # A -> I as dt -> 0
    A0, B0, _, _ = element_blocks(d, U, uh, 0.0)
    assert np.allclose(A0, np.eye(A.shape[1])[None]) and np.allclose(B0, 0.0)


def _hybrid_vs_monolithic(d, U, uh, a_dt):
    imp = d.imp_idx
    Jm = global_jacobian(d, U, uh, a_dt)
    R, Fn = d.residual(U, d.trace_view(uh))
    h = -a_dt * R[imp]
    gv = d.trace_weights(Fn)
    g = d.assemble_trace(gv)
    x = np.linalg.solve(Jm, -np.concatenate([h.reshape(-1), g.reshape(-1)]))
    A, B, C, D = element_blocks(d, U, uh, a_dt)
    nA, nT = A.shape[1], B.shape[2]
    XB, xr, S, t = condense(A[imp], B[imp], C[imp], D[imp], -h.reshape(-1, nA), -gv[imp].reshape(-1, nT))
    duh, _, _ = solve_trace(d, S, t, imp, method="direct")
    du = backsolve(XB, xr, d.trace_view(duh.reshape(d.ntrace, d.n, d.nv))[imp].reshape(-1, nT))
    xc = np.concatenate([du.reshape(-1), duh])
    return np.abs(xc - x).max() / np.abs(x).max()


def test_hybridized_solve_equals_monolithic_advdiff_c1():
    from workloads import make_config
    from oracle.physics import make_physics
    w = make_config("advdiff8")
    d = Discretisation(w.mesh, make_physics(w.physics))
    err = _hybrid_vs_monolithic(d, w.u0, d.initial_trace(w.u0), w.dt)
    assert err < 1e-12


def test_hybridized_solve_equals_monolithic_navier_stokes():
    d, mesh = _ns_disc(n=4, p=3)
    U = isentropic_vortex(d.geo.xy)
    err = _hybrid_vs_monolithic(d, U, d.initial_trace(U), 0.04)
    assert err < 1e-12


def test_hfr_equals_fr_upwind_for_linear_advection():
    """End of Sec. 4 / Sec. 5.1: with discontinuous traces the transmission
    conditions are pointwise and HFR reproduces standard FR (upwind) for linear
    advection."""
    n, p, dt = 5, 2, 0.05
    ph = AdvectionDiffusion((1.0, 0.5), 0.0)
    mesh = structured_quads(uniform_nodes(n, 0, 1), uniform_nodes(n, 0, 1), p=p)
    d = Discretisation(mesh, ph)
    xy = d.geo.xy
    U0 = np.exp(-20 * ((xy[..., 0] - 0.5) ** 2 + (xy[..., 1] - 0.4) ** 2))[..., None]
    U1, _, _ = newton_stage(d, U0, U0, d.initial_trace(U0), dt, tol=1e-14)
    mesh_ex = structured_quads(uniform_nodes(n, 0, 1), uniform_nodes(n, 0, 1), p=p,
                               implicit=np.zeros(n * n, bool))
    de = Discretisation(mesh_ex, ph)
    N = U0.size
    Jfr = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N, complex)
        e[j] = 1j * EPS
        R, _ = de.full_residual(e.reshape(U0.shape), np.zeros((0, p + 1, 1)))
        Jfr[:, j] = R.imag.reshape(-1) / EPS
    Ufr = np.linalg.solve(np.eye(N) - dt * Jfr, U0.reshape(-1))
    assert np.abs(Ufr - U1.reshape(-1)).max() < 1e-13


def test_gmres_matches_direct_solve():
    d, mesh = _ns_disc(n=4, p=2, mu=1e-3)
    U = isentropic_vortex(d.geo.xy)
    uh = d.initial_trace(U)
    imp = d.imp_idx
    A, B, C, D = element_blocks(d, U, uh, 0.05)
    R, Fn = d.residual(U, d.trace_view(uh))
    nA, nT = A.shape[1], B.shape[2]
    XB, xr, S, t = condense(A, B, C, D, (0.05 * R).reshape(-1, nA), -d.trace_weights(Fn).reshape(-1, nT))
    x0, _, _ = solve_trace(d, S, t, imp, method="direct")
    x1, its, rel = solve_trace(d, S, t, imp, method="gmres", rtol=1e-12)
    assert rel <= 1e-12 and its > 1
    assert np.abs(x1 - x0).max() <= 1e-9 * np.abs(x0).max()


def test_newton_converges_quadratically():
    d, mesh = _ns_disc(n=4, p=3, mu=1e-3)
    U = isentropic_vortex(d.geo.xy)
    _, _, info = newton_stage(d, U, U, d.initial_trace(U), 0.1, tol=1e-13)
    h = np.array(info["history"]) / info["history"][0]
    assert info["converged"]
    # e_{k+1} <= C e_k^2 once in the asymptotic range
    k = np.nonzero(h < 1e-2)[0][0]
    assert h[k + 1] < 50 * h[k] ** 2


# ---------------------------------------------------------------- time stepping
def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            vals[tuple(parts[:-1])] = float(parts[-1])
    return vals


def test_sdirk2_tableau_matches_paper():
    g = _read_golden("sdirk2_tableau.txt")
    t = TABLEAUX["sdirk2"]
    assert np.isclose(t["a"][0, 0], g[("a11",)], atol=1e-15)
    assert np.isclose(t["a"][1, 0], g[("a21",)], atol=1e-15)
    assert np.isclose(t["a"][1, 1], g[("a22",)], atol=1e-15)
    assert np.isclose(t["b"][0], g[("b1",)], atol=1e-15) and np.isclose(t["b"][1], g[("b2",)], atol=1e-15)
    for name, tab in TABLEAUX.items():
        a, b, ah, bh = tab["a"], tab["b"], tab["ahat"], tab["bhat"]
        c = a.sum(1)
        ch = ah.sum(1)
        assert np.isclose(b.sum(), 1) and np.isclose(bh.sum(), 1)
        assert np.allclose(ch[1:], c)  # c_hat = [0 c] (Table butcherimex)
        assert np.allclose(bh[1:], b) and bh[0] == 0.0  # conservative pairing
        if name == "sdirk2":
            assert np.isclose(b @ c, 0.5) and np.isclose(bh @ ch, 0.5)


def _band_problem(n=8, p=2):
    imp = np.zeros((n, n), bool)
    imp[3:5, :] = True
    mesh = structured_quads(uniform_nodes(n, 0, 1), uniform_nodes(n, 0, 1), p=p, implicit=imp.reshape(-1))
    d = Discretisation(mesh, AdvectionDiffusion((1.0, 0.5), 0.01))
    xy = d.geo.xy
    U0 = np.exp(-20 * ((xy[..., 0] - 0.5) ** 2 + (xy[..., 1] - 0.4) ** 2))[..., None]
    return d, U0


def test_imex_step_conserves_across_interface():
    d, U0 = _band_problem()
    W = np.outer(d.ref.w, d.ref.w).reshape(-1)
    U1, _, _ = imex_step(d, U0, d.initial_trace(U0), 0.01, "sdirk2", tol=1e-13)
    m0 = np.sum(W * d.geo.J * U0[..., 0])
    m1 = np.sum(W * d.geo.J * U1[..., 0])
    assert abs(m1 - m0) < 1e-14 * abs(m0) + 1e-15
    # Navier-Stokes band: conserved to the Newton tolerance
    imp = np.zeros((6, 6), bool)
    imp[2:4, :] = True
    dn, mesh = _ns_disc(n=6, p=2, mu=5e-3, implicit=imp.reshape(-1))
    U = isentropic_vortex(dn.geo.xy)
    W = np.outer(dn.ref.w, dn.ref.w).reshape(-1)
    U1, _, _ = imex_step(dn, U, dn.initial_trace(U), 0.05, "sdirk2", tol=1e-12)
    dm = np.einsum("s,es,esv->v", W, dn.geo.J, U1 - U)
    assert np.abs(dm).max() < 1e-11


@pytest.mark.slow
def test_imex32_second_order_in_time():
    gold = _read_golden("imex32_orders.txt")
    d, U0 = _band_problem(n=6, p=2)
    W = np.outer(d.ref.w, d.ref.w).reshape(-1)
    T = 0.008

    def run(dt):
        U, uh = U0.copy(), d.initial_trace(U0)
        for _ in range(int(round(T / dt))):
            U, uh, _ = imex_step(d, U, uh, dt, "sdirk2", tol=1e-13)
        return U

    # self-convergence: differences of successive halvings shrink by 2^order
    sols = [run(dt) for dt in (0.002, 0.001, 0.0005, 0.00025)]
    diffs = [math.sqrt(np.sum(W * d.geo.J * (sols[k] - sols[k + 1])[..., 0] ** 2)) for k in range(3)]
    orders = np.log2(np.array(diffs[:-1]) / np.array(diffs[1:]))
    for o in orders:
        assert abs(o - gold[("dt", "0.005", "order")]) < 0.15, orders


def test_euler_vortex_residual_converges_at_design_order():
    """Navier-Stokes path with mu = 0 (Euler) on the moving isentropic vortex, whose exact time
    derivative is -M du/dx (translation at the free-stream velocity; du/dx by complex step of the
    closed-form state).  The vortex sits in the middle of a 20 x 20 periodic box, so its tails
    (exp(-49.5)) leave the periodic seams exact.  On 20, 40, 80 quads per side:
    * the L2 error of R(u) at the solution points converges at p, the order of a flux divergence
      built from degree-p interpolants, for FR (all explicit) and HFR (all implicit, trace = the
      average of the two sides' states) alike;
    * tested against a fixed smooth function the error converges at least at p + 1, the design
      order of the solution (observed: p + 2 and more).
    A dropped or mis-signed flux, lift or metric term leaves an O(1) error and fails both."""
    L = 20.0
    for p in (2, 3):
        for implicit in (False, True):
            errs, werrs = [], []
            for n in (20, 40, 80):
                mesh = structured_quads(uniform_nodes(n, 0, L), uniform_nodes(n, 0, L), p=p,
                                        implicit=np.full(n * n, implicit))
                d = Discretisation(mesh, NavierStokes2D(1.4, 0.0, 0.72))
                xy = d.geo.xy
                U = isentropic_vortex(xy, mach=0.5, center=(L / 2, L / 2))
                dUdx = isentropic_vortex(xy + np.array([1e-30j, 0.0]), mach=0.5, center=(L / 2, L / 2)).imag / 1e-30
                exact = -0.5 * dUdx
                R, g = d.full_residual(U, d.initial_trace(U))
                W = np.outer(d.ref.w, d.ref.w).reshape(-1)[None, :] * d.geo.J
                errs.append(math.sqrt(np.sum(W[..., None] * (R - exact) ** 2)))
                psi = np.exp(-0.5 * ((xy[..., 0] - L / 2 - 0.3) ** 2 + (xy[..., 1] - L / 2 + 0.2) ** 2))
                werrs.append(np.abs(np.sum((W * psi)[..., None] * (R - exact), axis=(0, 1))).max())
                if implicit:
                    assert np.abs(g).max() < 1e-13  # average trace: the two one-sided fluxes cancel
            rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
            wrates = np.log2(np.array(werrs[:-1]) / np.array(werrs[1:]))
            assert np.all(rates > p - 0.15), (p, implicit, errs, rates)
            assert np.all(wrates > p + 1), (p, implicit, werrs, wrates)
