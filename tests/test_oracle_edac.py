"""Pins of the oracle's EDAC physics (Appendix A; stabilisation of Sec. 5.4) against facts fixed
by the equations: the eigenvalues of the normal flux Jacobian (which fix the Rusanov speed and
bound the hybridized stabilisation), rotation invariance of the flux, free-stream preservation,
the hybridized solve equal to the monolithic one, and conservation across an IMEX interface."""

import numpy as np

from oracle.blocks import EPS
from oracle.fr import Discretisation
from oracle.physics import EDAC2D
from oracle.stepping import imex_step
from test_oracle_pins import _hybrid_vs_monolithic
from workloads.mesh import structured_quads, uniform_nodes
from workloads.states import edac_vortex


def _normal_flux(ph, u, n):
    F = ph.conv(u)
    return F[..., 0, :] * n[0] + F[..., 1, :] * n[1]


def _flux_jacobian(ph, u, n):
    """d(F.n)/du by complex-step differentiation of the oracle's flux."""
    J = np.zeros((3, 3))
    for k in range(3):
        up = u.astype(np.complex128)
        up[k] += 1j * EPS
        J[:, k] = _normal_flux(ph, up, n).imag / EPS
    return J


def test_edac_flux_jacobian_eigenvalues_fix_the_wave_speed():
    rng = np.random.default_rng(3)
    ph = EDAC2D(theta=100.0, nu=0.0)
    for _ in range(20):
        u = np.array([rng.uniform(-5, 5), rng.uniform(-3, 3), rng.uniform(-3, 3)])
        a = rng.uniform(0, 2 * np.pi)
        n = np.array([np.cos(a), np.sin(a)])
        lam = np.linalg.eigvals(_flux_jacobian(ph, u, n))
        vn = u[1] * n[0] + u[2] * n[1]
        d = np.sqrt(0.25 * vn * vn + u[0] + 100.0)
        # eigenvalues v.n and 3/2 v.n +- sqrt((v.n)^2/4 + P + Theta)
        assert np.allclose(np.sort(lam.real), np.sort([vn, 1.5 * vn - d, 1.5 * vn + d]), atol=1e-10)
        assert np.abs(lam.imag).max() < 1e-10
        assert abs(ph.wave_speed(u, n) - np.abs(lam).max()) < 1e-10
        # the isotropic hybridized stabilisation bounds every normal speed, with equality along v
        assert ph.stab(u, n) >= np.abs(lam).max() - 1e-12
        nv = u[1:] / np.linalg.norm(u[1:])
        assert abs(ph.stab(u, nv) - np.abs(np.linalg.eigvals(_flux_jacobian(ph, u, nv))).max()) < 1e-10


def test_edac_flux_is_rotation_invariant():
    rng = np.random.default_rng(4)
    ph = EDAC2D(theta=50.0, nu=0.0)
    for _ in range(10):
        u = rng.standard_normal(3)
        a, b = rng.uniform(0, 2 * np.pi, 2)
        n = np.array([np.cos(a), np.sin(a)])
        R = np.array([[np.cos(b), -np.sin(b)], [np.sin(b), np.cos(b)]])
        ur = np.concatenate([[u[0]], R @ u[1:]])
        f, fr = _normal_flux(ph, u, n), _normal_flux(ph, ur, R @ n)
        assert abs(fr[0] - f[0]) < 1e-12
        assert np.abs(fr[1:] - R @ f[1:]).max() < 1e-12


def _edac_disc(n=4, p=3, jitter=0.0, seed=0, nu=1e-2, implicit=None, theta=100.0):
    mesh = structured_quads(uniform_nodes(n, 0, 10), uniform_nodes(n, 0, 10), jitter=jitter, seed=seed, p=p,
                            implicit=implicit)
    return Discretisation(mesh, EDAC2D(theta, nu)), mesh


def test_edac_free_stream_preservation_on_skewed_quads():
    for implicit in (None, np.arange(16) % 3 == 0):
        d, mesh = _edac_disc(jitter=0.2, seed=5, implicit=implicit)
        U = np.broadcast_to(np.array([0.3, 0.8, -0.4]), (mesh.nelem, d.ns, 3)).copy()
        R, g = d.full_residual(U, d.initial_trace(U))
        assert np.abs(R).max() < 1e-11 and np.abs(g).max() < 1e-11


def test_edac_hybridized_solve_equals_monolithic():
    d, mesh = _edac_disc(n=3, p=2)
    U = edac_vortex(d.geo.xy, center=(5.0, 5.0))
    assert _hybrid_vs_monolithic(d, U, d.initial_trace(U), 0.01) < 1e-12


def test_edac_imex_step_conserves_across_interface():
    imp = np.zeros((6, 6), bool)
    imp[2:4, :] = True
    d, mesh = _edac_disc(n=6, p=2, implicit=imp.reshape(-1))
    U = edac_vortex(d.geo.xy)
    W = np.outer(d.ref.w, d.ref.w).reshape(-1)
    U1, _, _ = imex_step(d, U, d.initial_trace(U), 0.01, "sdirk2", tol=1e-12)
    dm = np.einsum("s,es,esv->v", W, d.geo.J, U1 - U)
    assert np.abs(dm).max() < 1e-10
