"""Conservation laws u_t + div(F^c(u) - F^v(u, grad u)) = 0 used by the stage.

Every function accepts real or complex arrays (complex-step differentiation in
``blocks``): |x| is written as x * sign(Re x) and the branch of a maximum is
chosen on real parts, so derivatives are exact away from the kinks.

Shapes: u (..., nv); q = grad u of the conserved variables (..., d, nv) with
q[..., c, v] = du_v / dx_c; n (..., d) a unit normal.  Fluxes are (..., d, nv).

Readings (the paper gives no equations for these cases):
* advection-diffusion: F^c = beta u, F^v = nu grad u; HFR stabilisation
  s = |beta . n| + nu / lref (eq. hfrriemann says only that s follows the
  physics).
* Navier-Stokes (Sec. 5.2-5.3 use it without writing it): ideal gas with
  R = 1 (T = p / rho), constant viscosity mu, Stokes hypothesis, heat
  conductivity kappa = mu gamma / ((gamma - 1) Pr); standard-FR wave speed
  |v . n| + c (Sec. 2.1, Rusanov with the maximum local wave speed);
  HFR stabilisation s = (|v^ . n| + c^ + mu / (rho^ lref)) I evaluated at the
  trace state, the compressible counterpart of the isotropic Rusanov-type
  choice the paper prints for EDAC (Sec. 5.4).
"""

from __future__ import annotations

import numpy as np


def cabs(x):
    """|x| that stays analytic for complex-step perturbations."""
    return np.where(np.real(x) >= 0.0, x, -x)


def cmax(a, b):
    return np.where(np.real(a) >= np.real(b), a, b)


class AdvectionDiffusion:
    nv = 1

    def __init__(self, beta=(1.0, 0.5), nu=0.01, lref=1.0):
        self.beta = np.asarray(beta, dtype=np.float64)
        self.nu = float(nu)
        self.lref = float(lref)
        self.viscous = self.nu != 0.0

    def conv(self, u):
        return self.beta[:, None] * u[..., None, :]

    def visc(self, u, q):
        return self.nu * q

    def wave_speed(self, u, n):
        return cabs(np.einsum("...c,c->...", n, self.beta) + 0.0 * u[..., 0])

    def stab(self, uh, n):
        return self.wave_speed(uh, n) + self.nu / self.lref


class NavierStokes2D:
    nv = 4

    def __init__(self, gamma=1.4, mu=5e-5, Pr=0.72, lref=1.0):
        self.gamma = float(gamma)
        self.mu = float(mu)
        self.Pr = float(Pr)
        self.lref = float(lref)
        self.viscous = self.mu != 0.0

    def primitives(self, u):
        rho = u[..., 0]
        vx = u[..., 1] / rho
        vy = u[..., 2] / rho
        p = (self.gamma - 1.0) * (u[..., 3] - 0.5 * rho * (vx * vx + vy * vy))
        return rho, vx, vy, p

    def conv(self, u):
        rho, vx, vy, p = self.primitives(u)
        E = u[..., 3]
        F = np.empty(u.shape[:-1] + (2, 4), dtype=u.dtype)
        F[..., 0, 0] = rho * vx
        F[..., 0, 1] = rho * vx * vx + p
        F[..., 0, 2] = rho * vx * vy
        F[..., 0, 3] = (E + p) * vx
        F[..., 1, 0] = rho * vy
        F[..., 1, 1] = rho * vx * vy
        F[..., 1, 2] = rho * vy * vy + p
        F[..., 1, 3] = (E + p) * vy
        return F

    def visc(self, u, q):
        g = self.gamma
        rho, vx, vy, p = self.primitives(u)
        E = u[..., 3]
        # velocity and temperature gradients from conserved-variable gradients
        dvx = (q[..., :, 1] - vx[..., None] * q[..., :, 0]) / rho[..., None]
        dvy = (q[..., :, 2] - vy[..., None] * q[..., :, 0]) / rho[..., None]
        dT = (g - 1.0) * (
            (q[..., :, 3] - (E / rho)[..., None] * q[..., :, 0]) / rho[..., None]
            - vx[..., None] * dvx
            - vy[..., None] * dvy
        )
        div = dvx[..., 0] + dvy[..., 1]
        mu = self.mu
        kappa = mu * g / ((g - 1.0) * self.Pr)
        txx = mu * (2.0 * dvx[..., 0] - 2.0 / 3.0 * div)
        tyy = mu * (2.0 * dvy[..., 1] - 2.0 / 3.0 * div)
        txy = mu * (dvx[..., 1] + dvy[..., 0])
        F = np.zeros(u.shape[:-1] + (2, 4), dtype=np.result_type(u, q))
        F[..., 0, 1] = txx
        F[..., 0, 2] = txy
        F[..., 0, 3] = vx * txx + vy * txy + kappa * dT[..., 0]
        F[..., 1, 1] = txy
        F[..., 1, 2] = tyy
        F[..., 1, 3] = vx * txy + vy * tyy + kappa * dT[..., 1]
        return F

    def sound_speed(self, u):
        rho, _, _, p = self.primitives(u)
        return np.sqrt(self.gamma * p / rho)

    def wave_speed(self, u, n):
        _, vx, vy, _ = self.primitives(u)
        return cabs(vx * n[..., 0] + vy * n[..., 1]) + self.sound_speed(u)

    def stab(self, uh, n):
        return self.wave_speed(uh, n) + self.mu / (uh[..., 0] * self.lref)


class NavierStokes3D:
    """The Navier-Stokes readings above in three dimensions: u = (rho, rho v_x, rho v_y, rho v_z, E),
    p = (gamma - 1)(E - rho |v|^2 / 2), tau = mu (grad v + grad v^T - 2/3 div v I), heat flux
    kappa grad T with T = p / rho."""

    nv = 5

    def __init__(self, gamma=1.4, mu=5e-5, Pr=0.72, lref=1.0):
        self.gamma = float(gamma)
        self.mu = float(mu)
        self.Pr = float(Pr)
        self.lref = float(lref)
        self.viscous = self.mu != 0.0

    def primitives(self, u):
        rho = u[..., 0]
        v = u[..., 1:4] / rho[..., None]
        p = (self.gamma - 1.0) * (u[..., 4] - 0.5 * rho * np.sum(v * v, axis=-1))
        return rho, v, p

    def conv(self, u):
        rho, v, p = self.primitives(u)
        E = u[..., 4]
        F = np.empty(u.shape[:-1] + (3, 5), dtype=u.dtype)
        for d in range(3):
            F[..., d, 0] = rho * v[..., d]
            for k in range(3):
                F[..., d, 1 + k] = rho * v[..., d] * v[..., k] + (p if k == d else 0.0)
            F[..., d, 4] = (E + p) * v[..., d]
        return F

    def visc(self, u, q):
        g = self.gamma
        rho, v, p = self.primitives(u)
        E = u[..., 4]
        # dv[..., c, k] = d v_k / d x_c, dT[..., c] from the conserved-variable gradients
        dv = (q[..., :, 1:4] - v[..., None, :] * q[..., :, :1]) / rho[..., None, None]
        dT = (g - 1.0) * ((q[..., :, 4] - (E / rho)[..., None] * q[..., :, 0]) / rho[..., None]
                          - np.einsum("...k,...ck->...c", v, dv))
        div = dv[..., 0, 0] + dv[..., 1, 1] + dv[..., 2, 2]
        mu = self.mu
        kappa = mu * g / ((g - 1.0) * self.Pr)
        F = np.zeros(u.shape[:-1] + (3, 5), dtype=np.result_type(u, q))
        for c in range(3):
            for k in range(3):
                F[..., c, 1 + k] = mu * (dv[..., c, k] + dv[..., k, c] - (2.0 / 3.0 * div if c == k else 0.0))
            F[..., c, 4] = np.einsum("...k,...k->...", v, F[..., c, 1:4]) + kappa * dT[..., c]
        return F

    def sound_speed(self, u):
        rho, _, p = self.primitives(u)
        return np.sqrt(self.gamma * p / rho)

    def wave_speed(self, u, n):
        _, v, _ = self.primitives(u)
        return cabs(np.einsum("...c,...c->...", v, n)) + self.sound_speed(u)

    def stab(self, uh, n):
        return self.wave_speed(uh, n) + self.mu / (uh[..., 0] * self.lref)


class EDAC2D:
    """Entropically damped artificial compressibility (Appendix A): u = (P, v_x, v_y),
    F^c_i = (v_i (P + Theta), v_i v_x + P delta_ix, v_i v_y + P delta_iy), F^v_i = nu du/dx_i,
    Theta = 1 / M^2 (artificial Mach number), nu = 1 / Re.

    * Standard-FR Rusanov speed: the largest eigenvalue magnitude of the normal flux Jacobian,
      3/2 |v.n| + sqrt((v.n)^2 / 4 + P + Theta) (the eigenvalues are v.n and
      3/2 v.n +- sqrt((v.n)^2/4 + P + Theta)).
    * HFR stabilisation (Sec. 5.4): s = 3/2 |v^| + d^, d^2 = |v^|^2 / 4 + P^ + Theta, isotropic, at
      the trace state; plus nu / lref for the viscous terms (as for the other two laws).
      |v^| has no derivative at v^ = 0: states with a nonzero velocity everywhere are assumed.
    """

    nv = 3

    def __init__(self, theta=100.0, nu=1e-3, lref=1.0):
        self.theta = float(theta)
        self.nu = float(nu)
        self.lref = float(lref)
        self.viscous = self.nu != 0.0

    def conv(self, u):
        P, vx, vy = u[..., 0], u[..., 1], u[..., 2]
        Pt = P + self.theta
        Fx = np.stack([vx * Pt, vx * vx + P, vx * vy], axis=-1)
        Fy = np.stack([vy * Pt, vy * vx, vy * vy + P], axis=-1)
        return np.stack([Fx, Fy], axis=-2)

    def visc(self, u, q):
        return self.nu * q

    def wave_speed(self, u, n):
        P, vx, vy = u[..., 0], u[..., 1], u[..., 2]
        vn = vx * n[..., 0] + vy * n[..., 1]
        return 1.5 * cabs(vn) + np.sqrt(0.25 * vn * vn + P + self.theta)

    def stab(self, uh, n):
        P, vx, vy = uh[..., 0], uh[..., 1], uh[..., 2]
        v2 = vx * vx + vy * vy
        return 1.5 * np.sqrt(v2) + np.sqrt(0.25 * v2 + P + self.theta) + self.nu / self.lref


def make_physics(spec: dict):
    kind = spec["kind"]
    if kind == "advdiff":
        return AdvectionDiffusion(spec["beta"], spec["nu"], spec.get("lref", 1.0))
    if kind == "ns":
        return NavierStokes2D(spec["gamma"], spec["mu"], spec["Pr"], spec.get("lref", 1.0))
    if kind == "ns3d":
        return NavierStokes3D(spec["gamma"], spec["mu"], spec["Pr"], spec.get("lref", 1.0))
    if kind == "edac":
        return EDAC2D(spec["theta"], spec["nu"], spec.get("lref", 1.0))
    raise KeyError(kind)
