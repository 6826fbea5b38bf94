"""Named synthetic workloads (mesh + physics parameters + initial state + step).

Every workload is fully deterministic given its name and overrides.  The
physics parameters are plain numbers handed to both the oracle and the GPU
library; nothing here evaluates the discretisation.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .mesh import structured_quads, uniform_nodes
from .states import edac_vortex, sample_points, gaussian_scalar, isentropic_vortex, uniform_noise


@dataclass
class Workload:
    name: str
    mesh: object
    p: int
    physics: dict
    u0: np.ndarray  # (E, Ns, nv)
    dt: float
    tableau: str
    newton_tol: float = 1e-8
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.u0.shape[-1])

    @property
    def dofs_implicit(self) -> int:
        return int(self.mesh.implicit.sum()) * self.u0.shape[1] * self.u0.shape[2]


def _advdiff(n=8, p=2, dt=0.05, jitter=0.0, seed=0, implicit=None):
    mesh = structured_quads(uniform_nodes(n, 0.0, 1.0), uniform_nodes(n, 0.0, 1.0),
                            periodic=(True, True), jitter=jitter, seed=seed, p=p,
                            implicit=implicit)
    xy = sample_points(mesh, p)
    u0 = gaussian_scalar(xy, (0.5, 0.5), 50.0)
    phys = {"kind": "advdiff", "beta": (1.0, 0.5), "nu": 0.01, "lref": 1.0}
    return mesh, u0, phys, dt


def _vortex(n=64, p=3, noise=0.0, seed=1234, cfl_mult=10.0, jitter=0.0, implicit=None,
            re=1.0e4, mach=0.5, gamma=1.4):
    L = 10.0
    mesh = structured_quads(uniform_nodes(n, 0.0, L), uniform_nodes(n, 0.0, L),
                            periodic=(True, True), jitter=jitter, seed=seed, p=p,
                            implicit=implicit)
    xy = sample_points(mesh, p)
    u0 = isentropic_vortex(xy, gamma=gamma, mach=mach, strength=5.0, center=(5.0, 5.0))
    if noise > 0.0:
        u0 = u0 + uniform_noise(u0.shape, noise, seed)
    mu = 1.0 * mach * 1.0 / re  # rho_inf |v_inf| L_ref / Re with L_ref = 1
    phys = {"kind": "ns", "gamma": gamma, "mu": mu, "Pr": 0.72, "lref": 1.0}
    h = L / n
    c_inf = 1.0
    dt_ex = h / ((mach + c_inf) * (2 * p + 1))
    return mesh, u0, phys, cfl_mult * dt_ex


def _edac(n=16, p=3, theta=100.0, re=1.0e3, cfl_mult=10.0, jitter=0.0, seed=0, implicit=None, noise=0.0):
    L = 10.0
    mesh = structured_quads(uniform_nodes(n, 0.0, L), uniform_nodes(n, 0.0, L),
                            periodic=(True, True), jitter=jitter, seed=seed, p=p, implicit=implicit)
    u0 = edac_vortex(sample_points(mesh, p), strength=1.0, speed=1.0, center=(5.0, 5.0))
    if noise > 0.0:
        u0 = u0 + uniform_noise(u0.shape, noise, seed)
    phys = {"kind": "edac", "theta": theta, "nu": 1.0 / re, "lref": 1.0}
    lam = 1.5 + np.sqrt(0.25 + theta)  # largest wave speed of the uniform stream
    dt_ex = (L / n) / (lam * (2 * p + 1))
    return mesh, u0, phys, cfl_mult * dt_ex


def make_config(name: str, **kw) -> Workload:
    if name == "advdiff8":  # 8x8 p=2 advection-diffusion, one backward-Euler step
        mesh, u0, phys, dt = _advdiff(**kw)
        return Workload(name, mesh, int(mesh.p[0]), phys, u0, dt, "be")
    if name == "vortex64":  # 64x64 p=3 Navier-Stokes vortex, one SDIRK2 step at 10x CFL
        args = dict(n=64, p=3)
        args.update(kw)
        mesh, u0, phys, dt = _vortex(**args)
        return Workload(name, mesh, int(mesh.p[0]), phys, u0, dt, "sdirk2")
    if name == "vortex256":  # 256x256 p=4 vortex + 1e-3 seeded noise
        args = dict(n=256, p=4, noise=1.0e-3, seed=1234)
        args.update(kw)
        mesh, u0, phys, dt = _vortex(**args)
        return Workload(name, mesh, int(mesh.p[0]), phys, u0, dt, "sdirk2")
    if name == "vortex":  # generic vortex of any size for tests
        mesh, u0, phys, dt = _vortex(**kw)
        return Workload(name, mesh, int(mesh.p[0]), phys, u0, dt, "sdirk2")
    if name == "edac":  # EDAC vortex in a uniform stream (Theta = 100), one SDIRK2 step at 10x CFL
        mesh, u0, phys, dt = _edac(**kw)
        return Workload(name, mesh, int(mesh.p[0]), phys, u0, dt, "sdirk2")
    if name == "advdiff":
        mesh, u0, phys, dt = _advdiff(**kw)
        return Workload(name, mesh, int(mesh.p[0]), phys, u0, dt, "be")
    raise KeyError(name)


CONFIGS = {
    "advdiff8": "2D advection-diffusion, beta=(1,0.5), nu=0.01, periodic unit square, 8x8 quads, p=2, one backward-Euler step dt=0.05",
    "vortex64": "2D Navier-Stokes isentropic vortex, M=0.5, gamma=1.4, Re=1e4, periodic [0,10]^2, 64x64 quads, p=3, one SDIRK2 step at 10x the explicit CFL",
    "vortex256": "as vortex64 on 256x256 quads, p=4, plus U(-1e-3,1e-3) noise (seed 1234)",
}
