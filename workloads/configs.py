"""Named synthetic workloads (mesh + physics parameters + initial state + step).

Every workload is fully deterministic given its name and overrides.  The
physics parameters are plain numbers handed to both the oracle and the GPU
library; nothing here evaluates the discretisation.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .mesh import BC_FARFIELD, BC_WALL, structured_hexes, structured_quads, tanh_nodes, uniform_nodes
from .states import (channel_state, edac_vortex, freestream, gaussian_scalar, isentropic_vortex,
                     sample_points, sample_points_hex, uniform_noise)


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
        return int(self.u0[0].shape[-1])

    @property
    def dofs_implicit(self) -> int:
        """Implicit solution unknowns (u0 is an (E, Ns, nv) array, or a list of (Ns_e, nv) arrays
        when the degree varies per element)."""
        return int(sum(self.u0[e].size for e in np.nonzero(self.mesh.implicit)[0]))


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


def stiffness_indicator(verts: np.ndarray) -> np.ndarray:
    """E_s = |Omega_k| / |dOmega_k| of each quad (area over perimeter; Sec. 5)."""
    a, b, c, d = verts[:, 0], verts[:, 1], verts[:, 2], verts[:, 3]
    area = 0.5 * np.abs((d[:, 0] - a[:, 0]) * (c[:, 1] - b[:, 1]) - (d[:, 1] - a[:, 1]) * (c[:, 0] - b[:, 0]))
    perim = sum(np.linalg.norm(q - r, axis=1) for q, r in ((b, a), (d, b), (c, d), (a, c)))
    return area / perim


def _boundary_layer(nx=400, ny=500, h0=1.0e-5, ratio=1.15, dx=1.0e-2, degrees=(2, 3, 4, 5), if_target=0.2,
                    re=1.7e6, mach=0.2, gamma=1.4, noise=1.0e-3, seed=2024):
    """Stretched wall band: first cell h0 growing by ``ratio`` until the isotropic spacing dx, then
    isotropic cells; wall below, far field above, periodic streamwise.  Implicit elements: the
    if_target fraction with the smallest E_s, ties (equal cells) broken towards the wall."""
    yn = [0.0]
    h = h0
    for _ in range(ny):
        yn.append(yn[-1] + min(h, dx))
        h *= ratio
    mesh = structured_quads(uniform_nodes(nx, 0.0, nx * dx), np.asarray(yn), periodic=(True, False), p=2,
                            bc_y=(BC_WALL, BC_FARFIELD))
    es = stiffness_indicator(mesh.verts)
    es = np.round(es / es.max(), 10)  # equal cells compare equal despite coordinate rounding
    row = np.arange(mesh.nelem) // nx
    order = np.lexsort((row, es))
    imp = np.zeros(mesh.nelem, bool)
    imp[order[:int(round(if_target * mesh.nelem))]] = True
    mesh.implicit = imp
    rng = np.random.default_rng(seed)
    mesh.p = rng.choice(np.asarray(degrees), size=mesh.nelem).astype(np.int32)
    u_inf = freestream((), gamma=gamma, mach=mach)
    u0 = []
    for e in range(mesh.nelem):
        ns = (int(mesh.p[e]) + 1) ** 2
        u0.append(u_inf + rng.uniform(-noise, noise, size=(ns, 4)))
    phys = {"kind": "ns", "gamma": gamma, "mu": mach / re, "Pr": 0.72, "lref": 1.0, "u_inf": u_inf}
    dt = dx / ((mach + 1.0) * (2 * max(degrees) + 1))  # explicit limit of the isotropic region
    return mesh, u0, phys, dt


def _channel3d(n=(64, 32, 48), p=3, beta=2.5, layers=3, re=1.6e3, mach=0.1, gamma=1.4):
    """Box [0, 2 pi] x [-1, 1] x [0, pi], tanh-clustered in y, walls at y = +-1, periodic in x and z;
    implicit: ``layers`` cell layers on each wall."""
    nx, ny, nz = n
    j = np.arange(nx * ny * nz) // nx % ny
    imp = (j < layers) | (j >= ny - layers)
    mesh = structured_hexes(uniform_nodes(nx, 0.0, 2 * np.pi), tanh_nodes(ny, beta),
                            uniform_nodes(nz, 0.0, np.pi), periodic=(True, False, True), p=p,
                            implicit=imp, bc_y=(BC_WALL, BC_WALL))
    u0 = channel_state(sample_points_hex(mesh, p), gamma=gamma, mach=mach)
    phys = {"kind": "ns3d", "gamma": gamma, "mu": mach / re, "Pr": 0.72, "lref": 1.0}
    hx = min(2 * np.pi / nx, np.pi / nz)
    dt = hx / ((mach + 1.0) * (2 * p + 1))
    return mesh, u0, phys, dt


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
    if name == "boundary_layer":  # 400x500 stretched wall band, p in 2..5, IF = 0.2, IMEX stage
        mesh, u0, phys, dt = _boundary_layer(**kw)
        return Workload(name, mesh, -1, phys, u0, dt, "sdirk2")
    if name == "channel3d":  # 64x32x48 hexes, p = 3, three implicit wall layers per wall
        mesh, u0, phys, dt = _channel3d(**kw)
        return Workload(name, mesh, int(mesh.p[0]), phys, u0, dt, "sdirk2")
    raise KeyError(name)


CONFIGS = {
    "advdiff8": "2D advection-diffusion, beta=(1,0.5), nu=0.01, periodic unit square, 8x8 quads, p=2, one backward-Euler step dt=0.05",
    "vortex64": "2D Navier-Stokes isentropic vortex, M=0.5, gamma=1.4, Re=1e4, periodic [0,10]^2, 64x64 quads, p=3, one SDIRK2 step at 10x the explicit CFL",
    "vortex256": "as vortex64 on 256x256 quads, p=4, plus U(-1e-3,1e-3) noise (seed 1234)",
    "boundary_layer": "2D Navier-Stokes, Re=1.7e6, M=0.2: 400x500 quads, wall-normal growth 1.15 from 1e-5 to isotropic 1e-2 cells, wall below, far field above, p in {2,3,4,5} per element (seed 2024), the 20% stiffest elements by E_s implicit",
    "channel3d": "3D Navier-Stokes, Re=1.6e3, M=0.1 Taylor-Green-like field: 64x32x48 hexes, tanh clustering beta=2.5, walls at y=+-1, p=3, three implicit wall layers per wall",
}
