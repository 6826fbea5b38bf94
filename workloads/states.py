"""Initial states sampled at the solution points of a quad mesh.

The state array layout is ``u[e, pt, v]`` with ``pt = a + (p+1) b`` where
``a`` indexes the 1D Gauss-Legendre node along xi and ``b`` along eta, and
``v`` the conserved variable.  Node placement uses numpy's Gauss-Legendre
rule and the bilinear corner interpolation of the element; this module only
places input data and does no part of the discretisation.
"""

from __future__ import annotations

import numpy as np


def sample_points(mesh, p: int) -> np.ndarray:
    """Physical coordinates (E, (p+1)^2, 2) of the Gauss-Legendre tensor nodes."""
    xg, _ = np.polynomial.legendre.leggauss(p + 1)
    n = p + 1
    xi = np.tile(xg, n)  # a fastest
    eta = np.repeat(xg, n)
    N = np.stack(
        [
            0.25 * (1 - xi) * (1 - eta),
            0.25 * (1 + xi) * (1 - eta),
            0.25 * (1 - xi) * (1 + eta),
            0.25 * (1 + xi) * (1 + eta),
        ],
        axis=1,
    )  # (Ns, 4)
    return np.einsum("sk,ekd->esd", N, mesh.verts)


def sample_points_mixed(mesh) -> list:
    """Per-element physical coordinates ((p_e+1)^2, 2) of the Gauss-Legendre tensor nodes of a mesh
    whose elements carry their own degree mesh.p[e]."""
    return [sample_points(type("M", (), {"verts": mesh.verts[e:e + 1]}), int(mesh.p[e]))[0]
            for e in range(mesh.nelem)]


def gaussian_scalar(xy: np.ndarray, center=(0.5, 0.5), alpha=50.0) -> np.ndarray:
    """u = exp(-alpha |x - c|^2), shape (..., 1)."""
    r2 = (xy[..., 0] - center[0]) ** 2 + (xy[..., 1] - center[1]) ** 2
    return np.exp(-alpha * r2)[..., None]


def isentropic_vortex(
    xy: np.ndarray,
    gamma=1.4,
    mach=0.5,
    strength=5.0,
    center=(5.0, 5.0),
    rho_inf=1.0,
) -> np.ndarray:
    """Conserved variables (rho, rho u, rho v, E) of the isentropic vortex.

    Free stream: rho = rho_inf, p = rho_inf / gamma (unit sound speed),
    velocity (mach, 0).  Tangential velocity perturbation
    (strength / 2 pi) r exp((1 - r^2)/2) about ``center``; temperature
    T = p / rho lowered by (gamma - 1) strength^2 / (8 gamma pi^2) exp(1 - r^2);
    density from isentropy.
    """
    dx = xy[..., 0] - center[0]
    dy = xy[..., 1] - center[1]
    r2 = dx * dx + dy * dy
    amp = strength / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    u = mach - amp * dy
    v = amp * dx
    T_inf = 1.0 / gamma
    T = T_inf - (gamma - 1.0) * strength**2 / (8.0 * gamma * np.pi**2) * np.exp(1.0 - r2)
    rho = rho_inf * (T / T_inf) ** (1.0 / (gamma - 1.0))
    p = rho * T
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E], axis=-1)


def freestream(shape, gamma=1.4, mach=0.5, rho_inf=1.0, angle=0.0) -> np.ndarray:
    """Uniform state of the given leading shape: (..., 4)."""
    p = rho_inf / gamma
    u = mach * np.cos(angle)
    v = mach * np.sin(angle)
    E = p / (gamma - 1.0) + 0.5 * rho_inf * (u * u + v * v)
    out = np.empty(tuple(shape) + (4,))
    out[...] = np.array([rho_inf, rho_inf * u, rho_inf * v, E])
    return out


def uniform_noise(shape, amplitude: float, seed: int) -> np.ndarray:
    """Seeded U(-amplitude, amplitude) noise (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-amplitude, amplitude, size=shape)


def edac_vortex(xy: np.ndarray, strength=1.0, speed=1.0, center=(5.0, 5.0)) -> np.ndarray:
    """(P, v_x, v_y) of an incompressible vortex carried by a uniform stream (speed, 0): the
    velocity perturbation (strength / 2 pi) r exp((1 - r^2)/2) about ``center`` and the pressure
    -strength^2 / (8 pi^2) exp(1 - r^2) that balances it.  With strength < 2 pi speed / 1.2 the
    velocity never vanishes."""
    dx = xy[..., 0] - center[0]
    dy = xy[..., 1] - center[1]
    r2 = dx * dx + dy * dy
    amp = strength / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    vx = speed - amp * dy
    vy = amp * dx
    P = -strength**2 / (8.0 * np.pi**2) * np.exp(1.0 - r2)
    return np.stack([P, vx, vy], axis=-1)


def sample_points_hex(mesh, p: int) -> np.ndarray:
    """Physical coordinates (E, (p+1)^3, 3) of the Gauss-Legendre tensor nodes of a hex mesh,
    pt = a + n b + n^2 c, by trilinear corner interpolation."""
    xg, _ = np.polynomial.legendre.leggauss(p + 1)
    n = p + 1
    xi, eta, zeta = np.tile(xg, n * n), np.tile(np.repeat(xg, n), n), np.repeat(xg, n * n)
    sa = np.array([-1.0, 1, -1, 1, -1, 1, -1, 1])
    sb = np.array([-1.0, -1, 1, 1, -1, -1, 1, 1])
    sc = np.array([-1.0, -1, -1, -1, 1, 1, 1, 1])
    N = 0.125 * (1 + sa * xi[:, None]) * (1 + sb * eta[:, None]) * (1 + sc * zeta[:, None])
    return np.einsum("sk,ekd->esd", N, mesh.verts)


def channel_state(xyz: np.ndarray, gamma=1.4, mach=0.1, rho=1.0) -> np.ndarray:
    """(rho, rho v, E) of the Taylor-Green-like channel field: v = M (sin x cos y cos z,
    -cos x sin y cos z, 0) (1 - y^2) (zero on walls at y = +-1), uniform density and pressure
    1 / gamma (sound speed 1)."""
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    damp = 1.0 - y * y
    u = mach * np.sin(x) * np.cos(y) * np.cos(z) * damp
    v = -mach * np.cos(x) * np.sin(y) * np.cos(z) * damp
    w = np.zeros_like(u)
    p = np.full_like(u, 1.0 / gamma)
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([np.full_like(u, rho), rho * u, rho * v, rho * w, E], axis=-1)
