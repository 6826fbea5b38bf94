"""Modal filter of Appendix B (test infrastructure: the FP64 oracle; only tests, the smoke check
and the benchmark's CPU baseline use this package).

F = V Lambda* V^{-1} on the (p+1)^2 solution points of an element, with V_ij = Psi_j(x_i) the
tensor-product orthonormal Legendre basis Psi_(a,b)(xi, eta) = psi_a(xi) psi_b(eta),
psi_k = sqrt((2k+1)/2) P_k, and Lambda = diag(sigma(eta)) where eta = a + b is the sum of the
exponents of the mode's leading term and

    sigma(eta) = 1                                              0 <= eta < eta_c
               = exp(-alpha ((eta - eta_c) / (eta_max - eta_c))^s)  eta_c <= eta <= eta_max
               = 0                                              eta > eta_max,

eta_max = 2p.  Reading of the time-step normalisation (the paper defers it to its reference):
Lambda* = Lambda^(dt / dt_ref), so that filtering every step of size dt damps a mode over a
time interval as a step of dt_ref does; dt_ref = dt gives Lambda* = Lambda.
"""

from __future__ import annotations

import numpy as np

from .basis import gauss_legendre, legendre


def sigma(eta, alpha: float, s: float, eta_c: int, eta_max: int):
    eta = np.asarray(eta, dtype=np.float64)
    out = np.ones_like(eta)
    mid = (eta >= eta_c) & (eta <= eta_max)
    if eta_max > eta_c:
        out[mid] = np.exp(-alpha * ((eta[mid] - eta_c) / (eta_max - eta_c)) ** s)
    else:
        out[mid] = np.exp(-alpha * (eta[mid] >= eta_c))
    out[eta > eta_max] = 0.0
    return out


def vandermonde_2d(p: int) -> tuple[np.ndarray, np.ndarray]:
    """V (n^2 x n^2) at the Gauss points, point index a + n b, mode index i + n j (degrees i in
    xi, j in eta), and the exponent sums eta = i + j of the modes."""
    n = p + 1
    x, _ = gauss_legendre(n)
    V1 = np.stack([np.sqrt((2 * k + 1) / 2.0) * legendre(k, x)[0] for k in range(n)], axis=1)  # (pt, k)
    V = np.einsum("ai,bj->abij", V1, V1).reshape(n, n, n, n)
    # rows: point (a, b) -> a + n b; columns: mode (i, j) -> i + n j
    V = V.transpose(1, 0, 3, 2).reshape(n * n, n * n)
    i = np.arange(n)
    eta = (i[None, :] + i[:, None]).reshape(-1)  # mode i + n j -> i + j (symmetric)
    return V, eta


def filter_matrix(p: int, alpha: float, s: float, eta_c: int, dt_ratio: float = 1.0) -> np.ndarray:
    """F = V Lambda* V^{-1} with Lambda* = Lambda^dt_ratio (dt_ratio = dt / dt_ref)."""
    V, eta = vandermonde_2d(p)
    lam = sigma(eta, alpha, s, eta_c, 2 * p) ** dt_ratio
    return V @ np.diag(lam) @ np.linalg.inv(V)


def apply_filter(U: np.ndarray, p: int, alpha: float, s: float, eta_c: int, dt_ratio: float = 1.0,
                 elements=None) -> np.ndarray:
    """Filtered copy of U (E, n^2, nv); elements (optional): indices of the elements to filter."""
    F = filter_matrix(p, alpha, s, eta_c, dt_ratio)
    out = U.copy()
    idx = np.arange(U.shape[0]) if elements is None else np.asarray(elements)
    out[idx] = np.einsum("ik,ekv->eiv", F, U[idx])
    return out
