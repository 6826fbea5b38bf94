"""Reference-element operators (Sec. 2, eqs. frsolution, frfluxd, fluxcorrection).

* Solution points: Gauss-Legendre nodes (Sec. 2.2, last paragraph), found
  here by Newton's method on the Legendre polynomial P_{p+1}.
* Nodal basis: Lagrange polynomials on those nodes.
* Correction functions: the paper does not name its family; the reading used
  is the DG-recovering (right/left Radau) pair
      g_L(x) = (-1)^p / 2 (P_p(x) - P_{p+1}(x)),   g_R(x) = (P_p(x) + P_{p+1}(x)) / 2,
  with g_L(-1) = 1, g_L(1) = 0, g_R mirrored, so that n . g = 1 at its own
  flux point and 0 at the others (eq. dsklnf), in tensor-product form.
"""

from __future__ import annotations

import numpy as np


def legendre(n: int, x):
    """P_n(x) and P_n'(x) by the three-term recurrence
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and P'_{k+1} = P'_{k-1} + (2k+1) P_k."""
    x = np.asarray(x, dtype=np.float64)
    P = [np.ones_like(x), x.copy()]
    dP = [np.zeros_like(x), np.ones_like(x)]
    for k in range(1, n):
        P.append(((2 * k + 1) * x * P[k] - k * P[k - 1]) / (k + 1))
        dP.append(dP[k - 1] + (2 * k + 1) * P[k])
    return P[n], dP[n]


def gauss_legendre(n: int):
    """n-point Gauss-Legendre nodes (ascending) and weights.

    Newton's method on P_n from the Chebyshev-like initial guesses
    cos(pi (i + 3/4) / (n + 1/2)); weights w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2).
    """
    i = np.arange(n)
    x = np.cos(np.pi * (i + 0.75) / (n + 0.5))
    for _ in range(100):
        Pn, dPn = legendre(n, x)
        dx = Pn / dPn
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    _, dPn = legendre(n, x)
    w = 2.0 / ((1.0 - x * x) * dPn * dPn)
    order = np.argsort(x)
    return x[order], w[order]


def gauss_lobatto(n: int):
    """n-point Gauss-Lobatto-Legendre nodes (ascending, n >= 2) and weights: x = -1, +1 and the
    roots of P'_{n-1}, found by Newton's method with P''_m from Legendre's equation
    (1 - x^2) P''_m = 2 x P'_m - m (m + 1) P_m, started at cos(pi i / (n - 1));
    weights w_i = 2 / (n (n - 1) P_{n-1}(x_i)^2)."""
    m = n - 1
    x = -np.cos(np.pi * np.arange(1, m) / m)
    for _ in range(100):
        if x.size == 0:
            break
        P, dP = legendre(m, x)
        dx = (1.0 - x * x) * dP / (2.0 * x * dP - m * (m + 1) * P)
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    x = np.concatenate([[-1.0], np.sort(x), [1.0]])
    P, _ = legendre(m, x)
    return x, 2.0 / (n * m * P * P)


def lagrange(nodes: np.ndarray, x) -> np.ndarray:
    """Matrix L[k, j] = l_j(x_k) of the Lagrange basis on ``nodes``."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return L


def lagrange_derivative(nodes: np.ndarray, x) -> np.ndarray:
    """Matrix D[k, j] = l_j'(x_k), from the product rule on the Lagrange product."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((len(x), n))
    for j in range(n):
        for k in range(n):
            if k == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[k]))
            for m in range(n):
                if m != j and m != k:
                    term *= (x - nodes[m]) / (nodes[j] - nodes[m])
            D[:, j] += term
    return D


def radau_corrections(p: int, x):
    """Values and derivatives of the left/right DG-recovering correction
    functions g_L, g_R of degree p+1 at ``x``."""
    Pp, dPp = legendre(p, x)
    Pq, dPq = legendre(p + 1, x)
    s = (-1.0) ** p
    gL = 0.5 * s * (Pp - Pq)
    dgL = 0.5 * s * (dPp - dPq)
    gR = 0.5 * (Pp + Pq)
    dgR = 0.5 * (dPp + dPq)
    return gL, dgL, gR, dgR


class RefElement1D:
    """1D operators on p+1 Gauss-Legendre solution points."""

    def __init__(self, p: int):
        self.p = p
        self.n = p + 1
        self.x, self.w = gauss_legendre(self.n)
        # derivative matrix D[i, j] = l_j'(x_i)
        self.D = lagrange_derivative(self.x, self.x)
        # interpolation to the ends: l_j(-1), l_j(+1)
        self.lm = lagrange(self.x, -1.0)[0]
        self.lp = lagrange(self.x, +1.0)[0]
        # correction-function derivatives at the solution points
        _, dgL, _, dgR = radau_corrections(p, self.x)
        self.dgL = dgL
        self.dgR = dgR
