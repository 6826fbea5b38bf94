"""Pins of the oracle's modal filter (Appendix B) against facts fixed by its definition: identity
at zero damping, exact preservation of polynomials up to the cut-off degree, each orthonormal
mode scaled by sigma(exponent sum), the element mean kept, the top mode damped by exp(-alpha),
and the time-step normalisation composing (two half-ratio filters = one full-ratio filter)."""

import numpy as np

from oracle.basis import gauss_legendre
from oracle.filter import apply_filter, filter_matrix, sigma, vandermonde_2d


def _points(p):
    x, w = gauss_legendre(p + 1)
    n = p + 1
    xi = np.tile(x, n)       # point a + n b -> x_a
    et = np.repeat(x, n)     # -> x_b
    W = np.outer(w, w).reshape(-1)  # weight of point a + n b: w_b w_a (symmetric product)
    return xi, et, W


def test_zero_damping_is_the_identity():
    for p in (2, 3, 4):
        assert np.abs(filter_matrix(p, 0.0, 1.0, 1) - np.eye((p + 1) ** 2)).max() < 1e-12


def test_polynomials_below_the_cutoff_are_kept():
    for p in (3, 4):
        xi, et, _ = _points(p)
        F = filter_matrix(p, 100.0, 1.0, 3)
        # sigma(eta_c) = exp(0) = 1: total degree up to eta_c is kept
        for a in range(4):
            for b in range(4 - a):
                u = xi**a * et**b
                assert np.abs(F @ u - u).max() < 1e-12, (a, b)
        # a term of total degree 4 (mode (2, 2)) is damped
        u = xi**2 * et**2
        assert np.abs(F @ u - u).max() > 1e-3


def test_each_mode_is_scaled_by_sigma_of_its_exponent_sum():
    p, alpha, s, ec = 4, 7.0, 2.0, 2
    V, eta = vandermonde_2d(p)
    F = filter_matrix(p, alpha, s, ec)
    lam = sigma(eta, alpha, s, ec, 2 * p)
    n = p + 1
    for j in range(n):
        for i in range(n):
            m = i + n * j
            assert eta[m] == i + j
            assert np.abs(F @ V[:, m] - lam[m] * V[:, m]).max() < 1e-12
    # orthonormality of the basis under the tensor Gauss rule
    _, _, W = _points(p)
    assert np.abs(V.T @ (W[:, None] * V) - np.eye(n * n)).max() < 1e-12
    # the top mode (exponent sum 2p) is damped by exp(-alpha)
    assert abs(lam[n * n - 1] - np.exp(-alpha)) < 1e-14


def test_filter_keeps_the_element_mean_and_composes_in_time():
    rng = np.random.default_rng(2)
    p = 3
    _, _, W = _points(p)
    U = rng.standard_normal((5, (p + 1) ** 2, 4))
    Uf = apply_filter(U, p, 100.0, 1.0, 3)
    assert np.abs(np.einsum("q,eqv->ev", W, Uf - U)).max() < 1e-12
    F1 = filter_matrix(p, 10.0, 1.0, 2, 1.0)
    Fh = filter_matrix(p, 10.0, 1.0, 2, 0.5)
    assert np.abs(Fh @ Fh - F1).max() < 1e-12
