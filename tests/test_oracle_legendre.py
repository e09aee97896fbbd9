"""Pins of the oracle's Legendre functions (Sec. 2.3) against closed forms,
library routines, the Casoratian / Wronskian and asymptotics."""
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import legendre as L

XS = np.array([1.0005, 1.02, 1.1, 1.5, 2.0, 5.0, 30.0])
US = np.array([0.05, 0.2, 0.7, 1.5, 4.0, 25.0])


def test_P_matches_scipy_type3():
    N = 20
    P = L.legendre_P(XS, N)
    for i, x in enumerate(XS):
        for n in range(N + 1):
            for m in range(n + 1):
                ref = float(np.asarray(sp.assoc_legendre_p(n, m, x, branch_cut=3)).ravel()[0])
                assert abs(P[i, n, m] - ref) <= 2e-11 * abs(ref), (x, n, m)


def test_Q_matches_scipy_lqmn():
    N = 20
    Q = L.legendre_Q(XS, N)
    for i, x in enumerate(XS):
        q, _ = sp.lqmn(N, N, x)
        for n in range(N + 1):
            for m in range(n + 1):
                ref = q[m, n]
                assert abs(Q[i, n, m] - ref) <= 5e-13 * abs(ref), (x, n, m)


def test_Q_closed_forms_real():
    x = XS
    Q = L.legendre_Q(x, 4)
    Q0 = 0.5 * np.log((x + 1) / (x - 1))
    s = np.sqrt(x * x - 1)
    np.testing.assert_allclose(Q[:, 0, 0], Q0, rtol=1e-12)
    # the closed forms cancel at large x: absolute slack scaled by the cancelling term
    for got, ref, big in ((Q[:, 1, 0], x * Q0 - 1.0, x * Q0),
                          (Q[:, 2, 0], 0.5 * (3 * x * x - 1) * Q0 - 1.5 * x, 1.5 * x),
                          # Q_1^1 = sqrt(x^2-1) d/dx(x Q0 - 1) = s (Q0 - x/(x^2-1))
                          (Q[:, 1, 1], s * (Q0 - x / (x * x - 1)), s * x / (x * x - 1))):
        assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref) + 4e-15 * np.abs(big))


def test_oblate_closed_forms():
    z = 1j * US
    P = L.legendre_P(z, 3)
    Q = L.legendre_Q(z, 3, P)
    # Q_0(iu) = 1/2 log((iu+1)/(iu-1)) = -i arccot(u)
    np.testing.assert_allclose(Q[:, 0, 0], -1j * np.arctan(1.0 / US), rtol=1e-14, atol=1e-300)
    # (x^2-1)^{1/2} at x = iu is i sqrt(u^2+1)
    np.testing.assert_allclose(P[:, 1, 1], 1j * np.sqrt(US ** 2 + 1), rtol=1e-15)
    np.testing.assert_allclose(P[:, 2, 0], 0.5 * (3 * z * z - 1), rtol=1e-15)
    # i^-n P_n^m(iu) and i^{n+1} Q_n^m(iu) are real
    for n in range(4):
        for m in range(n + 1):
            assert np.all(np.abs((1j ** -n * P[:, n, m]).imag) <= 1e-14 * np.abs(P[:, n, m]) + 1e-300)
            assert np.all(np.abs((1j ** (n + 1) * Q[:, n, m]).imag) <= 1e-13 * np.abs(Q[:, n, m]) + 1e-290)


@pytest.mark.parametrize("arg", ["real", "imag"])
def test_casoratian(arg):
    """eq. (PQ): P_n Q_{n-1} - P_{n-1} Q_n = (n+m-1)!/(n-m)! (-1)^m."""
    x = XS if arg == "real" else 1j * US
    N = 18
    P = L.legendre_P(x, N)
    Q = L.legendre_Q(x, N, P)
    for n in range(1, N + 1):
        for m in range(0, n):
            lhs = P[:, n, m] * Q[:, n - 1, m] - P[:, n - 1, m] * Q[:, n, m]
            rhs = math.factorial(n + m - 1) / math.factorial(n - m) * (-1) ** m
            np.testing.assert_allclose(lhs, rhs, rtol=1e-11)
    # n = m = 1 needs Q_0^1 = -(x^2-1)^{-1/2} (closed form)
    Q01 = -1.0 / (np.sqrt(x + 1.0) * np.sqrt(x - 1.0))
    np.testing.assert_allclose(P[:, 1, 1] * Q01, -1.0, rtol=1e-14)


@pytest.mark.parametrize("arg", ["real", "imag"])
def test_wronskian(arg):
    """P Q' - P' Q = (-1)^{m+1} (n+m)! / ((n-m)! (x^2-1)) (derivatives d/dx)."""
    x = XS if arg == "real" else 1j * US
    N = 16
    P, Q, dP, dQ = L.legendre_PQ_with_derivatives(x, N)
    for n in range(N + 1):
        for m in range(n + 1):
            W = P[:, n, m] * dQ[:, n, m] - dP[:, n, m] * Q[:, n, m]
            ref = (-1) ** (m + 1) * math.factorial(n + m) / (math.factorial(n - m) * (x * x - 1))
            np.testing.assert_allclose(W, ref, rtol=1e-10)


def test_derivative_against_finite_difference():
    N = 8
    x = np.array([1.3, 2.5])
    h = 1e-6
    P, Q, dP, dQ = L.legendre_PQ_with_derivatives(x, N)
    Pp = L.legendre_P(x + h, N)
    Pm = L.legendre_P(x - h, N)
    Qp = L.legendre_Q(x + h, N)
    Qm = L.legendre_Q(x - h, N)
    np.testing.assert_allclose(dP, (Pp - Pm) / (2 * h), rtol=1e-7, atol=1e-7)
    np.testing.assert_allclose(dQ, (Qp - Qm) / (2 * h), rtol=1e-6, atol=1e-9)


def test_Q_large_argument_asymptotics():
    """Q_n^m(x) ~ (-1)^m 2^n n! (n+m)! / (2n+1)! x^{-n-1}."""
    x = np.array([1e4])
    N = 10
    Q = L.legendre_Q(x, N)
    for n in range(N + 1):
        for m in range(n + 1):
            ref = (-1) ** m * 2 ** n * math.factorial(n) * math.factorial(n + m) / math.factorial(2 * n + 1) * x[0] ** (-n - 1)
            assert abs(Q[0, n, m] / ref - 1) < 1e-6, (n, m)


def test_continued_fraction_iterations_grow_near_one():
    _, it_far = L.continued_fraction_H(np.array([3.0]), 16, 0)
    _, it_near = L.continued_fraction_H(np.array([1.0206]), 16, 0)
    assert it_near > 2 * it_far


def test_real_Y_orthonormal():
    p = 10
    v, wv = np.polynomial.legendre.leggauss(p + 2)
    nphi = 2 * (p + 2)
    phi = 2 * np.pi * np.arange(nphi) / nphi
    V = np.repeat(v, nphi)
    PHI = np.tile(phi, p + 2)
    W = np.repeat(wv, nphi) * 2 * np.pi / nphi
    Y = L.real_Y(V, PHI, p)
    G = Y.T @ (W[:, None] * Y)
    np.testing.assert_allclose(G, np.eye((p + 1) ** 2), atol=1e-13)


def test_real_Y_zonal_and_sectoral():
    v = np.linspace(-1, 1, 7)
    phi = np.linspace(0, 6, 7)
    Y = L.real_Y(v, phi, 5)
    for n in range(6):
        ref = np.sqrt((2 * n + 1) / (4 * np.pi)) * sp.eval_legendre(n, v)
        np.testing.assert_allclose(Y[:, n * n + n], ref, atol=1e-14)
    # Y_1^{+1} = sqrt(3/(4 pi)) sqrt(1-v^2) cos(phi), Y_1^{-1} with sin
    s = np.sqrt(1 - v * v)
    np.testing.assert_allclose(Y[:, 3], np.sqrt(3 / (4 * np.pi)) * s * np.cos(phi), atol=1e-14)
    np.testing.assert_allclose(Y[:, 1], np.sqrt(3 / (4 * np.pi)) * s * np.sin(phi), atol=1e-14)
