"""Pins of the oracle's Stokes single layer (Sec. 4.3, eq. (stokes))."""
import math

import numpy as np
import pytest

from oracle import brute as B
from oracle import geometry as G
from oracle import legendre as L
from oracle import stokes as ST

SHAPES = [(0, 0.7, 1.6), (1, 1.4, 0.6), (0, 0.35, 1.4), (1, 1.1, 0.3)]


def _single(kind, A, C, p, seed):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(4)
    c = rng.standard_normal(3)
    g = G.SuspensionGeom(np.array([kind]), np.array([A]), np.array([C]), c[None], q[None], p)
    return g, q, c, rng


def _laplace_to_stokes(O, P, f_t, x, p):
    cs = [O._ext_coef(0, np.pad(f_t[k], (0, (p + 2) ** 2 - (p + 1) ** 2)), p + 1) for k in range(3)]
    cy = O._ext_coef(0, ST.ydotf_modified_coefficients(P, f_t, p), p + 1)
    F, Gr = zip(*[ST.solid_value_and_gradient(P, cs[k], x, p + 1) for k in range(3)])
    _, Gy = ST.solid_value_and_gradient(P, cy, x, p + 1)
    xc = x - P.center
    U = np.zeros((len(x), 3))
    for k in range(3):
        U[:, k] = 0.5 * (F[k] + Gy[:, k] - sum(xc[:, j] * Gr[j][:, k] for j in range(3)))
    return U


@pytest.mark.parametrize("kind,A,C", SHAPES)
def test_laplace_to_stokes_matches_brute_stokeslet(kind, A, C):
    p = 5
    g, q, c, rng = _single(kind, A, C, p, 3)
    f = rng.standard_normal((3, (p + 1) ** 2))
    P = g.parts[0]
    idx = rng.integers(0, P.G, 5)
    h = 0.2 * min(A, C) + 0.15
    x = P.x[idx] + h * np.array([1.0, 2.0, 4.0, 8.0, 1.5])[:, None] * P.nrm[idx]
    U = _laplace_to_stokes(ST.StokesOracle(g), P, f, x, p)
    Ub = B.brute_stokeslet(kind, A, C, c, q, p, x, f, nv=220, nphi=440)
    assert np.max(np.abs(U - Ub)) / np.max(np.abs(Ub)) < 1e-11


@pytest.mark.parametrize("kind,A,C", SHAPES)
def test_translating_spheroid_uniform_velocity(kind, A, C):
    """f = e x (equilibrium density): the single layer is a rigid translation
    on the surface (uniform velocity), evaluated through the self limits."""
    p = 6
    g, q, c, rng = _single(kind, A, C, p, 5)
    f = np.zeros((1, 3, (p + 1) ** 2))
    e = np.array([0.3, -0.5, 0.8])
    f[0, :, 0] = e
    U = ST.StokesOracle(g).apply(f, "method")
    assert np.max(np.ptp(U, axis=0)) < 1e-12 * np.max(np.abs(U))
    # continuity: the exterior formula 1e-7 outside the surface gives the same velocity
    P = g.parts[0]
    xo = P.x[:5] + 1e-7 * P.nrm[:5]
    Uo = _laplace_to_stokes(ST.StokesOracle(g), P, f[0], xo, p)
    assert np.max(np.abs(Uo - U[:5])) < 1e-5 * np.max(np.abs(U))


def test_sphere_limit_two_thirds():
    """Nearly spherical prolate (a -> 0): S_stk[f] = (2/3) f for uniform f on
    the unit sphere."""
    p = 4
    g, q, c, rng = _single(0, 1.0, 1.0 + 1e-6, p, 1)
    P = g.parts[0]
    f = np.zeros((1, 3, (p + 1) ** 2))
    e = np.array([1.0, -2.0, 0.5])
    # sigma = e * Y00 / sqrt(u0^2 - v^2) ~ e * Y00 / u0
    f[0, :, 0] = e
    U = ST.StokesOracle(g).apply(f, "method")
    sigma = (1 / math.sqrt(4 * math.pi)) / P.u0
    np.testing.assert_allclose(U.mean(0), 2.0 / 3.0 * sigma * e, rtol=1e-6)


@pytest.mark.parametrize("kind,A,C", SHAPES[:2])
def test_ydotf_transform_exact(kind, A, C):
    p = 4
    g, q, c, rng = _single(kind, A, C, p, 8)
    P = g.parts[0]
    f = rng.standard_normal((3, (p + 1) ** 2))
    cy = ST.ydotf_modified_coefficients(P, f, p)
    v = rng.uniform(-1, 1, 20)
    ph = rng.uniform(0, 2 * np.pi, 20)
    sgn = -1 if kind == 0 else 1
    sw = np.sqrt(P.u0 ** 2 + sgn * v * v)
    fv = np.stack([L.real_Y(v, ph, p) @ f[k] / sw for k in range(3)], -1)
    y = G.local_point(kind, P.a, P.u0, v, ph) @ P.R.T
    ref = np.sum(y * fv, -1) * sw
    np.testing.assert_allclose(L.real_Y(v, ph, p + 1) @ cy, ref, atol=1e-13 * np.abs(ref).max())


def test_two_particle_method_vs_exact():
    """Method (near analytic + Stokeslet far quadrature) converges to the
    exact operator on a well separated pair."""
    from paper_2506_20809_gb300 import inputs as I

    s = I.Suspension(np.array([0, 1], np.int32), np.array([0.6, 1.2]), np.array([1.3, 0.5]),
                     np.array([[0.0, 0, 0], [3.2, 0.4, -0.2]]),
                     np.array([[1.0, 0, 0, 0], [0.8, 0.2, -0.5, 0.26]]), 10)
    s.quat /= np.linalg.norm(s.quat, axis=1, keepdims=True)
    g = G.SuspensionGeom.from_suspension(s, near_factor=0.5)
    f = np.random.default_rng(2).standard_normal((2, 3, 121)) / (1 + np.floor(np.sqrt(np.arange(121)))) ** 2
    O = ST.StokesOracle(g)
    Um = O.apply(f, "method")
    Ue = O.apply(f, "exact")
    assert np.max(np.abs(Um - Ue)) / np.max(np.abs(Ue)) < 1e-6


# ---------------------------------------------------------------------------
# velocity and pressure at arbitrary points


def _two_for_points(p):
    from paper_2506_20809_gb300 import inputs as I
    from oracle import geometry as G

    kind = np.array([0, 1], np.int32)
    A = np.array([0.6, 1.1])
    C = np.array([1.3, 0.5])
    cen = np.array([[0.0, 0.0, 0.0], [3.2, 0.3, -0.2]])
    quat = np.random.default_rng(8).standard_normal((2, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    s = I.Suspension(kind, A, C, cen, quat, p)
    return s, G.SuspensionGeom.from_suspension(s)


def test_points_velocity_and_pressure_match_brute_force():
    """Exact mode at points around two particles against oversampled direct
    quadrature of the Stokeslet and of the printed pressure kernel."""
    from oracle import brute as BR
    from oracle import stokes as OSK
    from paper_2506_20809_gb300 import inputs as I

    p = 5
    s, g = _two_for_points(p)
    f = np.random.default_rng(3).standard_normal((2, 3, (p + 1) ** 2))
    X = I.shell_points(s, distances=(0.3, 0.8), per_particle=4, seed=4)
    U, Pr = OSK.StokesOracle(g).eval_points(X, f, "exact")
    Ub, Pb = np.zeros_like(U), np.zeros_like(Pr)
    for i, P in enumerate(g.parts):
        Ub += BR.brute_stokeslet(P.kind, P.A, P.C, P.center, s.quat[i], p, X, f[i], nv=200, nphi=400)
        Pb += BR.brute_stokes_pressure(P.kind, P.A, P.C, P.center, s.quat[i], p, X, f[i], nv=200, nphi=400)
    assert np.max(np.abs(U - Ub)) < 1e-10 * np.max(np.abs(Ub))
    assert np.max(np.abs(Pr - Pb)) < 1e-10 * np.max(np.abs(Pb))


def test_points_satisfy_the_stokes_equations():
    """-Laplace u + grad p = 0 and div u = 0 (viscosity 1) at points in the
    fluid, by central differences of the exact-mode velocity and pressure;
    this fixes the sign of the pressure independently of any printed
    kernel."""
    from oracle import stokes as OSK

    p = 5
    s, g = _two_for_points(p)
    f = np.random.default_rng(5).standard_normal((2, 3, (p + 1) ** 2))
    O = OSK.StokesOracle(g)
    x0 = np.array([[1.6, 0.9, 0.4], [-0.4, 1.5, 0.9]])
    h = 2e-3
    E = np.eye(3)
    U0, P0 = O.eval_points(x0, f, "exact")
    lap = np.zeros_like(U0)
    gradp = np.zeros((2, 3))
    div = np.zeros(2)
    for k in range(3):
        Up, Pp = O.eval_points(x0 + h * E[k], f, "exact")
        Um, Pm = O.eval_points(x0 - h * E[k], f, "exact")
        lap += (Up - 2 * U0 + Um) / h ** 2
        gradp[:, k] = (Pp - Pm) / (2 * h)
        div += (Up[:, k] - Um[:, k]) / (2 * h)
    scale = np.max(np.abs(lap))
    assert np.max(np.abs(-lap + gradp)) < 1e-4 * scale
    assert np.max(np.abs(div)) < 1e-5 * scale
    # the opposite sign fails
    assert np.max(np.abs(-lap - gradp)) > 0.1 * scale


def test_points_method_matches_exact_near_surfaces():
    from oracle import stokes as OSK
    from paper_2506_20809_gb300 import inputs as I

    p = 8
    s, g = _two_for_points(p)
    f = np.random.default_rng(6).standard_normal((2, 3, (p + 1) ** 2)) / (1 + np.arange((p + 1) ** 2))
    X = I.shell_points(s, distances=(1e-1, 1e-3, 1e-5), per_particle=5, seed=7)
    O = OSK.StokesOracle(g)
    Um, Pm = O.eval_points(X, f, "method")
    Ue, Pe = O.eval_points(X, f, "exact")
    # far pairs carry the smooth quadrature's error (p = 8, one major
    # semi-axis away at least); near pairs are analytic in both modes
    assert np.max(np.abs(Um - Ue)) < 1e-5 * np.max(np.abs(Ue))
    assert np.max(np.abs(Pm - Pe)) < 1e-5 * np.max(np.abs(Pe))
