"""Pins of the oracle's Laplace layer potentials (Theorems 1-2, Algorithm 1)
against what the mathematics fixes: sphere limits, the spheroid capacitance,
Gauss's law, the jump relations, Green's representation formula and
oversampled direct quadrature."""
import math

import numpy as np
import pytest

from oracle import brute as B
from oracle import geometry as G
from oracle import laplace as LP
from oracle import legendre as L

SHAPES = [(0, 1.0, 2.0), (1, 1.5, 0.75), (0, 0.3, 1.5), (1, 1.2, 0.24), (0, 0.9, 1.0), (1, 1.0, 0.95)]


def _particle(kind, A, C, p, seed=0, center=None):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(4)
    c = rng.standard_normal(3) if center is None else np.asarray(center, float)
    return G.Particle(kind, A, C, c, q, p), q, c


@pytest.mark.parametrize("kind", [0, 1])
def test_sphere_limit_eigenvalues(kind):
    """a u0 = 1, u0 -> inf: the unit sphere, where S[Y_n] = Y_n/(2n+1) and the
    principal-value D[Y_n] = -Y_n/(2(2n+1)); errors decay like u0^-2."""
    p = 8
    errs_S, errs_D = [], []
    for u0 in (10.0, 100.0, 1000.0):
        a = 1.0 / u0
        mu = LP.multipliers(kind, a, u0, p)
        n = np.arange(p + 1)[:, None] * np.ones((1, p + 1), int)
        m = np.arange(p + 1)[None, :] * np.ones((p + 1, 1), int)
        ok = m <= n
        # sigma = Y (plain) corresponds to sigma~ ~= u0 Y in the modified basis
        lamS = np.real(mu["self_S"]) * u0
        lamD = np.real(mu["self_D"])
        errs_S.append(np.max(np.abs(lamS * (2 * n + 1) - 1)[ok]))
        errs_D.append(np.max(np.abs(lamD + 1.0 / (2 * (2 * n + 1)))[ok]))
        assert np.max(np.abs(mu["self_S"].imag)) < 1e-12
    for e in (errs_S, errs_D):
        assert e[2] < 1e-5
        assert e[1] / e[2] > 50 and e[0] / e[1] > 50     # O(u0^-2)


@pytest.mark.parametrize("kind,A,C", SHAPES)
def test_capacitance(kind, A, C):
    """Equilibrium density: sigma~ = e_00 gives a constant surface potential V
    and total charge q; q / V is the textbook capacitance
    prolate 8 pi a / log((u0+1)/(u0-1)), oblate 4 pi a / arccot(u0)."""
    P, _, _ = _particle(kind, A, C, 10)
    mult = LP.multipliers(kind, P.a, P.u0, 10)
    sig = np.zeros(121)
    sig[0] = 1.0
    S, _ = LP.self_values(P, mult, sig, None)
    assert np.ptp(S) < 1e-13 * abs(S.mean())
    sval, _ = LP.density_values(P, sig, None)
    q = np.sum(P.w * sval)
    cap = q / S.mean()
    u0, a = P.u0, P.a
    ref = 8 * math.pi * a / math.log((u0 + 1) / (u0 - 1)) if kind == 0 else 4 * math.pi * a / math.atan(1 / u0)
    assert abs(cap / ref - 1) < 1e-12
    # exterior potential q Q_0(u) / (4 pi a) (prolate) / q arccot(u)/(4 pi a) (oblate)
    x = P.x[:5] + np.array([0.3, 0.7, 1.5, 3.0, 9.0])[:, None] * P.nrm[:5]
    Sx, _ = LP.solid_eval(P, mult, x, sig, None)
    u, _, _ = P.to_spheroidal(x)
    radial = 0.5 * np.log((u + 1) / (u - 1)) if kind == 0 else np.arctan(1 / u)
    np.testing.assert_allclose(Sx, q * radial / (4 * math.pi * a), rtol=1e-12)


@pytest.mark.parametrize("kind,A,C", [(0, 1 / 64, 1.0), (1, 1.0, 1 / 64), (0, 1 / 26, 1.0), (1, 1.0, 0.1)])
def test_capacitance_high_aspect_ratio(kind, A, C):
    """The conductor at aspect ratios up to 64 (the paper's stress tests):
    constant surface potential, the textbook capacitance, and the exterior
    potential q Q_0(u) / (4 pi a) down to 1e-3 from the surface, where u is
    within 1e-4 of u0 = 1 (prolate) and Q_0 varies fastest."""
    p = 12
    P, _, _ = _particle(kind, A, C, p)
    mult = LP.multipliers(kind, P.a, P.u0, p)
    sig = np.zeros((p + 1) ** 2)
    sig[0] = 1.0
    S, _ = LP.self_values(P, mult, sig, None)
    assert np.ptp(S) < 1e-12 * abs(S.mean())
    sval, _ = LP.density_values(P, sig, None)
    q = np.sum(P.w * sval)
    u0, a = P.u0, P.a
    ref = 8 * math.pi * a / math.log((u0 + 1) / (u0 - 1)) if kind == 0 else 4 * math.pi * a / math.atan(1 / u0)
    assert abs(q / S.mean() / ref - 1) < 1e-11
    k = np.arange(0, len(P.x), 7)
    x = np.concatenate([P.x[k] + d * P.nrm[k] for d in (1e-3, 1e-2, 1e-1, 1.0)])
    Sx, _ = LP.solid_eval(P, mult, x, sig, None)
    u, _, _ = P.to_spheroidal(x)
    radial = 0.5 * np.log((u + 1) / (u - 1)) if kind == 0 else np.arctan(1 / u)
    np.testing.assert_allclose(Sx, q * radial / (4 * math.pi * a), rtol=1e-11)


@pytest.mark.parametrize("kind,A,C", SHAPES)
def test_gauss_law_double_layer(kind, A, C):
    """D[1] = -1/2 on the surface (principal value), 0 outside, -1 inside."""
    P, _, c = _particle(kind, A, C, 6)
    mult = LP.multipliers(kind, P.a, P.u0, 6)
    mu = np.zeros(49)
    mu[0] = math.sqrt(4 * math.pi)
    _, D = LP.self_values(P, mult, None, mu)
    np.testing.assert_allclose(D, -0.5, atol=1e-13)
    xo = P.x[::7] + 0.4 * P.nrm[::7]
    _, Do = LP.solid_eval(P, mult, xo, None, mu, "exterior")
    np.testing.assert_allclose(Do, 0.0, atol=1e-13)
    xi = c + 0.6 * (P.x[::7] - c)
    _, Di = LP.solid_eval(P, mult, xi, None, mu, "interior")
    np.testing.assert_allclose(Di, -1.0, atol=1e-13)
    # the smooth quadrature of the same density gives 0 at a far point too
    _, Df = LP.quadrature_eval(P, c + np.array([[6.0, 1.0, -2.0]]), None, mu)
    assert abs(Df[0]) < 1e-8          # quadrature error of the 7 x 14 rule


@pytest.mark.parametrize("kind,A,C", SHAPES)
def test_solid_expansions_match_brute_force(kind, A, C):
    """Exterior and interior formulas of Theorems 1-2 agree with an
    oversampled direct quadrature of the band-limited density."""
    p = 6
    P, q, c = _particle(kind, A, C, p, seed=11)
    mult = LP.multipliers(kind, P.a, P.u0, p)
    rng = np.random.default_rng(5)
    sig = rng.standard_normal((p + 1) ** 2)
    mu = rng.standard_normal((p + 1) ** 2)
    idx = rng.integers(0, P.G, 6)
    h = 0.25 * min(A, C) + 0.1
    xo = P.x[idx] + h * np.array([1.0, 1.5, 2.0, 4.0, 8.0, 1.2])[:, None] * P.nrm[idx]
    xi = c + np.array([0.5, 0.3, 0.7, 0.2, 0.6, 0.4])[:, None] * (P.x[idx] - c)
    for side, x in (("exterior", xo), ("interior", xi)):
        S, D = LP.solid_eval(P, mult, x, sig, mu, side)
        Sb, Db = B.brute_layers(kind, A, C, c, q, p, x, sig, mu, nv=220, nphi=440)
        assert LP.normwise_rel_err(S, Sb) < 1e-11, side
        assert LP.normwise_rel_err(D, Db) < 1e-11, side


@pytest.mark.parametrize("kind,A,C", SHAPES[:4])
def test_jump_relations(kind, A, C):
    """u -> u0 from outside / inside: S is continuous, D -> D_pv +- mu/2."""
    p = 8
    P, _, _ = _particle(kind, A, C, p, seed=2)
    mult = LP.multipliers(kind, P.a, P.u0, p)
    rng = np.random.default_rng(9)
    sig = rng.standard_normal((p + 1) ** 2)
    mu = rng.standard_normal((p + 1) ** 2)
    S0, D0 = LP.self_values(P, mult, sig, mu)
    _, mval = LP.density_values(P, None, mu)
    sub = np.arange(0, P.G, 5)
    scale = np.max(np.abs(mval))
    one_sided, d_avg = [], []
    for eps in (1e-3, 1e-5):
        vals = {}
        for sgn in (+1, -1):
            u = P.u0 * (1 + sgn * eps)
            xl = G.local_point(kind, P.a, u, P.v[sub], P.phi[sub])
            x = xl @ P.R.T + P.center
            vals[sgn] = LP.solid_eval(P, mult, x, sig, mu, "exterior" if sgn > 0 else "interior")
        (Sp, Dp), (Sm, Dm) = vals[1], vals[-1]
        # one-sided limits: S+ = S- = S, D+- = D -+ ... = D +- mu/2, first order in eps
        one_sided.append(max(np.max(np.abs(Sp - S0[sub])), np.max(np.abs(Sm - S0[sub])),
                             np.max(np.abs(Dp - (D0[sub] + 0.5 * mval[sub]))),
                             np.max(np.abs(Dm - (D0[sub] - 0.5 * mval[sub])))) / scale)
        # dD/dnu is continuous, so the two-sided average of D is second order
        d_avg.append(np.max(np.abs(0.5 * (Dp + Dm) - D0[sub])) / scale)
    assert one_sided[1] < 0.02 * one_sided[0] and one_sided[1] < 1e-2
    assert d_avg[1] < 2e-3 * d_avg[0] + 1e-12 and d_avg[1] < 1e-7


def _analysis(P, fn, p, modified=False, nv=64, nphi=128):
    """Coefficients of a surface function (oracle-only forward transform by a
    fine GL x trapezoid rule); `modified` gives the Sec. 3.2 basis."""
    v, wv = np.polynomial.legendre.leggauss(nv)
    phi = 2 * np.pi * np.arange(nphi) / nphi
    V = np.repeat(v, nphi)
    PHI = np.tile(phi, nv)
    W = np.repeat(wv, nphi) * 2 * np.pi / nphi
    xl = G.local_point(P.kind, P.a, P.u0, V, PHI)
    x = xl @ P.R.T + P.center
    g = xl / np.array([P.A ** 2, P.A ** 2, P.C ** 2])
    nrm = (g / np.linalg.norm(g, axis=1, keepdims=True)) @ P.R.T
    val = fn(x, nrm)
    if modified:
        sgn = -1 if P.kind == 0 else 1
        val = val * np.sqrt(P.u0 ** 2 + sgn * V * V)
    return L.real_Y(V, PHI, p).T @ (W * val)


@pytest.mark.parametrize("kind,A,C", [(0, 1.0, 1.8), (1, 1.5, 0.9)])
def test_green_representation_on_surface(kind, A, C):
    """f harmonic outside (charges inside): D[f] - S[df/dnu] = f/2 on the
    surface; f harmonic inside (charge outside): S[df/dnu] - D[f] = f/2.
    Pins the on-surface (self) multipliers; the error decays with p."""
    rng = np.random.default_rng(4)
    q = rng.standard_normal(4)
    c = np.zeros(3)
    P0 = G.Particle(kind, A, C, c, q, 2)
    xin = (rng.uniform(-0.15, 0.15, (3, 3)) * np.array([A, A, C])) @ P0.R.T
    qin = rng.uniform(-0.5, 0.5, 3)
    xout = np.array([[3.5 * max(A, C), 0.5, -0.3]])
    qout = np.array([0.7])

    def make(xs, qs):
        def f(x, n):
            r = x[:, None, :] - xs[None]
            return (qs / (4 * np.pi * np.linalg.norm(r, axis=-1))).sum(1)

        def df(x, n):
            r = x[:, None, :] - xs[None]
            d = np.linalg.norm(r, axis=-1)
            return -(qs * np.einsum("tsk,tk->ts", r, n) / (4 * np.pi * d ** 3)).sum(1)
        return f, df

    for (xs, qs, sign) in ((xin, qin, +1), (xout, qout, -1)):
        f, df = make(xs, qs)
        errs = []
        for p in (6, 12, 18):
            P = G.Particle(kind, A, C, c, q, p)
            mult = LP.multipliers(kind, P.a, P.u0, p)
            fh = _analysis(P, f, p)
            st = _analysis(P, df, p, modified=True)
            Sv, _ = LP.self_values(P, mult, st, None)
            _, Dv = LP.self_values(P, mult, None, fh)
            fx = f(P.x, P.nrm)
            errs.append(np.max(np.abs(sign * (Dv - Sv) - fx / 2)) / np.max(np.abs(fx)))
        assert errs[2] < 1e-5 and errs[2] < errs[1] < errs[0], errs


def test_far_quadrature_converges_to_exact():
    """Smooth quadrature (Sec. 4.1) of a band-limited density at a target one
    diameter away converges spectrally to the exterior formula."""
    kind, A, C = 0, 0.6, 1.4
    rng = np.random.default_rng(8)
    sig6 = rng.standard_normal(49)
    mu6 = rng.standard_normal(49)
    errs = []
    for p in (6, 10, 16, 24):
        P, _, c = _particle(kind, A, C, p, seed=1)
        mult = LP.multipliers(kind, P.a, P.u0, p)
        sig = np.zeros((p + 1) ** 2)
        sig[:49] = sig6
        mu = np.zeros((p + 1) ** 2)
        mu[:49] = mu6
        x = c + np.array([[2.8, 0.4, 0.1], [0.0, -3.0, 1.0]])
        Se, De = LP.solid_eval(P, mult, x, sig, mu)
        Sq, Dq = LP.quadrature_eval(P, x, sig, mu)
        errs.append(max(LP.normwise_rel_err(Sq, Se), LP.normwise_rel_err(Dq, De)))
    assert errs[-1] < 1e-12 and errs[0] > errs[1] > errs[2]


@pytest.mark.parametrize("kind,A,C", SHAPES[:4])
def test_point_spheroid_distance(kind, A, C):
    rng = np.random.default_rng(3)
    # axis and equator special cases
    np.testing.assert_allclose(G.point_spheroid_distance(np.array([[0, 0, C + 0.7]]), A, C), 0.7, atol=1e-13)
    np.testing.assert_allclose(G.point_spheroid_distance(np.array([[0.6 + A, 0, 0]]), A, C), 0.6, atol=1e-13)
    # random exterior points vs dense sampling of the surface
    x = rng.standard_normal((40, 3)) * 1.5 * max(A, C)
    x = x[(x[:, 0] ** 2 + x[:, 1] ** 2) / A ** 2 + x[:, 2] ** 2 / C ** 2 > 1.05]
    d = G.point_spheroid_distance(x, A, C)
    th = np.linspace(0, np.pi, 1601)
    ph = np.linspace(0, 2 * np.pi, 1600, endpoint=False)
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    y = np.stack([A * np.sin(TH) * np.cos(PH), A * np.sin(TH) * np.sin(PH), C * np.cos(TH)], -1).reshape(-1, 3)
    for xi, di in zip(x, d):
        ds = np.min(np.linalg.norm(y - xi, axis=1))
        assert di <= ds + 1e-12 and ds - di < 2e-5


def test_near_sets_lattice():
    from paper_2506_20809_gb300 import inputs as I
    s = I.config_suspension(1)
    g = G.SuspensionGeom.from_suspension(s)
    near = g.near_matrix()
    assert not np.any(near[np.arange(g.N), g.owner])
    assert g.near_margin() > 1e-9
    D = g.distances()
    thr = np.array([P.major for P in g.parts])
    other = np.ones_like(near)
    other[np.arange(g.N), g.owner] = False
    assert np.all((D < thr[None]) == near | ~other)
    assert np.all(D[other] > 0)           # no target inside another particle


def test_planted_sign_error_is_caught(monkeypatch):
    """Planting a dropped (-1)^m in the oracle's single-layer constant makes
    the brute-force pin fail (checks the pin's sensitivity)."""
    p = 4
    P, q, c = _particle(0, 0.8, 1.6, p, seed=21)
    good = LP.multipliers(0, P.a, P.u0, p)
    bad = {k: v.copy() for k, v in good.items()}
    for m in range(1, p + 1, 2):
        bad["ext_S"][:, m] *= -1
    rng = np.random.default_rng(1)
    sig = rng.standard_normal((p + 1) ** 2)
    x = P.x[:4] + 0.5 * P.nrm[:4]
    Sb, _ = B.brute_layers(0, 0.8, 1.6, c, q, p, x, sig, None, nv=120, nphi=240)
    Sg, _ = LP.solid_eval(P, good, x, sig, None)
    Sx, _ = LP.solid_eval(P, bad, x, sig, None)
    assert LP.normwise_rel_err(Sg, Sb) < 1e-11
    assert LP.normwise_rel_err(Sx, Sb) > 1e-3


@pytest.mark.parametrize("kind,A,C", [(0, 1 / 64, 1.0), (1, 1.0, 0.1), (0, 1.0, 2.0), (1, 1.5, 0.75)])
def test_coordinate_inverse_round_trip(kind, A, C):
    """Table 1 and its inverse: points built from (u, v, phi) come back to
    (u, v) within rounding, including points on the symmetry axis (v = +-1
    exactly, so every m > 0 harmonic vanishes there), next to the focal
    segment or ring, and close to the equator."""
    a, u0 = G.spheroid_params(kind, A, C)
    rng = np.random.default_rng(3)
    for u in (u0 * (1 + 1e-3), u0 * 1.5, 3.0 * u0 + 0.5):
        v = np.concatenate([[-1.0, 1.0, 0.0, 1e-9, -1e-9], rng.uniform(-1, 1, 40), 1 - 10.0 ** -rng.uniform(2, 9, 10)])
        phi = rng.uniform(0, 2 * math.pi, v.shape)
        xl = G.local_point(kind, a, np.full(v.shape, u), v, phi)
        u2, v2, _ = G.cart_to_spheroidal(xl, kind, a)
        np.testing.assert_allclose(u2, u, rtol=1e-13)
        np.testing.assert_allclose(v2, v, atol=2e-13)
        assert v2[0] == -1.0 and v2[1] == 1.0
