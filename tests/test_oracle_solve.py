"""Pins of the oracle's forward transform and exterior boundary-value solves
(Sec. 5.1) against what the mathematics fixes: exactness of the transform
on band-limited functions, the sphere-limit spectrum of the completed
double-layer and single-layer Neumann operators, the paper's completion
scaling table at its breakpoints, and the paper's own test: the potential of
point charges inside the particles is recovered at shell points outside
them by the Dirichlet and Neumann solves, with errors decaying in p."""
import math

import numpy as np
import pytest

from oracle import geometry as G
from oracle import legendre as L
from oracle import solve as SV
from paper_2506_20809_gb300 import inputs as I


@pytest.mark.parametrize("kind,A,C", [(0, 0.6, 1.4), (1, 1.3, 0.5)])
def test_transform_is_exact_on_band_limited(kind, A, C):
    p = 7
    P = G.Particle(kind, A, C, np.zeros(3), np.array([0.3, 0.5, -0.2, 0.8]), p)
    c = np.random.default_rng(1).standard_normal((p + 1) ** 2)
    for mod in (False, True):
        back = SV.analysis(P, SV.synthesis(P, c, mod), mod)
        assert np.max(np.abs(back - c)) < 1e-13 * np.max(np.abs(c))


def test_eta_table_breakpoints():
    """Values of the heuristic table at chosen aspect ratios."""
    e2 = math.sqrt(0.75)
    area_pro_2 = 2 * math.pi * 0.25 * (1 + math.asin(e2) / (0.5 * e2))
    assert SV.eta_table(0, 0.5, 1.0, "etaCI") == pytest.approx(0.5 / area_pro_2, rel=1e-14)
    assert SV.eta_table(1, 1.0, 0.2, "etaCI") == 0.06
    assert SV.eta_table(0, 0.5, 1.0, "etaS") == 0.5
    assert SV.eta_table(0, 0.25, 1.0, "etaS") == pytest.approx(1 / (2 * 0.25 * math.log(4)), rel=1e-14)
    assert SV.eta_table(1, 1.0, 0.5, "etaS") == pytest.approx(0.75, rel=1e-14)
    assert SV.eta_table(1, 1.0, 0.2, "etaS") == 1.0
    assert SV.eta_table(0, 0.3, 1.0, "S") == SV.eta_table(1, 1.0, 0.3, "CI") == 1.0
    # the unit-major area at eps = 1 is the sphere's
    assert SV.surface_area_unit_major(0, 1.0 - 1e-12) == pytest.approx(4 * math.pi, rel=1e-6)
    assert SV.surface_area_unit_major(1, 1.0 - 1e-12) == pytest.approx(4 * math.pi, rel=1e-6)


def _single(kind, u0, p):
    a = 1.0 / u0
    if kind == 0:
        C, A = a * u0, a * math.sqrt(u0 * u0 - 1)
    else:
        C, A = a * u0, a * math.sqrt(u0 * u0 + 1)
    s = I.Suspension(np.array([kind], np.int32), np.array([A]), np.array([C]), np.zeros((1, 3)),
                     np.array([[1.0, 0.0, 0.0, 0.0]]), p)
    return G.SuspensionGeom.from_suspension(s)


@pytest.mark.parametrize("kind", [0, 1])
def test_sphere_limit_spectra(kind):
    """Near-sphere (u0 = 200): 1/2 + D has eigenvalue n/(2n+1) on Y_n (the
    n = 0 null mode is lifted by the completion), and the Neumann operator
    -1/2 + S' has -(n+1)/(2n+1)."""
    p = 5
    g = _single(kind, 200.0, p)
    B = SV.BVPOracle(g, mode="exact")
    for n, m in ((1, 0), (2, -1), (3, 2), (5, 5)):
        e = np.zeros((1, (p + 1) ** 2))
        e[0, L.coeff_index(n, m)] = 1.0
        y = B.dirichlet_apply(e, "S")
        assert y[0, L.coeff_index(n, m)] == pytest.approx(n / (2 * n + 1) + 1 / (2 * n + 1), abs=1e-3)
        y = B.dirichlet_apply(e, "CI")
        assert y[0, L.coeff_index(n, m)] == pytest.approx(n / (2 * n + 1), abs=1e-3)
        assert np.max(np.abs(np.delete(y[0], L.coeff_index(n, m)))) < 1e-3
        y = B.neumann_apply(e)
        assert y[0, L.coeff_index(n, m)] == pytest.approx(-(n + 1) / (2 * n + 1), abs=1e-3)
    e = np.zeros((1, (p + 1) ** 2))
    e[0, 0] = 1.0
    # n = 0: 1/2 + D annihilates the constant; C_I adds (int Y_00 dS)/|x - c| = sqrt(4 pi)
    y = B.dirichlet_apply(e, "CI")
    assert y[0, 0] == pytest.approx(math.sqrt(4 * math.pi) * math.sqrt(4 * math.pi), rel=2e-3)


def _charges_setup(p, seed=0):
    """Three spheroids as in the paper's Dirichlet test (centres (0,0,0),
    (5,0,0), (3.2,3.2,3.2), aspect ratio about 1.8) with two charges of
    strength in [-0.5, 0.5] near each centre; one oblate to cover both kinds."""
    rng = np.random.default_rng(seed)
    kind = np.array([0, 1, 0], np.int32)
    A = np.array([0.8, 1.3, 0.75])
    C = np.array([1.4, 0.72, 1.35])
    cen = np.array([[0.0, 0, 0], [5, 0, 0], [3.2, 3.2, 3.2]])
    quat = I.random_quaternions(rng, 3)
    R = I._quat_to_matrix(quat)
    xs = np.concatenate([cen[i] + (rng.uniform(-0.05, 0.05, (2, 3)) * np.array([A[i], A[i], C[i]])) @ R[i].T
                         for i in range(3)])
    qs = rng.uniform(-0.5, 0.5, len(xs))
    s = I.Suspension(kind, A, C, cen, quat, p)
    return s, xs, qs


def _f(xs, qs, x):
    return (qs / (4 * np.pi * np.linalg.norm(np.atleast_2d(x)[:, None, :] - xs[None], axis=-1))).sum(1)


def _dfdn(xs, qs, x, n):
    r = x[:, None, :] - xs[None]
    d = np.linalg.norm(r, axis=-1)
    return -(qs * np.einsum("tsk,tk->ts", r, n) / (4 * np.pi * d ** 3)).sum(1)


def test_dirichlet_and_neumann_recover_the_charges_potential():
    """The paper's Laplace BVP test: f from charges inside the particles;
    the completed double-layer (etaS) Dirichlet solve and the single-layer
    Neumann solve reproduce f at shells 1e-1 .. 1e-5 outside the surfaces,
    with the error decaying in p."""
    errs = {"D": [], "N": []}
    for p in (4, 6, 8):
        s, xs, qs = _charges_setup(p)
        g = G.SuspensionGeom.from_suspension(s)
        X = I.shell_points(s, distances=(1e-1, 1e-3, 1e-5), per_particle=4, seed=1)
        B = SV.BVPOracle(g)
        ref = _f(xs, qs, X)
        mu, st, q = B.solve_dirichlet(_f(xs, qs, g.x), "etaS")
        errs["D"].append(np.max(np.abs(B.eval_dirichlet(X, mu, st, q) - ref)) / np.max(np.abs(ref)))
        rho = B.solve_neumann(_dfdn(xs, qs, g.x, g.nrm))
        errs["N"].append(np.max(np.abs(B.eval_neumann(X, rho) - ref)) / np.max(np.abs(ref)))
    for k, e in errs.items():
        assert e[2] < 1e-2 and e[2] < e[1] / 2 < e[0] / 4, (k, e)


@pytest.mark.parametrize("completion", ["CI", "etaCI", "S"])
def test_other_completions_solve_the_same_problem(completion):
    """Every completion yields a density whose representation matches f."""
    s, xs, qs = _charges_setup(6, seed=2)
    g = G.SuspensionGeom.from_suspension(s)
    X = I.shell_points(s, distances=(1e-2,), per_particle=4, seed=3)
    B = SV.BVPOracle(g)
    mu, st, q = B.solve_dirichlet(_f(xs, qs, g.x), completion)
    ref = _f(xs, qs, X)
    assert np.max(np.abs(B.eval_dirichlet(X, mu, st, q) - ref)) / np.max(np.abs(ref)) < 5e-2
