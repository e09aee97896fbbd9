"""Pins of the oracle's Stokes double layer (Laplace form of Sec. 4.3's
remark) against oversampled direct quadrature of the stresslet, the
constant-density identity, rigid-body motions (annihilated outside, -q/2 on
the surface), the jump across the surface, and the method's split."""
import math

import numpy as np
import pytest

from oracle import brute as BR
from oracle import geometry as G
from oracle import solve as SV
from oracle import stokes_dl as SD
from paper_2506_20809_gb300 import inputs as I


def _two(p, gap=0.9):
    kind = np.array([0, 1], np.int32)
    A = np.array([0.6, 1.1])
    C = np.array([1.3, 0.5])
    cen = np.array([[0.0, 0.0, 0.0], [1.3 + 1.1 + gap, 0.3, -0.2]])
    quat = np.random.default_rng(8).standard_normal((2, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    s = I.Suspension(kind, A, C, cen, quat, p)
    return s, G.SuspensionGeom.from_suspension(s)


def test_exact_matches_brute_force():
    p = 6
    s, g = _two(p)
    q = np.random.default_rng(1).standard_normal((2, 3, (p + 1) ** 2))
    X = I.shell_points(s, distances=(0.3, 0.8), per_particle=4, seed=2)
    U = SD.StokesDLOracle(g).eval_points(X, q, "exact")
    Ub = sum(BR.brute_stresslet(P.kind, P.A, P.C, P.center, s.quat[i], p, X, q[i], nv=200, nphi=400)
             for i, P in enumerate(g.parts))
    assert np.max(np.abs(U - Ub)) < 1e-11 * np.max(np.abs(Ub))


def _rigid(g, i, U, Om):
    P = g.parts[i]
    vals = U[None, :] + np.cross(Om[None, :], P.x - P.center)
    return np.stack([SV.analysis(P, vals[:, k]) for k in range(3)])


@pytest.mark.parametrize("which", ["constant", "rigid"])
def test_rigid_motions(which):
    """A rigid-body motion q = U + Omega x (y - c) on one particle: the double
    layer vanishes outside that particle and equals -q/2 on its surface
    (principal value); constants are the special case Omega = 0."""
    p = 5
    s, g = _two(p)
    rng = np.random.default_rng(3)
    q = np.zeros((2, 3, (p + 1) ** 2))
    Om = np.zeros(3) if which == "constant" else rng.standard_normal(3)
    q[1] = _rigid(g, 1, rng.standard_normal(3), Om)
    O = SD.StokesDLOracle(g)
    out = O.apply(q, "exact")
    P = g.parts[1]
    Y = np.stack([SV.synthesis(P, q[1, k]) for k in range(3)], -1)
    assert np.max(np.abs(out[g.G:] + 0.5 * Y)) < 1e-12 * np.max(np.abs(Y))
    assert np.max(np.abs(out[:g.G])) < 1e-12 * np.max(np.abs(Y))
    X = I.shell_points(s, distances=(1e-3, 0.5), per_particle=4, seed=4)
    assert np.max(np.abs(O.eval_points(X, q, "exact"))) < 1e-11 * np.max(np.abs(Y))


def test_jump_to_the_exterior_limit():
    """Points approaching a surface along its normal: D_stk -> D_pv + q/2."""
    p = 6
    s, g = _two(p)
    q = np.random.default_rng(5).standard_normal((2, 3, (p + 1) ** 2))
    O = SD.StokesDLOracle(g)
    idx = np.arange(0, g.G, 9)
    pv = O.apply(q, "exact", targets=idx)
    P = g.parts[0]
    qv = np.stack([SV.synthesis(P, q[0, k]) for k in range(3)], -1)[idx]
    errs = []
    for h in (1e-4, 1e-6):
        out = O.eval_points(g.x[idx] + h * g.nrm[idx], q, "exact")
        errs.append(np.max(np.abs(out - (pv + 0.5 * qv))) / np.max(np.abs(qv)))
    assert errs[1] < 1e-4 and errs[1] < errs[0] / 10, errs


def test_method_close_to_exact():
    p = 8
    s, g = _two(p, gap=2.5)
    q = np.random.default_rng(6).standard_normal((2, 3, (p + 1) ** 2)) / (1 + np.arange((p + 1) ** 2))
    O = SD.StokesDLOracle(g)
    assert np.max(np.abs(O.apply(q, "method") - O.apply(q, "exact"))) < 1e-5 * np.max(np.abs(O.apply(q, "exact")))
