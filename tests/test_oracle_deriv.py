"""Pins of the oracle's normal-derivative operators S' and D' (Theorem 3,
eq. (dSLevalformula)) and of the point-target evaluation (Sec. 4.1,
particle-to-target algorithm) against what the mathematics fixes: sphere
limits, the jump of S', the conductor's field, finite differences of the
(independently pinned) potentials, Green's representation formula
differentiated along the normal, and oversampled direct quadrature."""
import math

import numpy as np
import pytest

from oracle import brute as B
from oracle import deriv as DV
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
    """a u0 = 1, u0 -> inf (unit sphere): S'+[Y_n] = -(n+1)/(2n+1) Y_n,
    S'-[Y_n] = n/(2n+1) Y_n, S' = -1/(2(2n+1)) Y_n and
    D'[Y_n] = -n(n+1)/(2n+1) Y_n (derivatives of r^-(n+1) and r^n); errors
    decay like u0^-2."""
    p = 8
    n = np.arange(p + 1)[:, None] * np.ones((1, p + 1), int)
    m = np.arange(p + 1)[None, :] * np.ones((p + 1, 1), int)
    ok = m <= n
    ref = {"dS_plus": -(n + 1) / (2 * n + 1), "dS_minus": n / (2 * n + 1), "dS": -1 / (2 * (2 * n + 1)),
           "dD": -n * (n + 1) / (2 * n + 1)}
    errs = {k: [] for k in ref}
    sgn = -1 if kind == 0 else 1
    for u0 in (10.0, 100.0, 1000.0):
        a = 1.0 / u0
        dm = DV.deriv_multipliers(kind, a, u0, p)
        inv_hu = math.sqrt(u0 * u0 + sgn) / (a * u0)       # 1/h_u at v = 0
        for k in ref:
            lam = np.real(dm[k]) * inv_hu * (u0 if k != "dD" else 1.0)   # modified basis for S
            errs[k].append(np.max(np.abs(lam - ref[k])[ok]))
            assert np.max(np.abs(np.imag(dm[k]))) < 1e-12
    for k, e in errs.items():
        assert e[2] < 2e-5, k
        assert e[1] / e[2] > 50 and e[0] / e[1] > 50, k


@pytest.mark.parametrize("kind,A,C", SHAPES)
def test_single_layer_derivative_jump(kind, A, C):
    """S'+ - S'- = -sigma at every node, for every mode (the Wronskian of
    P and Q at u0 against the modified-basis weight)."""
    p = 10
    P, _, _ = _particle(kind, A, C, p, seed=3)
    dm = DV.deriv_multipliers(kind, P.a, P.u0, p)
    sig = np.random.default_rng(1).standard_normal((p + 1) ** 2)
    Sp, _ = DV.self_deriv_values(P, dm, sig, None, "+")
    Sm, _ = DV.self_deriv_values(P, dm, sig, None, "-")
    s, _ = LP.density_values(P, sig, None)
    assert np.max(np.abs(Sp - Sm + s)) < 1e-12 * np.max(np.abs(s))


@pytest.mark.parametrize("kind,A,C", SHAPES)
def test_conductor_field(kind, A, C):
    """Equilibrium density (sigma~ = e_00): the potential is constant inside,
    so S'- = 0, S'+ = -sigma and the principal value is -sigma/2."""
    p = 8
    P, _, _ = _particle(kind, A, C, p)
    dm = DV.deriv_multipliers(kind, P.a, P.u0, p)
    sig = np.zeros((p + 1) ** 2)
    sig[0] = 1.0
    s, _ = LP.density_values(P, sig, None)
    for side, ref in (("+", -s), ("-", 0 * s), ("pv", -0.5 * s)):
        Sv, _ = DV.self_deriv_values(P, dm, sig, None, side)
        assert np.max(np.abs(Sv - ref)) < 1e-12 * np.max(np.abs(s)), side


@pytest.mark.parametrize("kind,A,C", SHAPES[:4])
def test_one_sided_finite_differences(kind, A, C):
    """S'+-, D' against second-order one-sided differences in u of the
    exterior / interior potentials (Theorems 1-2, pinned elsewhere), scaled
    by 1/h_u; the error falls like h^2."""
    p = 8
    P, _, _ = _particle(kind, A, C, p, seed=2)
    mult = LP.multipliers(kind, P.a, P.u0, p)
    dm = DV.deriv_multipliers(kind, P.a, P.u0, p)
    rng = np.random.default_rng(7)
    sig = rng.standard_normal((p + 1) ** 2)
    mu = rng.standard_normal((p + 1) ** 2)
    sub = np.arange(0, P.G, 4)
    S0, D0 = LP.self_values(P, mult, sig, mu)
    _, mval = LP.density_values(P, None, mu)
    f = DV.inv_hu_surface(P)[sub]
    Spl, Dpl = DV.self_deriv_values(P, dm, sig, mu, "+")
    Smi, _ = DV.self_deriv_values(P, dm, sig, mu, "-")
    errs = []
    for h in (1e-4 * P.u0, 2.5e-5 * P.u0):
        vals = {}
        for sgn in (+1, -1):
            pts = []
            for k in (1, 2):
                xl = G.local_point(kind, P.a, P.u0 + sgn * k * h, P.v[sub], P.phi[sub])
                pts.append(LP.solid_eval(P, mult, xl @ P.R.T + P.center, sig, mu,
                                         "exterior" if sgn > 0 else "interior"))
            vals[sgn] = pts
        # exterior: S(u0) = S0, D+(u0) = D0 + mu/2; interior: D-(u0) = D0 - mu/2
        dS_out = (-3 * S0[sub] + 4 * vals[1][0][0] - vals[1][1][0]) / (2 * h) * f
        dS_in = (3 * S0[sub] - 4 * vals[-1][0][0] + vals[-1][1][0]) / (2 * h) * f
        Dp0 = D0[sub] + 0.5 * mval[sub]
        dD_out = (-3 * Dp0 + 4 * vals[1][0][1] - vals[1][1][1]) / (2 * h) * f
        sc = max(np.max(np.abs(Spl)), np.max(np.abs(Dpl)))
        errs.append(max(np.max(np.abs(dS_out - Spl[sub])), np.max(np.abs(dS_in - Smi[sub])),
                        np.max(np.abs(dD_out - Dpl[sub]))) / sc)
    assert errs[1] < 1e-5 and (errs[1] < errs[0] / 8 or errs[1] < 1e-8), errs


@pytest.mark.parametrize("kind,A,C", SHAPES[:4])
def test_gradient_of_exterior_expansion(kind, A, C):
    """d/dnu of the exterior expansions at off-surface points against
    central differences of the potentials along nu."""
    p = 7
    P, _, _ = _particle(kind, A, C, p, seed=5)
    mult = LP.multipliers(kind, P.a, P.u0, p)
    rng = np.random.default_rng(2)
    sig = rng.standard_normal((p + 1) ** 2)
    mu = rng.standard_normal((p + 1) ** 2)
    idx = rng.integers(0, P.G, 8)
    x = P.x[idx] + (0.1 + 0.5 * rng.random(8))[:, None] * max(A, C) * P.nrm[idx]
    nx = rng.standard_normal((8, 3))
    nx /= np.linalg.norm(nx, axis=1, keepdims=True)
    Sg, Dg = DV.solid_normal_derivative(P, mult, x, nx, sig, mu)
    h = 1e-5
    Sa, Da = LP.solid_eval(P, mult, x + h * nx, sig, mu)
    Sb, Db = LP.solid_eval(P, mult, x - h * nx, sig, mu)
    assert LP.normwise_rel_err(Sg, (Sa - Sb) / (2 * h)) < 1e-7
    assert LP.normwise_rel_err(Dg, (Da - Db) / (2 * h)) < 1e-7


def test_far_quadrature_of_derivatives():
    """The differentiated quadrature equals central differences of the
    quadrature of the potentials, and converges spectrally to the gradient
    of the exterior expansion one diameter away."""
    kind, A, C = 1, 1.3, 0.6
    rng = np.random.default_rng(4)
    sig = rng.standard_normal(36)
    mu = rng.standard_normal(36)
    x = np.array([[3.1, 0.4, -0.8], [-0.5, 2.9, 1.7]])
    nx = rng.standard_normal((2, 3))
    nx /= np.linalg.norm(nx, axis=1, keepdims=True)
    P, _, _ = _particle(kind, A, C, 5, seed=1, center=np.zeros(3))
    Sq, Dq = DV.quadrature_deriv_eval(P, x, nx, sig, mu)
    h = 1e-5
    Sa, Da = LP.quadrature_eval(P, x + h * nx, sig, mu)
    Sb, Db = LP.quadrature_eval(P, x - h * nx, sig, mu)
    assert LP.normwise_rel_err(Sq, (Sa - Sb) / (2 * h)) < 1e-8
    assert LP.normwise_rel_err(Dq, (Da - Db) / (2 * h)) < 1e-8
    errs = []
    for p in (5, 10, 20):
        Pp, _, _ = _particle(kind, A, C, p, seed=1, center=np.zeros(3))
        s = np.zeros((p + 1) ** 2)
        m = np.zeros((p + 1) ** 2)
        s[:36], m[:36] = sig, mu
        mult = LP.multipliers(kind, Pp.a, Pp.u0, p)
        Se, De = DV.solid_normal_derivative(Pp, mult, x, nx, s, m)
        Sq, Dq = DV.quadrature_deriv_eval(Pp, x, nx, s, m)
        errs.append(max(LP.normwise_rel_err(Sq, Se), LP.normwise_rel_err(Dq, De)))
    assert errs[2] < 1e-10 and errs[2] < errs[1] < errs[0], errs


def _forward(P, fn, p, modified=False, nv=64, nphi=128):
    """Coefficients of a surface function by a fine GL x trapezoid rule
    (oracle-only forward transform); `modified` gives the Sec. 3.2 basis."""
    v, wv = np.polynomial.legendre.leggauss(nv)
    phi = 2 * np.pi * np.arange(nphi) / nphi
    V, PHI = np.repeat(v, nphi), np.tile(phi, nv)
    W = np.repeat(wv, nphi) * 2 * np.pi / nphi
    xl = G.local_point(P.kind, P.a, P.u0, V, PHI)
    gl = xl / np.array([P.A ** 2, P.A ** 2, P.C ** 2])
    nrm = (gl / np.linalg.norm(gl, axis=1, keepdims=True)) @ P.R.T
    val = fn(xl @ P.R.T + P.center, nrm)
    if modified:
        val = val * np.sqrt(P.u0 ** 2 + (-1 if P.kind == 0 else 1) * V * V)
    return L.real_Y(V, PHI, p).T @ (W * val)


def _charges(xs, qs):
    def f(x, n):
        r = x[:, None, :] - xs[None]
        return (qs / (4 * np.pi * np.linalg.norm(r, axis=-1))).sum(1)

    def df(x, n):
        r = x[:, None, :] - xs[None]
        d = np.linalg.norm(r, axis=-1)
        return -(qs * np.einsum("tsk,tk->ts", r, n) / (4 * np.pi * d ** 3)).sum(1)
    return f, df


@pytest.mark.parametrize("kind,A,C", [(0, 1.0, 1.8), (1, 1.5, 0.9)])
def test_green_representation_differentiated(kind, A, C):
    """Green's formula along the normal: f harmonic outside (charges inside)
    gives D'[f] - S'[df/dnu] = (df/dnu)/2 on the surface; f harmonic inside
    (a charge outside) gives S'[df/dnu] - D'[f] = (df/dnu)/2.  Pins the
    hypersingular D' and the principal-value S' together; spectral in p."""
    rng = np.random.default_rng(4)
    q = rng.standard_normal(4)
    c = np.zeros(3)
    P0 = G.Particle(kind, A, C, c, q, 2)
    xin = (rng.uniform(-0.15, 0.15, (3, 3)) * np.array([A, A, C])) @ P0.R.T
    qin = rng.uniform(-0.5, 0.5, 3)
    xout = np.array([[3.5 * max(A, C), 0.5, -0.3]])
    qout = np.array([0.7])
    for xs, qs, sign in ((xin, qin, +1), (xout, qout, -1)):
        f, df = _charges(xs, qs)
        errs = []
        for p in (6, 12, 18):
            P = G.Particle(kind, A, C, c, q, p)
            dm = DV.deriv_multipliers(kind, P.a, P.u0, p)
            fh = _forward(P, f, p)
            st = _forward(P, df, p, modified=True)
            Sv, _ = DV.self_deriv_values(P, dm, st, None)
            _, Dv = DV.self_deriv_values(P, dm, None, fh)
            g = df(P.x, P.nrm)
            errs.append(np.max(np.abs(sign * (Dv - Sv) - g / 2)) / np.max(np.abs(g)))
        assert errs[2] < 1e-4 and errs[2] < errs[1] < errs[0], errs


QUAT2 = np.random.default_rng(3).standard_normal((2, 4))


def _two_particles(p, gap=0.3):
    s_kind = np.array([0, 1])
    A = np.array([0.6, 1.1])
    C = np.array([1.3, 0.5])
    cen = np.array([[0.0, 0.0, 0.0], [1.1 + 1.3 + gap, 0.2, -0.1]])
    return G.SuspensionGeom(s_kind, A, C, cen, QUAT2, p, near_factor=1.0)


def test_suspension_green_identity_exact_mode():
    """Two particles, charges inside both: f is harmonic outside their union,
    so D'[f] - S'[df/dnu] = (df/dnu)/2 at every node when self and neighbour
    interactions are all analytic (exact mode); spectral in p."""
    rng = np.random.default_rng(6)
    errs = []
    for p in (8, 14, 20):
        g = _two_particles(p, gap=1.0)
        xs = np.concatenate([P.center + 0.1 * rng.uniform(-1, 1, (2, 3)) * min(P.A, P.C) for P in g.parts])
        qs = rng.uniform(-0.5, 0.5, len(xs))
        f, df = _charges(xs, qs)
        fh = np.stack([_forward(P, f, p) for P in g.parts])
        st = np.stack([_forward(P, df, p, modified=True) for P in g.parts])
        Sp, _ = DV.DerivOracle(g).apply(st, None, "exact")
        _, Dp = DV.DerivOracle(g).apply(None, fh, "exact")
        gv = df(g.x, g.nrm)
        errs.append(np.max(np.abs(Dp - Sp - gv / 2)) / np.max(np.abs(gv)))
    assert errs[2] < 1e-3 and errs[2] < errs[1] < errs[0], errs


def test_method_vs_exact_and_parts():
    """The method (near analytic, far quadrature) agrees with the exact
    operator up to the far-quadrature error, and its parts add up."""
    p = 10
    g = _two_particles(p, gap=2.5)
    rng = np.random.default_rng(1)
    sig = rng.standard_normal((2, (p + 1) ** 2)) / (1 + np.arange((p + 1) ** 2)) ** 0.5
    mu = rng.standard_normal((2, (p + 1) ** 2)) / (1 + np.arange((p + 1) ** 2)) ** 0.5
    O = DV.DerivOracle(g)
    Sm, Dm = O.apply(sig, mu, "method")
    Se, De = O.apply(sig, mu, "exact")
    assert LP.normwise_rel_err(Sm, Se) < 1e-5 and LP.normwise_rel_err(Dm, De) < 1e-5
    tot = [O.apply(sig, mu, "method", parts=(k,)) for k in ("self", "near", "far")]
    assert np.allclose(sum(t[0] for t in tot), Sm, rtol=0, atol=1e-13 * np.max(np.abs(Sm)))
    assert np.allclose(sum(t[1] for t in tot), Dm, rtol=0, atol=1e-13 * np.max(np.abs(Dm)))


def test_planted_error_in_dD_is_caught(monkeypatch):
    """A dropped factor j (the d/du of F(i u)) in D' breaks the differentiated
    Green identity for an oblate."""
    orig = DV.deriv_multipliers

    def bad(kind, a, u0, p):
        out = orig(kind, a, u0, p)
        if kind == 1:
            out["dD"] = out["dD"] / 1j
        return out
    monkeypatch.setattr(DV, "deriv_multipliers", bad)
    with pytest.raises(AssertionError):
        test_green_representation_differentiated(1, 1.5, 0.9)


# ---------------------------------------------------------------------------
# particle-to-target evaluation at arbitrary points


def _shell_points(g, dists, per, seed=0):
    """Points at distance ~d along the outward normal of random nodes."""
    rng = np.random.default_rng(seed)
    pts = []
    for d in dists:
        idx = rng.integers(0, g.N, per)
        pts.append(g.x[idx] + d * g.nrm[idx])
    return np.concatenate(pts)


def test_points_exact_matches_brute_force():
    """eval_points in exact mode is the exterior expansion at every particle:
    it matches an oversampled direct quadrature of both particles' densities."""
    p = 6
    g = _two_particles(p, gap=0.8)
    rng = np.random.default_rng(2)
    sig = rng.standard_normal((2, (p + 1) ** 2))
    mu = rng.standard_normal((2, (p + 1) ** 2))
    X = _shell_points(g, [0.25, 0.5, 1.0], 4, seed=1)
    S, D = LP.LaplaceOracle(g).eval_points(X, sig, mu, "exact")
    Sb, Db = np.zeros(len(X)), np.zeros(len(X))
    for i, P in enumerate(g.parts):
        s_i, d_i = B.brute_layers(P.kind, P.A, P.C, P.center, QUAT2[i], p, X, sig[i], mu[i], nv=220, nphi=440)
        Sb += s_i
        Db += d_i
    assert LP.normwise_rel_err(S, Sb) < 1e-10
    assert LP.normwise_rel_err(D, Db) < 1e-10


def test_points_method_classification_and_consistency():
    """Shell points at distances 10^-k (the paper's shell test): pairs inside
    the near threshold use the analytic expansion, so points close to a
    surface agree with the exact operator to rounding; far pairs carry only
    the smooth-quadrature error.  At a surface node the point path gives the
    exterior limits: S (continuous) and D+ = D + mu/2."""
    p = 10
    g = _two_particles(p, gap=2.0)
    rng = np.random.default_rng(5)
    sig = rng.standard_normal((2, (p + 1) ** 2)) / (1 + np.arange((p + 1) ** 2))
    mu = rng.standard_normal((2, (p + 1) ** 2)) / (1 + np.arange((p + 1) ** 2))
    O = LP.LaplaceOracle(g)
    X = _shell_points(g, [1e-1, 1e-2, 1e-3, 1e-4], 6, seed=2)
    near = g.point_near_matrix(X)
    assert near.sum(1).min() >= 1            # every shell point is near its own particle
    Sm, Dm = O.eval_points(X, sig, mu, "method")
    Se, De = O.eval_points(X, sig, mu, "exact")
    assert LP.normwise_rel_err(Sm, Se) < 1e-6 and LP.normwise_rel_err(Dm, De) < 1e-6
    assert O.point_far_pair_count(X) == int((~near).sum()) * g.G
    # at the nodes themselves: exterior limits of the on-surface apply
    idx = np.arange(0, g.N, 37)
    Sn, Dn = O.eval_points(g.x[idx], sig, mu, "exact")
    Sa, Da = O.apply(sig, mu, "exact", targets=idx)
    mval = np.concatenate([LP.density_values(P, None, mu[i])[1] for i, P in enumerate(g.parts)])[idx]
    assert LP.normwise_rel_err(Sn, Sa) < 1e-10
    assert LP.normwise_rel_err(Dn, Da + 0.5 * mval) < 1e-9


def test_points_inside_a_spheroid_are_rejected():
    g = _two_particles(4)
    O = LP.LaplaceOracle(g)
    inside = g.parts[1].center[None, :] + 0.01
    with pytest.raises(ValueError):
        O.eval_points(inside, np.zeros((2, 25)), None)


def test_point_derivatives_are_gradients_of_the_point_values():
    """Directional derivatives at points equal central differences of the
    point values along the direction (method mode, the same near/far split)."""
    p = 8
    g = _two_particles(p, gap=1.5)
    rng = np.random.default_rng(12)
    sig = rng.standard_normal((2, (p + 1) ** 2)) / (1 + np.arange((p + 1) ** 2))
    mu = rng.standard_normal((2, (p + 1) ** 2)) / (1 + np.arange((p + 1) ** 2))
    X = _shell_points(g, [0.05, 0.3, 2.0], 4, seed=3)
    NX = rng.standard_normal(X.shape)
    NX /= np.linalg.norm(NX, axis=1, keepdims=True)
    Sp, Dp = DV.DerivOracle(g).eval_points(X, NX, sig, mu, "exact")
    O = LP.LaplaceOracle(g)
    h = 1e-5
    Sa, Da = O.eval_points(X + h * NX, sig, mu, "exact")
    Sb, Db = O.eval_points(X - h * NX, sig, mu, "exact")
    assert LP.normwise_rel_err(Sp, (Sa - Sb) / (2 * h)) < 1e-7
    assert LP.normwise_rel_err(Dp, (Da - Db) / (2 * h)) < 1e-7
