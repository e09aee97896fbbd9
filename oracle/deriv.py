"""Normal derivatives S' and D' of the Laplace layer potentials at every
surface node (test infrastructure only).

Sec. 3.3 (Theorem 3 and eq. (dSLevalformula)): with the exterior expansions
of Theorems 1-2,
    S[sigma] = sum b~ sigma~ P(u0) Q(u) Y,   D[mu] = sum b mu^ P'(u0) Q(u) Y
(prolate; oblate with c, c~ and x = i u), the derivative along the outward
normal of the own surface is d/du divided by the scale factor
h_u = a sqrt((u0^2 -+ v^2)/(u0^2 -+ 1)) (Table 2), so on the surface
    S'+ = sum b~ sigma~ P(u0) Q'(u0) j Y / h_u       (exterior limit)
    S'- = sum b~ sigma~ Q(u0) P'(u0) j Y / h_u       (interior limit)
    S'  = (S'+ + S'-)/2                                (Theorem 3, last line)
    D'  = sum b mu^ P'(u0) Q'(u0) j Y / h_u           (continuous across)
with j = 1 (prolate) or i (oblate: d/du of F(i u) is i F'(i u)).
For a target on another particle, the gradient of that particle's exterior
expansion (eq. (dSLevalformula) in Cartesian form, oracle.stokes) is dotted
with the target's normal; far particles use the smooth quadrature of the
differentiated kernels
    dG/dnu_x      = -nu_x . r / (4 pi |r|^3),
    d2G/dnu_x dnu_y = (nu_x . nu_y / |r|^3 - 3 (nu_x . r)(nu_y . r)/|r|^5) / (4 pi),
r = x - y.  Modes as in oracle.laplace: method (self + near + far
quadrature) and exact (self + exterior expansion for every other particle).
"""
from __future__ import annotations

import math

import numpy as np

from . import legendre as L
from .geometry import PROLATE
from .laplace import FOUR_PI, _expand, density_values, multipliers
from .stokes import solid_value_and_gradient


def deriv_multipliers(kind: int, a: float, u0: float, p: int):
    """Per-(n, m>=0) factors k with K'[dens] = Re sum k dens Y / h_u on the
    own surface: dS_plus, dS_minus, dS (average), dD (complex for oblate)."""
    x0 = u0 if kind == PROLATE else 1j * u0
    j = 1.0 if kind == PROLATE else 1j
    _, _, dP, dQ = L.legendre_PQ_with_derivatives(np.array(x0), p)
    mu = multipliers(kind, a, u0, p)
    out = {}
    out["dS_plus"] = mu["ext_S"] * dQ * j
    out["dS_minus"] = mu["int_S"] * dP * j
    out["dS"] = 0.5 * (out["dS_plus"] + out["dS_minus"])
    out["dD"] = mu["ext_D"] * dQ * j
    n = np.arange(p + 1)[:, None]
    m = np.arange(p + 1)[None, :]
    for k in out:
        out[k] = np.where(m <= n, out[k], 0.0)
    return out


def inv_hu_surface(part):
    """1 / h_u at the particle's own nodes: sqrt(u0^2 -+ 1) / (a sqrt(u0^2 -+ v^2))."""
    sgn = -1.0 if part.kind == PROLATE else 1.0
    return math.sqrt(part.u0 ** 2 + sgn) / (part.a * part.sqrt_w)


def self_deriv_values(part, dmult, sigma_t=None, mu_h=None, s_side="pv"):
    """S'[sigma] and D'[mu] of a particle at its own nodes."""
    p = part.p
    Y = L.real_Y(part.v, part.phi, p)
    f = inv_hu_surface(part)
    Sp = Dp = None
    if sigma_t is not None:
        key = {"pv": "dS", "+": "dS_plus", "-": "dS_minus"}[s_side]
        Sp = f * np.real(Y @ (_expand(dmult[key], p) * sigma_t))
    if mu_h is not None:
        Dp = f * np.real(Y @ (_expand(dmult["dD"], p) * mu_h))
    return Sp, Dp


def solid_normal_derivative(part, mult, x, nx, sigma_t=None, mu_h=None):
    """d/dnu_x of the exterior expansions of S[sigma] and D[mu] of one
    particle at global points x with unit directions nx (eq. (dSLevalformula))."""
    p = part.p
    Sp = Dp = None
    if sigma_t is not None:
        _, g = solid_value_and_gradient(part, _expand(mult["ext_S"], p) * sigma_t, x, p)
        Sp = np.sum(g * nx, -1)
    if mu_h is not None:
        _, g = solid_value_and_gradient(part, _expand(mult["ext_D"], p) * mu_h, x, p)
        Dp = np.sum(g * nx, -1)
    return Sp, Dp


def quadrature_deriv_eval(part, x, nx, sigma_t=None, mu_h=None, chunk=2048):
    """Smooth GL x trapezoid quadrature of S' and D' of one particle at
    points x with unit directions nx."""
    s_val, m_val = density_values(part, sigma_t, mu_h)
    x = np.atleast_2d(x)
    nx = np.atleast_2d(nx)
    Sp = np.zeros(x.shape[0]) if sigma_t is not None else None
    Dp = np.zeros(x.shape[0]) if mu_h is not None else None
    for c0 in range(0, x.shape[0], chunk):
        xc, nc = x[c0:c0 + chunk], nx[c0:c0 + chunk]
        r = xc[:, None, :] - part.x[None, :, :]
        d = np.linalg.norm(r, axis=-1)
        rnx = np.einsum("tjk,tk->tj", r, nc)
        if Sp is not None:
            Sp[c0:c0 + chunk] = (-rnx / (FOUR_PI * d ** 3)) @ (part.w * s_val)
        if Dp is not None:
            rny = np.einsum("tjk,jk->tj", r, part.nrm)
            nn = nc @ part.nrm.T
            ker = (nn / d ** 3 - 3.0 * rnx * rny / d ** 5) / FOUR_PI
            Dp[c0:c0 + chunk] = ker @ (part.w * m_val)
    return Sp, Dp


class DerivOracle:
    """S' and D' at the surface nodes of a suspension (Algorithm 1 with the
    differentiated operators, Sec. 4.2 "Other layer potentials")."""

    def __init__(self, geom):
        self.g = geom
        self.mult = [multipliers(P.kind, P.a, P.u0, P.p) for P in geom.parts]
        self.dmult = [deriv_multipliers(P.kind, P.a, P.u0, P.p) for P in geom.parts]

    def apply(self, sigma_t=None, mu_h=None, mode="method", targets=None, parts=("self", "near", "far"),
              s_side="pv"):
        """S'[sigma] and D'[mu] at the node indices `targets` (default all)."""
        g = self.g
        tgt = np.arange(g.N) if targets is None else np.asarray(targets)
        Sp = np.zeros(tgt.shape[0]) if sigma_t is not None else None
        Dp = np.zeros(tgt.shape[0]) if mu_h is not None else None
        owner = g.owner[tgt]
        near = g.near_matrix(None if targets is None else tgt) if mode == "method" else None
        for i, P in enumerate(g.parts):
            si = None if sigma_t is None else sigma_t[i]
            mi = None if mu_h is None else mu_h[i]
            own = owner == i
            if "self" in parts and np.any(own):
                Ss, Ds = self_deriv_values(P, self.dmult[i], si, mi, s_side)
                local = tgt[own] - i * g.G
                if Sp is not None:
                    Sp[own] += Ss[local]
                if Dp is not None:
                    Dp[own] += Ds[local]
            other = ~own
            if mode == "method":
                sel_near, sel_far = other & near[:, i], other & ~near[:, i]
            else:
                sel_near, sel_far = other, np.zeros_like(other)
            for sel, kind in ((sel_near, "near"), (sel_far, "far")):
                if kind not in parts or not np.any(sel):
                    continue
                x, nx = g.x[tgt[sel]], g.nrm[tgt[sel]]
                if kind == "near":
                    Sv, Dv = solid_normal_derivative(P, self.mult[i], x, nx, si, mi)
                else:
                    Sv, Dv = quadrature_deriv_eval(P, x, nx, si, mi)
                if Sp is not None:
                    Sp[sel] += Sv
                if Dp is not None:
                    Dp[sel] += Dv
        return Sp, Dp

    def eval_points(self, X, NX, sigma_t=None, mu_h=None, mode="method"):
        """Directional derivatives d/dn S[sigma] and d/dn D[mu] at arbitrary
        points X (T, 3) in the fluid along unit directions NX (T, 3), with the
        per-point near/far classification of the particle-to-target algorithm
        (Sec. 4.1): near particles by the gradient of the exterior expansion,
        far particles by the differentiated quadrature."""
        g = self.g
        X = np.atleast_2d(np.asarray(X, dtype=np.float64))
        NX = np.atleast_2d(np.asarray(NX, dtype=np.float64))
        near = g.point_near_matrix(X)
        if mode == "exact":
            near = np.ones_like(near)
        Sp = np.zeros(len(X)) if sigma_t is not None else None
        Dp = np.zeros(len(X)) if mu_h is not None else None
        for i, P in enumerate(g.parts):
            si = None if sigma_t is None else sigma_t[i]
            mi = None if mu_h is None else mu_h[i]
            for sel, kind in ((near[:, i], "near"), (~near[:, i], "far")):
                if not np.any(sel):
                    continue
                if kind == "near":
                    Sv, Dv = solid_normal_derivative(P, self.mult[i], X[sel], NX[sel], si, mi)
                else:
                    Sv, Dv = quadrature_deriv_eval(P, X[sel], NX[sel], si, mi)
                if Sp is not None:
                    Sp[sel] += Sv
                if Dp is not None:
                    Dp[sel] += Dv
        return Sp, Dp

