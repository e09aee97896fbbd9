"""Laplace single / double layer apply for the oracle (test infrastructure only).

Theorem 1 (double layer, Sec. 3.1) and Theorem 2 (single layer in the
modified basis Y/sqrt(u0^2 -+ v^2), Sec. 3.2), m >= 0, with
    prolate: b = K (-1)^m (u0^2-1),        b~ = a K (-1)^m sqrt(u0^2-1)
    oblate:  c = K (-1)^{m+1} (u0^2+1),    c~ = i a K (-1)^m sqrt(u0^2+1)
    K = (n-m)!/(n+m)!;  oblate Legendre arguments are x = i u, P' = dP/dx.
    exterior (u > u0):  S: b~ P(u0) Q(u) Y     D: b P'(u0) Q(u) Y
    interior (u < u0):  S: b~ Q(u0) P(u) Y     D: b Q'(u0) P(u) Y
    on the surface:     S: b~ P Q (u0)         D (principal value): the average
                        of D+ = b P' Q and D- = b Q' P at u0.
The real basis (cosine / sine per |m|) uses the |m| multipliers: the operator
commutes with rotation about, and reflection through a plane containing, the
symmetry axis, so the m and -m modes share one eigenvalue.

Sec. 4 / Algorithm 1: u(x) = sum_i K_i[sigma_i](x) at every surface node,
self term by the diagonal multipliers, near particles by the exterior
expansion, far particles by the smooth GL x trapezoid quadrature
    S: sum_j w_j sigma(y_j) G(x, y_j),  D: sum_j w_j mu(y_j) dG/dnu_y(x, y_j),
    G = 1/(4 pi |x - y|),  dG/dnu_y = nu(y).(x - y) / (4 pi |x - y|^3).
Input densities: sigma by its modified-basis coefficients sigma~ (Sec. 3.2,
Sec. 4.2 "Other layer potentials"), mu by its plain coefficients mu^.

Two apply modes:
  method : self + near (analytic) + far (quadrature): what the GPU computes.
  exact  : self + exterior expansion for every other particle: the exact
           operator applied to the band-limited density.
"""
from __future__ import annotations

import math

import numpy as np

from . import legendre as L
from .geometry import PROLATE, SuspensionGeom

FOUR_PI = 4.0 * math.pi


def multipliers(kind: int, a: float, u0: float, p: int):
    """Per-(n, m>=0) factors of Theorems 1-2 (complex for oblate).
    Returns dict of arrays [n, m]: ext_S, ext_D, int_S, int_D, self_S, self_D,
    self_Dp (D+), self_Dm (D-)."""
    x0 = u0 if kind == PROLATE else 1j * u0
    P, Q, dP, dQ = L.legendre_PQ_with_derivatives(np.array(x0), p)
    out = {k: np.zeros((p + 1, p + 1), dtype=np.complex128) for k in
           ("ext_S", "ext_D", "int_S", "int_D", "self_S", "self_D", "self_Dp", "self_Dm")}
    for n in range(p + 1):
        for m in range(n + 1):
            K = math.factorial(n - m) / math.factorial(n + m)
            if kind == PROLATE:
                b = K * (-1) ** m * (u0 * u0 - 1.0)
                bt = a * K * (-1) ** m * math.sqrt(u0 * u0 - 1.0)
            else:
                b = K * (-1) ** (m + 1) * (u0 * u0 + 1.0)
                bt = 1j * a * K * (-1) ** m * math.sqrt(u0 * u0 + 1.0)
            Pn, Qn, dPn, dQn = P[n, m], Q[n, m], dP[n, m], dQ[n, m]
            out["ext_S"][n, m] = bt * Pn
            out["ext_D"][n, m] = b * dPn
            out["int_S"][n, m] = bt * Qn
            out["int_D"][n, m] = b * dQn
            out["self_S"][n, m] = bt * Pn * Qn
            out["self_Dp"][n, m] = b * dPn * Qn
            out["self_Dm"][n, m] = b * dQn * Pn
            out["self_D"][n, m] = 0.5 * (out["self_Dp"][n, m] + out["self_Dm"][n, m])
    return out


def _expand(table, p):
    """[n, m>=0] table -> per-coefficient-index vector (|m| shared)."""
    ns, ms = L.abs_m_table(p)
    return table[ns, ms]


def synth(coef, v, phi, p):
    """sum_nm coef_nm Y_nm(v, phi): inverse surface transform (dense)."""
    return L.real_Y(v, phi, p) @ coef


def density_values(part, sigma_t=None, mu_h=None):
    """Node values of sigma (from modified coefficients) and mu (plain)."""
    p = part.p
    Y = L.real_Y(part.v, part.phi, p)
    s = None if sigma_t is None else (Y @ sigma_t) / part.sqrt_w
    m = None if mu_h is None else Y @ mu_h
    return s, m


def self_values(part, mult, sigma_t=None, mu_h=None, d_side="pv"):
    """On-surface S[sigma] and D[mu] of a particle at its own nodes."""
    p = part.p
    Y = L.real_Y(part.v, part.phi, p)
    S = D = None
    if sigma_t is not None:
        lam = _expand(mult["self_S"], p)
        S = np.real(Y @ (lam * sigma_t))
    if mu_h is not None:
        key = {"pv": "self_D", "+": "self_Dp", "-": "self_Dm"}[d_side]
        lam = _expand(mult[key], p)
        D = np.real(Y @ (lam * mu_h))
    return S, D


def solid_eval(part, mult, x, sigma_t=None, mu_h=None, side="exterior"):
    """S and D of one particle at global points x using the exterior (u > u0)
    or interior (u < u0) expansions of Theorems 1-2."""
    p = part.p
    u, v, phi = part.to_spheroidal(x)
    xa = u if part.kind == PROLATE else 1j * u
    P = L.legendre_P(xa, p + 1)
    if side == "exterior":
        F = L.legendre_Q(xa, p + 1, P)[..., :p + 1, :p + 1]
        kS, kD = "ext_S", "ext_D"
    else:
        F = P[..., :p + 1, :p + 1]
        kS, kD = "int_S", "int_D"
    ns, ms = L.abs_m_table(p)
    Fe = F[..., ns, ms]                         # (T, ncoef) radial factor per index
    Y = L.real_Y(v, phi, p)
    S = D = None
    if sigma_t is not None:
        S = np.real(np.sum(Fe * Y * (_expand(mult[kS], p) * sigma_t), axis=-1))
    if mu_h is not None:
        D = np.real(np.sum(Fe * Y * (_expand(mult[kD], p) * mu_h), axis=-1))
    return S, D


def quadrature_eval(part, x, sigma_t=None, mu_h=None, chunk=4096):
    """Smooth GL x trapezoid quadrature of S and D of one particle at points x."""
    s_val, m_val = density_values(part, sigma_t, mu_h)
    x = np.atleast_2d(x)
    S = np.zeros(x.shape[0]) if sigma_t is not None else None
    D = np.zeros(x.shape[0]) if mu_h is not None else None
    for c0 in range(0, x.shape[0], chunk):
        xc = x[c0:c0 + chunk]
        r = xc[:, None, :] - part.x[None, :, :]
        dist = np.linalg.norm(r, axis=-1)
        if S is not None:
            S[c0:c0 + chunk] = (1.0 / (FOUR_PI * dist)) @ (part.w * s_val)
        if D is not None:
            rn = np.einsum("tjk,jk->tj", r, part.nrm)
            D[c0:c0 + chunk] = (rn / (FOUR_PI * dist ** 3)) @ (part.w * m_val)
    return S, D


class LaplaceOracle:
    """Apply of S and D at all surface nodes of a suspension (Algorithm 1)."""

    def __init__(self, geom: SuspensionGeom):
        self.g = geom
        self.mult = [multipliers(P.kind, P.a, P.u0, P.p) for P in geom.parts]

    def apply(self, sigma_t=None, mu_h=None, mode="method", targets=None, parts=("self", "near", "far")):
        """S and D at the target node indices `targets` (default: all nodes).
        sigma_t, mu_h: (M, (p+1)^2).  Returns (S, D) arrays (or None)."""
        g = self.g
        tgt = np.arange(g.N) if targets is None else np.asarray(targets)
        S = np.zeros(tgt.shape[0]) if sigma_t is not None else None
        D = np.zeros(tgt.shape[0]) if mu_h is not None else None
        owner = g.owner[tgt]
        near = g.near_matrix(None if targets is None else tgt) if mode == "method" else None
        for i, P in enumerate(g.parts):
            si = None if sigma_t is None else sigma_t[i]
            mi = None if mu_h is None else mu_h[i]
            own = owner == i
            if "self" in parts and np.any(own):
                Ss, Ds = self_values(P, self.mult[i], si, mi)
                local = tgt[own] - i * g.G
                if S is not None:
                    S[own] += Ss[local]
                if D is not None:
                    D[own] += Ds[local]
            other = ~own
            if mode == "method":
                sel_near = other & near[:, i]
                sel_far = other & ~near[:, i]
            else:
                sel_near = other
                sel_far = np.zeros_like(other)
            if "near" in parts and np.any(sel_near):
                Sn, Dn = solid_eval(P, self.mult[i], g.x[tgt[sel_near]], si, mi, "exterior")
                if S is not None:
                    S[sel_near] += Sn
                if D is not None:
                    D[sel_near] += Dn
            if "far" in parts and np.any(sel_far):
                Sf, Df = quadrature_eval(P, g.x[tgt[sel_far]], si, mi)
                if S is not None:
                    S[sel_far] += Sf
                if D is not None:
                    D[sel_far] += Df
        return S, D

    def eval_points(self, X, sigma_t=None, mu_h=None, mode="method"):
        """S and D at arbitrary points X (T, 3) in the fluid (Sec. 4.1,
        particle-to-target algorithm): every (point, particle) pair is
        classified by the point's own exact distance; near particles by the
        exterior expansion of Theorems 1-2, far particles by the smooth
        quadrature.  mode 'exact': exterior expansion for every particle.
        Raises ValueError for a point inside a spheroid."""
        g = self.g
        X = np.atleast_2d(np.asarray(X, dtype=np.float64))
        near = g.point_near_matrix(X)
        if mode == "exact":
            near = np.ones_like(near)
        S = np.zeros(X.shape[0]) if sigma_t is not None else None
        D = np.zeros(X.shape[0]) if mu_h is not None else None
        for i, P in enumerate(g.parts):
            si = None if sigma_t is None else sigma_t[i]
            mi = None if mu_h is None else mu_h[i]
            for sel, fn in ((near[:, i], "near"), (~near[:, i], "far")):
                if not np.any(sel):
                    continue
                if fn == "near":
                    Sv, Dv = solid_eval(P, self.mult[i], X[sel], si, mi, "exterior")
                else:
                    Sv, Dv = quadrature_eval(P, X[sel], si, mi)
                if S is not None:
                    S[sel] += Sv
                if D is not None:
                    D[sel] += Dv
        return S, D

    def point_far_pair_count(self, X):
        """(point, far source node) pairs of eval_points in method mode."""
        near = self.g.point_near_matrix(X)
        return int(np.sum(~near) * self.g.G)

    def far_pair_count(self, targets=None):
        """Number of (target, far source node) pairs of the method."""
        g = self.g
        tgt = np.arange(g.N) if targets is None else np.asarray(targets)
        near = g.near_matrix(None if targets is None else tgt)
        n_skip = near.sum(axis=1) + 1
        return int(np.sum((g.M - n_skip) * g.G))


def normwise_rel_err(x, ref):
    """max |x - ref| / max |ref|."""
    x = np.asarray(x)
    ref = np.asarray(ref)
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(x - ref)) / den) if den > 0 else float(np.max(np.abs(x - ref)))
