"""Stokes double layer (viscosity 1) through Laplace potentials (test
infrastructure only).

The paper remarks (Sec. 4.3) that the Stokes double layer can be written in
terms of Laplace double-layer potentials and their gradients and evaluated
with the same methodology.  With the stresslet
    D_stk[q](x)_i = 3/(4 pi) int (r . q)(r . nu) r_i / |r|^5 dS(y),  r = x - y,
(nu the outward normal; the sign that gives D_stk[const] = -q inside and 0
outside, like the Laplace double layer D used throughout) and the identity
    r_i r_j r_k / |r|^5 = (1/3) r_i d_j d_k (1/|r|) + (1/3) delta_jk r_i / |r|^3,
one gets, with S[s] = int s / (4 pi |r|) and D[m] = int nu . r m / (4 pi |r|^3),
    D_stk[q]_i = -x_i sum_j d_j D[q_j] + sum_j d_j D[y_i q_j] - d_i S[q . nu],
x and y measured from the source particle's centre (translation invariant).
The densities q_j are band-limited of order p (plain coefficients, the D
input convention); y_i q_j is band-limited of order p + 1 (y is a degree-one
function on the spheroid), and so is (q . nu) sqrt(u0^2 -+ v^2) (nu times the
modified-basis weight is degree one), so all thirteen expansions are exact at
order p + 1; their coefficients come from a product quadrature exact for
that degree.

Near particles: the gradients of the exterior expansions at the target.
Own particle: the same formulas at u = u0 give the exterior limit D_stk^+;
the principal value on the surface is D_stk^+ - q/2 (the jump across the
surface is q, as for the Laplace double layer).  Far particles: the smooth
quadrature of the stresslet.
"""
from __future__ import annotations

import math

import numpy as np

from . import legendre as L
from .geometry import PROLATE, local_point
from .laplace import multipliers
from .stokes import solid_value_and_gradient


def dl_coefficients(part, q_h, p):
    """Order-(p+1) coefficients: q_j (plain, zero-padded), y_i q_j (plain,
    [i][j]) and (q . nu) in the modified basis, by a product GL x trapezoid
    rule exact for degree 2p + 2."""
    nq = p + 3
    v, wv = np.polynomial.legendre.leggauss(nq)
    nph = 2 * nq + 2
    phi = 2 * np.pi * np.arange(nph) / nph
    V, PHI = np.repeat(v, nph), np.tile(phi, nq)
    W = np.repeat(wv, nph) * 2 * np.pi / nph
    sgn = -1.0 if part.kind == PROLATE else 1.0
    sw = np.sqrt(part.u0 ** 2 + sgn * V * V)
    qv = np.stack([L.real_Y(V, PHI, p) @ q_h[k] for k in range(3)], -1)      # q at the points (global frame)
    yl = local_point(part.kind, part.a, part.u0, V, PHI)
    yg = yl @ part.R.T
    gl = yl / np.array([part.A ** 2, part.A ** 2, part.C ** 2])
    nu = (gl / np.linalg.norm(gl, axis=1, keepdims=True)) @ part.R.T
    Y1 = L.real_Y(V, PHI, p + 1)
    nc1 = (p + 2) ** 2
    cq = np.zeros((3, nc1))
    cq[:, :(p + 1) ** 2] = q_h
    cyq = np.stack([[Y1.T @ (W * yg[:, i] * qv[:, j]) for j in range(3)] for i in range(3)])
    cqn = Y1.T @ (W * np.sum(qv * nu, -1) * sw)
    return cq, cyq, cqn


class StokesDLOracle:
    """Stokes double layer at the surface nodes and at arbitrary points."""

    def __init__(self, geom):
        self.g = geom
        p = geom.p
        self.mult = [multipliers(P.kind, P.a, P.u0, p + 1) for P in geom.parts]
        ns, ms = L.abs_m_table(p + 1)
        self.extD = [m["ext_D"][ns, ms] for m in self.mult]
        self.extS = [m["ext_S"][ns, ms] for m in self.mult]

    def _analytic(self, i, q_h, x, u_override=None):
        """Exterior-expansion value of D_stk for particle i at global points x."""
        g = self.g
        P = g.parts[i]
        p = g.p
        cq, cyq, cqn = dl_coefficients(P, q_h, p)
        xc = x - P.center
        gq = [solid_value_and_gradient(P, self.extD[i] * cq[j], x, p + 1, u_override)[1] for j in range(3)]
        gs = solid_value_and_gradient(P, self.extS[i] * cqn, x, p + 1, u_override)[1]
        div_q = sum(gq[j][:, j] for j in range(3))
        out = np.zeros((len(x), 3))
        for k in range(3):
            gyk = [solid_value_and_gradient(P, self.extD[i] * cyq[k, j], x, p + 1, u_override)[1] for j in range(3)]
            out[:, k] = -xc[:, k] * div_q + sum(gyk[j][:, j] for j in range(3)) - gs[:, k]
        return out

    def _quadrature(self, i, q_h, x, chunk=2048):
        P = self.g.parts[i]
        Y = L.real_Y(P.v, P.phi, P.p)
        q = np.stack([Y @ q_h[k] for k in range(3)], -1) * P.w[:, None]
        x = np.atleast_2d(x)
        out = np.zeros((len(x), 3))
        for c0 in range(0, len(x), chunk):
            r = x[c0:c0 + chunk, None, :] - P.x[None]
            d = np.linalg.norm(r, axis=-1)
            s = np.einsum("tjk,jk->tj", r, q) * np.einsum("tjk,jk->tj", r, P.nrm) / d ** 5
            out[c0:c0 + chunk] = 3.0 / (4 * math.pi) * np.einsum("tjk,tj->tk", r, s)
        return out

    def apply(self, q_h, mode="method", targets=None):
        """Principal-value D_stk[q] at the node indices `targets` (default all);
        q_h: (M, 3, (p+1)^2) plain coefficients.  Returns (T, 3)."""
        g = self.g
        tgt = np.arange(g.N) if targets is None else np.asarray(targets)
        out = np.zeros((len(tgt), 3))
        owner = g.owner[tgt]
        near = g.near_matrix(None if targets is None else tgt) if mode == "method" else None
        for i, P in enumerate(g.parts):
            own = owner == i
            if np.any(own):
                x = g.x[tgt[own]]
                Y = L.real_Y(P.v, P.phi, P.p)
                qn = np.stack([Y @ q_h[i, k] for k in range(3)], -1)[tgt[own] - i * g.G]
                out[own] += self._analytic(i, q_h[i], x, P.u0) - 0.5 * qn
            other = ~own
            sel_near = other & near[:, i] if mode == "method" else other
            sel_far = other & ~near[:, i] if mode == "method" else np.zeros_like(other)
            if np.any(sel_near):
                out[sel_near] += self._analytic(i, q_h[i], g.x[tgt[sel_near]])
            if np.any(sel_far):
                out[sel_far] += self._quadrature(i, q_h[i], g.x[tgt[sel_far]])
        return out

    def eval_points(self, X, q_h, mode="method"):
        """D_stk[q] at arbitrary points in the fluid (per-point near/far)."""
        g = self.g
        X = np.atleast_2d(np.asarray(X, dtype=np.float64))
        near = g.point_near_matrix(X)
        if mode == "exact":
            near = np.ones_like(near)
        out = np.zeros((len(X), 3))
        for i in range(g.M):
            if np.any(near[:, i]):
                out[near[:, i]] += self._analytic(i, q_h[i], X[near[:, i]])
            if np.any(~near[:, i]):
                out[~near[:, i]] += self._quadrature(i, q_h[i], X[~near[:, i]])
        return out
