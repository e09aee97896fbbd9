"""Stokes single layer through Laplace potentials (test infrastructure only).

Sec. 4.3, eq. (stokes), viscosity 1:
    S_stk[f](x)_k = 1/2 { S[f_k](x) - sum_j x_j d_k S[f_j](x) + d_k S[y . f](x) },
which follows from G_stk = (I/r + r r^T/r^3)/(8 pi) and G = 1/(4 pi r).  The
identity is translation invariant, so x and y are measured from the source
particle's centre.  Densities: f_k = sum f~_{k,nm} Y_nm / sqrt(u0^2 -+ v^2)
(modified basis, Theorem 2); y . f has a band-limited modified expansion of
order p + 1 (y is a degree-one harmonic on the surface), obtained here by a
quadrature forward transform that is exact for that degree.

Near particles: S and grad S of the exterior expansion (Theorem 2) at the
target; the gradient is the chain rule in the spheroidal unit vectors,
    grad F = e_u dF/du / h_u + e_v dF/dv / h_v + e_phi dF/dphi / h_phi,
with dP/dv from eq. (derivative) -- the quantity of eq. (dSLevalformula) with
nu replaced by the Cartesian unit vectors.  Own particle: the same formulas at
u = u0 (exterior limit; the jumps of grad S cancel in eq. (stokes) because
x = y there).  Far particles: the Stokeslet with the smooth quadrature.
"""
from __future__ import annotations

import math

import numpy as np

from . import legendre as L
from .geometry import PROLATE
from .laplace import multipliers

EIGHT_PI = 8.0 * math.pi


def _unit_vectors(kind, a, u, v, phi):
    """Local-frame e_u, e_v, e_phi and scale factors h_u, h_v, h_phi (Table 2)."""
    sgn = -1.0 if kind == PROLATE else 1.0
    su = np.sqrt(u * u + sgn)
    sv = np.sqrt(np.maximum(1.0 - v * v, 0.0))
    c, s = np.cos(phi), np.sin(phi)
    # derivatives of the Table 1 map
    xu = np.stack([a * u / su * sv * c, a * u / su * sv * s, a * v * np.ones_like(u)], -1)
    xv = np.stack([-a * su * v / sv * c, -a * su * v / sv * s, a * u * np.ones_like(v)], -1)
    xp = np.stack([-a * su * sv * s, a * su * sv * c, np.zeros_like(u)], -1)
    hu = np.linalg.norm(xu, axis=-1)
    hv = np.linalg.norm(xv, axis=-1)
    hp = np.linalg.norm(xp, axis=-1)
    return xu / hu[..., None], xv / hv[..., None], xp / hp[..., None], hu, hv, hp


def _basis_and_derivs(v, phi, p):
    """Real basis Y_nm(v, phi) and its v- and phi-derivatives, [..., coef]."""
    P = L.ferrers_P(v, p + 1)
    Y = np.zeros(v.shape + ((p + 1) ** 2,))
    Yv = np.zeros_like(Y)
    Yp = np.zeros_like(Y)
    omv2 = 1.0 - v * v
    for n in range(p + 1):
        for m in range(-n, n + 1):
            am = abs(m)
            N = L.norm_factor(n, am) * (math.sqrt(2.0) if m else 1.0)
            Pn = P[..., n, am]
            # eq. (derivative) on the cut: (1 - v^2) P' = (n+1) v P_n - (n-m+1) P_{n+1}
            dP = ((n + 1) * v * Pn - (n - am + 1) * P[..., n + 1, am]) / omv2
            if m > 0:
                t, dt = np.cos(am * phi), -am * np.sin(am * phi)
            elif m < 0:
                t, dt = np.sin(am * phi), am * np.cos(am * phi)
            else:
                t, dt = np.ones_like(phi), np.zeros_like(phi)
            k = L.coeff_index(n, m)
            Y[..., k] = N * Pn * t
            Yv[..., k] = N * dP * t
            Yp[..., k] = N * Pn * dt
    return Y, Yv, Yp


def solid_value_and_gradient(part, coef_ext, x, p, u_override=None):
    """F and grad F (global frame) of the exterior expansion
    F = sum_nm coef_ext[nm] R_n^|m|(u) Y_nm(v, phi), R = Q (x = u or i u),
    at global points x.  coef_ext already contains the Theorem 2 factor.
    u_override: evaluate at this u (the own surface, u = u0)."""
    u, v, phi = part.to_spheroidal(x)
    if u_override is not None:
        u = np.full_like(u, u_override)
    xa = u if part.kind == PROLATE else 1j * u
    Pq = L.legendre_P(xa, p + 2)
    Q = L.legendre_Q(xa, p + 2, Pq)
    dQ = L.derivative(Q, xa, p + 1)          # d/dx
    dudx = 1.0 if part.kind == PROLATE else 1j
    ns, ms = L.abs_m_table(p)
    R = Q[..., ns, ms]
    dR = dQ[..., ns, ms] * dudx              # d/du
    Y, Yv, Yp = _basis_and_derivs(v, phi, p)
    F = np.real(np.sum(coef_ext * R * Y, -1))
    Fu = np.real(np.sum(coef_ext * dR * Y, -1))
    Fv = np.real(np.sum(coef_ext * R * Yv, -1))
    Fp = np.real(np.sum(coef_ext * R * Yp, -1))
    eu, ev, ep, hu, hv, hp = _unit_vectors(part.kind, part.a, u, v, phi)
    g_loc = eu * (Fu / hu)[..., None] + ev * (Fv / hv)[..., None] + ep * (Fp / hp)[..., None]
    return F, g_loc @ part.R.T


def ydotf_modified_coefficients(part, f_t, p):
    """Modified-basis coefficients (order p+1) of (y - c) . f, by a product
    GL x trapezoid forward transform exact for degree 2p + 2."""
    q = p + 3
    v, wv = np.polynomial.legendre.leggauss(q)
    nph = 2 * q + 2
    phi = 2 * np.pi * np.arange(nph) / nph
    V = np.repeat(v, nph)
    PHI = np.tile(phi, q)
    W = np.repeat(wv, nph) * 2 * np.pi / nph
    sgn = -1.0 if part.kind == PROLATE else 1.0
    sw = np.sqrt(part.u0 ** 2 + sgn * V * V)
    Yp = L.real_Y(V, PHI, p)
    fvals = np.stack([(Yp @ f_t[k]) / sw for k in range(3)], -1)           # f at the points
    from .geometry import local_point
    yl = local_point(part.kind, part.a, part.u0, V, PHI)
    yg = yl @ part.R.T                                                     # y - c, global frame
    g = np.sum(yg * fvals, -1) * sw
    Y1 = L.real_Y(V, PHI, p + 1)
    return Y1.T @ (W * g)


class StokesOracle:
    """Stokes single-layer apply at every surface node (eq. (stokes))."""

    def __init__(self, geom):
        self.g = geom
        p = geom.p
        self.mult = [multipliers(P.kind, P.a, P.u0, p + 1) for P in geom.parts]

    def _ext_coef(self, i, coef, order):
        ns, ms = L.abs_m_table(order)
        return self.mult[i]["ext_S"][ns, ms] * coef

    def apply(self, f_t, mode="method", targets=None):
        """f_t: (M, 3, (p+1)^2).  Returns (T, 3) velocities."""
        g = self.g
        p = g.p
        tgt = np.arange(g.N) if targets is None else np.asarray(targets)
        U = np.zeros((len(tgt), 3))
        owner = g.owner[tgt]
        near = g.near_matrix(None if targets is None else tgt) if mode == "method" else None
        for i, P in enumerate(g.parts):
            own = owner == i
            other = ~own
            if mode == "method":
                sel_an = other & near[:, i]
                sel_far = other & ~near[:, i]
            else:
                sel_an = other
                sel_far = np.zeros_like(other)
            cs = [self._ext_coef(i, np.pad(f_t[i, k], (0, (p + 2) ** 2 - (p + 1) ** 2)), p + 1) for k in range(3)]
            cy = self._ext_coef(i, ydotf_modified_coefficients(P, f_t[i], p), p + 1)
            for sel, u_ov in ((own, P.u0), (sel_an, None)):
                if not np.any(sel):
                    continue
                x = g.x[tgt[sel]]
                xc = x - P.center
                Fk, Gk = [], []
                for k in range(3):
                    F, Gr = solid_value_and_gradient(P, cs[k], x, p + 1, u_ov)
                    Fk.append(F)
                    Gk.append(Gr)
                Fy, Gy = solid_value_and_gradient(P, cy, x, p + 1, u_ov)
                for k in range(3):
                    val = Fk[k] + Gy[:, k]
                    for j in range(3):
                        val = val - xc[:, j] * Gk[j][:, k]
                    U[sel, k] += 0.5 * val
            if np.any(sel_far):
                U[sel_far] += stokeslet_quadrature(P, f_t[i], g.x[tgt[sel_far]])
        return U

    def eval_points(self, X, f_t, mode="method"):
        """Velocity (T, 3) and pressure (T,) of the single layer at arbitrary
        points in the fluid (Sec. 4.1 particle-to-target algorithm with
        eq. (stokes)).  Pressure p = -sum_j d_j S[f_j]: the printed pressure
        kernel r / (4 pi |r|^3); the printed identity in terms of gradients of
        S carries the opposite sign (d_j (1/r) = -r_j / r^3)."""
        g = self.g
        p = g.p
        X = np.atleast_2d(np.asarray(X, dtype=np.float64))
        near = g.point_near_matrix(X)
        if mode == "exact":
            near = np.ones_like(near)
        U = np.zeros((len(X), 3))
        Pr = np.zeros(len(X))
        for i, P in enumerate(g.parts):
            sel = near[:, i]
            if np.any(sel):
                x = X[sel]
                xc = x - P.center
                cs = [self._ext_coef(i, np.pad(f_t[i, k], (0, (p + 2) ** 2 - (p + 1) ** 2)), p + 1) for k in range(3)]
                cy = self._ext_coef(i, ydotf_modified_coefficients(P, f_t[i], p), p + 1)
                Fk, Gk = zip(*[solid_value_and_gradient(P, cs[k], x, p + 1) for k in range(3)])
                _, Gy = solid_value_and_gradient(P, cy, x, p + 1)
                for k in range(3):
                    val = Fk[k] + Gy[:, k]
                    for j in range(3):
                        val = val - xc[:, j] * Gk[j][:, k]
                    U[sel, k] += 0.5 * val
                Pr[sel] -= Gk[0][:, 0] + Gk[1][:, 1] + Gk[2][:, 2]
            far = ~sel
            if np.any(far):
                U[far] += stokeslet_quadrature(P, f_t[i], X[far])
                Pr[far] += pressure_quadrature(P, f_t[i], X[far])
        return U, Pr


def pressure_quadrature(part, f_t, x, chunk=2048):
    """sum_j w_j P(x, y_j) . f(y_j), P = r / (4 pi |r|^3)."""
    Y = L.real_Y(part.v, part.phi, part.p)
    f = np.stack([(Y @ f_t[k]) / part.sqrt_w for k in range(3)], -1) * part.w[:, None]
    x = np.atleast_2d(x)
    out = np.zeros(len(x))
    for c0 in range(0, len(x), chunk):
        r = x[c0:c0 + chunk, None, :] - part.x[None]
        d = np.linalg.norm(r, axis=-1)
        out[c0:c0 + chunk] = (np.einsum("tjk,jk->tj", r, f) / d ** 3).sum(1) / (4 * math.pi)
    return out


def stokeslet_quadrature(part, f_t, x, chunk=2048):
    """sum_j w_j G_stk(x, y_j) f(y_j) over the particle's nodes."""
    Y = L.real_Y(part.v, part.phi, part.p)
    f = np.stack([(Y @ f_t[k]) / part.sqrt_w for k in range(3)], -1) * part.w[:, None]
    x = np.atleast_2d(x)
    U = np.zeros((len(x), 3))
    for c0 in range(0, len(x), chunk):
        r = x[c0:c0 + chunk, None, :] - part.x[None]
        d = np.linalg.norm(r, axis=-1)
        rf = np.einsum("tjk,jk->tj", r, f)
        U[c0:c0 + chunk] = (np.einsum("jk,tj->tk", f, 1.0 / d) + np.einsum("tjk,tj->tk", r, rf / d ** 3)) / EIGHT_PI
    return U
