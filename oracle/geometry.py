"""Spheroid geometry for the oracle (test infrastructure only).

Sec. 2.1 / Table 1: prolate  x = (a sqrt(u^2-1) sqrt(1-v^2) cos phi, ..., a u v), u > 1
                    oblate   x = (a sqrt(u^2+1) sqrt(1-v^2) cos phi, ..., a u v), u > 0
The surface u = u0 has semi-axes A = a sqrt(u0^2 -+ 1) (equatorial) and
C = a u0 (polar), so  prolate: a = sqrt(C^2 - A^2), oblate: a = sqrt(A^2 - C^2),
u0 = C / a.  Table 2 gives dS = a^2 sqrt(u0^2 -+ v^2) sqrt(u0^2 -+ 1) dv dphi.

Sec. 4 ("Integral density representation"): nodes are the (p+1) Gauss-Legendre
points in v times n_phi equispaced points in phi.  The paper prints
n_phi = 2p; this build uses n_phi = 2(p+1) by default (with 2p the sin(p phi)
mode vanishes at every node).  The node order is v-major, phi-minor.

Sec. 4.1: target x is near to particle i iff d(x, Gamma_i) < eta diam(Gamma_i);
here the threshold is near_factor x (major semi-axis of i), i.e. eta = 1/2
with diam = 2 x major semi-axis.  Distances are exact point-to-spheroid
distances (meridian-plane point-to-ellipse, golden-section search over the
ellipse parameter).
"""
from __future__ import annotations

import math

import numpy as np

PROLATE = 0
OBLATE = 1


def spheroid_params(kind, A, C):
    """(a, u0) from the semi-axes (Sec. 2.1)."""
    kind = np.asarray(kind)
    A = np.asarray(A, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    a = np.where(kind == PROLATE, np.sqrt(np.abs(C * C - A * A)), np.sqrt(np.abs(A * A - C * C)))
    return a, C / a


def quat_to_R(q):
    """Rotation matrix of a unit quaternion (w, x, y, z)."""
    q = np.asarray(q, dtype=np.float64)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([
        np.stack([w * w + x * x - y * y - z * z, 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), w * w - x * x + y * y - z * z, 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), w * w - x * x - y * y + z * z], -1),
    ], -2)


def gauss_legendre(n: int):
    """Gauss-Legendre nodes (ascending) and weights on [-1, 1]."""
    v, w = np.polynomial.legendre.leggauss(n)
    return v, w


def grid(p: int, n_phi: int | None = None):
    """Tensor grid (v_j, phi_k), v-major, and the GL weights."""
    if n_phi is None:
        n_phi = 2 * (p + 1)
    v, wv = gauss_legendre(p + 1)
    phi = 2.0 * math.pi * np.arange(n_phi) / n_phi
    V = np.repeat(v, n_phi)
    PHI = np.tile(phi, p + 1)
    WV = np.repeat(wv, n_phi)
    return V, PHI, WV, n_phi


def local_point(kind, a, u, v, phi):
    """Table 1 map (u, v, phi) -> local Cartesian."""
    su = np.sqrt(u * u - 1.0) if kind == PROLATE else np.sqrt(u * u + 1.0)
    sv = np.sqrt(np.maximum(1.0 - v * v, 0.0))
    return np.stack([a * su * sv * np.cos(phi), a * su * sv * np.sin(phi), a * u * v], axis=-1)


class Particle:
    """One spheroid with its quadrature nodes."""

    def __init__(self, kind, A, C, center, quat, p, n_phi=None):
        self.kind = int(kind)
        self.A = float(A)
        self.C = float(C)
        a, u0 = spheroid_params(kind, A, C)
        self.a = float(a)
        self.u0 = float(u0)
        self.center = np.asarray(center, dtype=np.float64)
        self.R = quat_to_R(np.asarray(quat, dtype=np.float64) / np.linalg.norm(quat))
        self.p = p
        V, PHI, WV, self.n_phi = grid(p, n_phi)
        self.v, self.phi = V, PHI
        sgn = -1.0 if self.kind == PROLATE else 1.0
        u0 = self.u0
        # Table 2: dS = a^2 sqrt(u0^2 -+ v^2) sqrt(u0^2 -+ 1) dv dphi
        self.dS_factor = self.a ** 2 * np.sqrt(u0 * u0 + sgn * V * V) * np.sqrt(u0 * u0 + sgn)
        self.w = WV * (2.0 * math.pi / self.n_phi) * self.dS_factor
        xl = local_point(self.kind, self.a, u0, V, PHI)
        # outward unit normal: gradient of x1^2/A^2 + x2^2/A^2 + x3^2/C^2
        g = xl / np.array([self.A ** 2, self.A ** 2, self.C ** 2])
        nl = g / np.linalg.norm(g, axis=1, keepdims=True)
        self.x = xl @ self.R.T + self.center
        self.nrm = nl @ self.R.T
        self.x_local = xl
        # modified-basis weight sqrt(u0^2 -+ v^2) of Sec. 3.2
        self.sqrt_w = np.sqrt(u0 * u0 + sgn * V * V)

    @property
    def G(self):
        return self.v.shape[0]

    @property
    def major(self):
        return max(self.A, self.C)

    def to_local(self, x):
        return (np.asarray(x) - self.center) @ self.R

    def to_spheroidal(self, x):
        """(u, v, phi) of global points in this particle's coordinates."""
        return cart_to_spheroidal(self.to_local(x), self.kind, self.a)


def cart_to_spheroidal(xl, kind, a):
    """Inverse of Table 1.  With X = rho/a, Z = z/a and s = u^2 - 1 (prolate)
    or s = u^2 (oblate), Table 1 gives X^2 = s (1 - v^2) and Z^2 = (s + 1) v^2
    (prolate), X^2 = (s + 1)(1 - v^2) and Z^2 = s v^2 (oblate), so s is the
    positive root of
        prolate: s^2 + (1 - X^2 - Z^2) s - X^2 = 0,
        oblate:  s^2 + (1 - X^2 - Z^2) s - Z^2 = 0,
    taken in the form without cancellation (c / q or q with the sign of the
    linear coefficient).  sqrt(1 - v^2) = X / sqrt(s) (prolate) or
    X / sqrt(s + 1) (oblate) is exact on the symmetry axis, so v is taken from
    it where |v| > 1/2 (v = +-1 exactly on the axis) and as Z / u elsewhere."""
    xl = np.asarray(xl, dtype=np.float64)
    rho = np.hypot(xl[..., 0], xl[..., 1])
    z = xl[..., 2]
    phi = np.arctan2(xl[..., 1], xl[..., 0])
    X = rho / a
    Z = z / a
    B = (1.0 - X) * (1.0 + X) - Z * Z
    c = X * X if kind == PROLATE else Z * Z
    disc = np.sqrt(B * B + 4.0 * c)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(B > 0.0, 2.0 * c / (B + disc), 0.5 * (disc - B))
        if kind == PROLATE:
            u = np.sqrt(1.0 + s)
            sv = np.where(s > 0.0, X / np.sqrt(s), 1.0)
        else:
            u = np.sqrt(s)
            sv = X / np.sqrt(1.0 + s)
        sv = np.minimum(sv, 1.0)
        v_lin = np.where(u > 0.0, Z / u, 0.0)
    v_pol = np.sign(Z) * np.sqrt(np.maximum(1.0 - sv * sv, 0.0))
    v = np.clip(np.where(np.abs(v_lin) > 0.5, v_pol, v_lin), -1.0, 1.0)
    return u, v, phi


def point_spheroid_distance(xl, A, C, iters: int = 90):
    """Distance from local points to the spheroid surface (positive outside),
    minimising |(A cos t, C sin t) - (rho, |z|)| over t in [0, pi/2] by
    golden-section search (unimodal for exterior points)."""
    xl = np.asarray(xl, dtype=np.float64)
    rho = np.hypot(xl[..., 0], xl[..., 1])
    z = np.abs(xl[..., 2])
    inside = (rho / A) ** 2 + (z / C) ** 2 < 1.0
    g = (math.sqrt(5.0) - 1.0) / 2.0
    lo = np.zeros_like(rho)
    hi = np.full_like(rho, math.pi / 2)

    def f(t):
        return (A * np.cos(t) - rho) ** 2 + (C * np.sin(t) - z) ** 2

    c = hi - g * (hi - lo)
    d = lo + g * (hi - lo)
    fc, fd = f(c), f(d)
    for _ in range(iters):
        left = fc < fd
        hi = np.where(left, d, hi)
        lo = np.where(left, lo, c)
        c_new = hi - g * (hi - lo)
        d_new = lo + g * (hi - lo)
        c, d = c_new, d_new
        fc, fd = f(c), f(d)
    t = 0.5 * (lo + hi)
    dist = np.sqrt(np.minimum(np.minimum(f(t), f(np.zeros_like(t))), f(np.full_like(t, math.pi / 2))))
    return np.where(inside, -dist, dist)


class SuspensionGeom:
    """All particles of a suspension and the per-target near sets."""

    def __init__(self, kind, A, C, center, quat, p, n_phi=None, near_factor=1.0):
        self.parts = [Particle(kind[i], A[i], C[i], center[i], quat[i], p, n_phi) for i in range(len(kind))]
        self.p = p
        self.M = len(self.parts)
        self.G = self.parts[0].G if self.M else 0
        self.N = self.M * self.G
        self.near_factor = near_factor
        self.x = np.concatenate([P.x for P in self.parts]) if self.M else np.zeros((0, 3))
        self.nrm = np.concatenate([P.nrm for P in self.parts]) if self.M else np.zeros((0, 3))
        self.owner = np.repeat(np.arange(self.M), self.G)
        self._near = None
        self._dist = None

    @classmethod
    def from_suspension(cls, s, near_factor=1.0, n_phi=None):
        return cls(s.kind, s.A, s.C, s.center, s.quat, s.p, n_phi, near_factor)

    def distances(self, targets=None):
        """(T, M) signed target-to-spheroid distances (own particle: 0) for the
        target node indices `targets` (default all).  Pairs whose bounding
        sphere is already farther than the near threshold get the lower bound
        |x - c| - major instead of the exact distance."""
        if targets is None and self._dist is not None:
            return self._dist
        tg = np.arange(self.N) if targets is None else np.asarray(targets)
        x = self.x[tg]
        D = np.zeros((len(tg), self.M))
        for i, P in enumerate(self.parts):
            lb = np.linalg.norm(x - P.center, axis=1) - P.major
            exact = lb < 2.0 * self.near_factor * P.major
            D[:, i] = lb
            if np.any(exact):
                D[exact, i] = point_spheroid_distance(P.to_local(x[exact]), P.A, P.C)
            D[self.owner[tg] == i, i] = 0.0
        if targets is None:
            self._dist = D
        return D

    def point_distances(self, X):
        """(T, M) signed distances from arbitrary points X (T, 3) to every
        spheroid (negative inside), with the same bounding-sphere shortcut as
        distances() for pairs that are certainly far."""
        X = np.atleast_2d(np.asarray(X, dtype=np.float64))
        D = np.zeros((X.shape[0], self.M))
        for i, P in enumerate(self.parts):
            lb = np.linalg.norm(X - P.center, axis=1) - P.major
            exact = lb < 2.0 * self.near_factor * P.major
            D[:, i] = lb
            if np.any(exact):
                D[exact, i] = point_spheroid_distance(P.to_local(X[exact]), P.A, P.C)
        return D

    def point_near_matrix(self, X):
        """(T, M) bool for arbitrary points in the fluid: particle i is near
        point x iff dist(x, Gamma_i) < near_factor x major semi-axis of i
        (Sec. 4.1, particle-to-target algorithm: classification per point).
        Raises ValueError for a point inside a spheroid."""
        D = self.point_distances(X)
        thr = np.array([self.near_factor * P.major for P in self.parts])
        # a point on a surface to rounding (|D| <= 1e-12 x major) is taken
        # as the exterior limit
        maj = np.array([P.major for P in self.parts])
        bad = D < -1e-12 * maj[None, :]
        if np.any(bad):
            t, i = np.argwhere(bad)[0]
            raise ValueError(f"point {t} lies inside spheroid {i}")
        return D < thr[None, :]

    def near_matrix(self, targets=None):
        """(T, M) bool: source i is near target t (own particle excluded)."""
        if targets is None and self._near is not None:
            return self._near
        tg = np.arange(self.N) if targets is None else np.asarray(targets)
        D = self.distances(targets)
        thr = np.array([self.near_factor * P.major for P in self.parts])
        near = D < thr[None, :]
        near[np.arange(len(tg)), self.owner[tg]] = False
        if targets is None:
            self._near = near
        return near

    def near_margin(self):
        """Smallest relative distance of any (target, other particle) from the
        near threshold; the near sets are well defined when this is not tiny."""
        D = self.distances()
        thr = np.array([self.near_factor * P.major for P in self.parts])
        rel = np.abs(D - thr[None, :]) / thr[None, :]
        rel[np.arange(self.N), self.owner] = np.inf
        return float(rel.min()) if rel.size else np.inf
