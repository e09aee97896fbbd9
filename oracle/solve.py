"""Forward spheroidal transform and the exterior Laplace boundary-value
solves of the numerical section (test infrastructure only).

Forward transform (Sec. 2.3 / Sec. 4 "Integral density representation"):
the coefficients of a surface function f in the real orthonormal basis are
    f^_nm = int int f Y_nm dv dphi ~ sum_j w_j (2 pi / n_phi) sum_k f(v_j, phi_k) Y_nm(v_j, phi_k),
exact for band-limited f of degree <= p on the (p+1) GL x n_phi >= 2p+1 grid;
the modified-basis coefficients (Sec. 3.2) are those of f sqrt(u0^2 -+ v^2).

Exterior Dirichlet problem (Sec. 5.1): u = D+[sigma] + C[sigma] with
    1/2 sigma + D[sigma] + C[sigma] = f on the surfaces,
completions C_I[sigma](x) = sum_i (int sigma_i dS) / |x - c_i|, its scaled
form eta_i C_I, the single layer S[sigma] and eta_i S[sigma], eta_i from the
paper's heuristic table (per particle, from the aspect ratio).
Exterior Neumann problem: u = S+[rho] with -1/2 rho + S'[rho] = g.
Both are written in coefficient space: the unknown is the density's
coefficient vector (plain for Dirichlet, modified for Neumann), and the
operator is the forward transform of the operator's node values, so that the
identity term is exact.  Solved densely (numpy.linalg.solve) on small cases.
"""
from __future__ import annotations

import math

import numpy as np

from . import legendre as L
from .deriv import DerivOracle
from .geometry import PROLATE
from .laplace import LaplaceOracle, density_values

COMPLETIONS = ("CI", "etaCI", "S", "etaS")


def analysis(part, values, modified=False):
    """Forward transform of node values of one particle -> (p+1)^2 coefficients."""
    W = np.repeat(np.polynomial.legendre.leggauss(part.p + 1)[1], part.n_phi) * (2 * math.pi / part.n_phi)
    f = values * part.sqrt_w if modified else values
    return L.real_Y(part.v, part.phi, part.p).T @ (W * f)


def synthesis(part, coef, modified=False):
    """Node values of sum coef Y (divided by sqrt(u0^2 -+ v^2) if modified)."""
    f = L.real_Y(part.v, part.phi, part.p) @ coef
    return f / part.sqrt_w if modified else f


def surface_area_unit_major(kind, eps):
    """Area of the spheroid with major semi-axis 1 and aspect ratio 1/eps."""
    if eps >= 1.0:
        return 4 * math.pi
    e = math.sqrt(1 - eps * eps)
    if kind == PROLATE:          # semi-axes (eps, eps, 1)
        return 2 * math.pi * eps * eps * (1 + math.asin(e) / (eps * e))
    return 2 * math.pi * (1 + eps * eps / e * math.atanh(e))     # semi-axes (1, 1, eps)


def eta_table(kind, A, C, completion):
    """Scaling eta of a completion term for one particle (the paper's
    heuristic table; eps = 1 / aspect ratio)."""
    R = max(A, C) / min(A, C)
    eps = 1.0 / R
    if completion in ("CI", "S"):
        return 1.0
    if completion == "etaCI":
        if kind == PROLATE or R <= 3:
            return eps / surface_area_unit_major(kind, eps)
        return 0.06
    if kind == PROLATE:
        return 0.5 if R <= 3 else 1.0 / (2 * eps * math.log(1 / eps))
    return 1.0 / (4 * eps) + 0.25 if R <= 3 else 1.0


class BVPOracle:
    """Coefficient-space operators and solves of the exterior Dirichlet and
    Neumann problems on a suspension."""

    def __init__(self, geom, mode="method"):
        self.g = geom
        self.mode = mode
        self.lo = LaplaceOracle(geom)
        self.do = DerivOracle(geom)
        self.nc = (geom.p + 1) ** 2

    def _split(self, nodes):
        G = self.g.G
        return [nodes[i * G:(i + 1) * G] for i in range(self.g.M)]

    def transform(self, nodes, modified=False):
        """(N,) node values -> (M, (p+1)^2) coefficients."""
        return np.stack([analysis(P, v, modified) for P, v in zip(self.g.parts, self._split(nodes))])

    def etas(self, completion):
        return np.array([eta_table(P.kind, P.A, P.C, completion) for P in self.g.parts])

    def completion_terms(self, mu_h, completion):
        """Modified coefficients sigma~ (S completions) or centre charges q
        (C_I completions) of the completion applied to the density sum mu^ Y."""
        eta = self.etas(completion)
        sig_nodes = [synthesis(P, mu_h[i]) for i, P in enumerate(self.g.parts)]
        if completion in ("S", "etaS"):
            st = np.stack([eta[i] * analysis(P, sig_nodes[i], modified=True) for i, P in enumerate(self.g.parts)])
            return st, np.zeros(self.g.M)
        q = np.array([eta[i] * np.sum(P.w * sig_nodes[i]) for i, P in enumerate(self.g.parts)])
        return np.zeros_like(mu_h), q

    def charges_field(self, q, X):
        """sum_i q_i / |x - c_i| (the C_I kernel as printed: no 1/(4 pi))."""
        cen = np.array([P.center for P in self.g.parts])
        return (q[None, :] / np.linalg.norm(np.atleast_2d(X)[:, None, :] - cen[None], axis=-1)).sum(1)

    def dirichlet_apply(self, mu_h, completion):
        """K x = 1/2 x + T(D[x] + C[x]) for plain coefficients x = mu^."""
        st, q = self.completion_terms(mu_h, completion)
        has_s = completion in ("S", "etaS")
        Sv, Dv = self.lo.apply(st if has_s else None, mu_h, self.mode)
        u = Dv + (Sv if has_s else self.charges_field(q, self.g.x))
        return 0.5 * mu_h + self.transform(u)

    def neumann_apply(self, rho_t):
        """K x = -1/2 x + T_mod(S'[x]) for modified coefficients x = rho~."""
        Sp, _ = self.do.apply(rho_t, None, self.mode)
        return -0.5 * rho_t + self.transform(Sp, modified=True)

    def _dense(self, op):
        n = self.g.M * self.nc
        K = np.zeros((n, n))
        for k in range(n):
            e = np.zeros(n)
            e[k] = 1.0
            K[:, k] = op(e.reshape(self.g.M, self.nc)).ravel()
        return K

    def solve_dirichlet(self, f_nodes, completion="etaS"):
        """Returns (mu^, sigma~, q): the density's plain coefficients and the
        completion's modified coefficients / centre charges."""
        b = self.transform(f_nodes).ravel()
        K = self._dense(lambda x: self.dirichlet_apply(x, completion))
        mu = np.linalg.solve(K, b).reshape(self.g.M, self.nc)
        st, q = self.completion_terms(mu, completion)
        return mu, st, q

    def solve_neumann(self, g_nodes):
        """Returns rho~ (modified coefficients) with u = S[rho]."""
        b = self.transform(g_nodes, modified=True).ravel()
        K = self._dense(self.neumann_apply)
        return np.linalg.solve(K, b).reshape(self.g.M, self.nc)

    def eval_dirichlet(self, X, mu, st, q):
        S, D = self.lo.eval_points(X, st, mu, self.mode)
        return D + S + self.charges_field(q, X)

    def eval_neumann(self, X, rho_t):
        S, _ = self.lo.eval_points(X, rho_t, None, self.mode)
        return S
