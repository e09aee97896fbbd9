"""Oversampled direct quadrature (test infrastructure only).

Used only to pin the analytic formulas of the oracle: for a target at a
positive distance from the surface, the layer-potential integrands
    S: G(x, y) sigma(y) dS(y),   D: dG/dnu_y(x, y) mu(y) dS(y)
are smooth, and a Gauss-Legendre (in v) x trapezoid (in phi) product rule on a
fine grid converges spectrally.  The rule, the surface element and the normal
are those of Sec. 2.1-2.2 (Tables 1-2); the density is the band-limited
expansion itself (sigma from modified coefficients, mu from plain ones).
"""
from __future__ import annotations

import math

import numpy as np

from . import legendre as L
from .geometry import PROLATE, local_point, quat_to_R, spheroid_params


def fine_surface(kind, A, C, center, quat, nv, nphi):
    a, u0 = spheroid_params(kind, A, C)
    a, u0 = float(a), float(u0)
    v, wv = np.polynomial.legendre.leggauss(nv)
    phi = 2.0 * math.pi * np.arange(nphi) / nphi
    V = np.repeat(v, nphi)
    PHI = np.tile(phi, nv)
    W = np.repeat(wv, nphi) * 2.0 * math.pi / nphi
    sgn = -1.0 if kind == PROLATE else 1.0
    W = W * a * a * np.sqrt(u0 * u0 + sgn * V * V) * math.sqrt(u0 * u0 + sgn)
    xl = local_point(kind, a, u0, V, PHI)
    g = xl / np.array([A * A, A * A, C * C])
    nl = g / np.linalg.norm(g, axis=1, keepdims=True)
    R = quat_to_R(np.asarray(quat, dtype=np.float64) / np.linalg.norm(quat))
    y = xl @ R.T + np.asarray(center)
    ny = nl @ R.T
    return V, PHI, W, y, ny, np.sqrt(u0 * u0 + sgn * V * V)


def brute_layers(kind, A, C, center, quat, p, x, sigma_t=None, mu_h=None,
                 nv=160, nphi=320, chunk=64):
    """S[sigma](x), D[mu](x) by an nv x nphi product rule."""
    V, PHI, W, y, ny, sw = fine_surface(kind, A, C, center, quat, nv, nphi)
    Y = L.real_Y(V, PHI, p)
    sv = None if sigma_t is None else (Y @ sigma_t) / sw
    mv = None if mu_h is None else Y @ mu_h
    x = np.atleast_2d(x)
    S = np.zeros(len(x)) if sv is not None else None
    D = np.zeros(len(x)) if mv is not None else None
    for c0 in range(0, len(x), chunk):
        r = x[c0:c0 + chunk, None, :] - y[None, :, :]
        d = np.linalg.norm(r, axis=-1)
        if S is not None:
            S[c0:c0 + chunk] = (1.0 / (4 * math.pi * d)) @ (W * sv)
        if D is not None:
            rn = np.einsum("tjk,jk->tj", r, ny)
            D[c0:c0 + chunk] = (rn / (4 * math.pi * d ** 3)) @ (W * mv)
    return S, D


def brute_stokeslet(kind, A, C, center, quat, p, x, f_t, nv=160, nphi=320, chunk=64):
    """Stokes single layer u(x) = int G_stk(x, y) f(y) dS(y), viscosity 1,
    G_stk = (I/r + r r^T / r^3) / (8 pi); f given by three modified-basis
    expansions f_t[k] (one per Cartesian component)."""
    V, PHI, W, y, ny, sw = fine_surface(kind, A, C, center, quat, nv, nphi)
    Y = L.real_Y(V, PHI, p)
    f = np.stack([(Y @ f_t[k]) / sw for k in range(3)], axis=-1) * W[:, None]
    x = np.atleast_2d(x)
    U = np.zeros((len(x), 3))
    for c0 in range(0, len(x), chunk):
        r = x[c0:c0 + chunk, None, :] - y[None, :, :]
        d = np.linalg.norm(r, axis=-1)
        rf = np.einsum("tjk,jk->tj", r, f)
        U[c0:c0 + chunk] = (np.einsum("jk,tj->tk", f, 1.0 / d) + np.einsum("tjk,tj->tk", r, rf / d ** 3)) / (8 * math.pi)
    return U


def brute_stokes_pressure(kind, A, C, center, quat, p, x, f_t, nv=160, nphi=320, chunk=64):
    """Pressure of the Stokes single layer, p(x) = int P(x, y) . f(y) dS(y)
    with the printed kernel P = r / (4 pi |r|^3), r = x - y."""
    V, PHI, W, y, ny, sw = fine_surface(kind, A, C, center, quat, nv, nphi)
    Y = L.real_Y(V, PHI, p)
    f = np.stack([(Y @ f_t[k]) / sw for k in range(3)], axis=-1) * W[:, None]
    x = np.atleast_2d(x)
    out = np.zeros(len(x))
    for c0 in range(0, len(x), chunk):
        r = x[c0:c0 + chunk, None, :] - y[None, :, :]
        d = np.linalg.norm(r, axis=-1)
        out[c0:c0 + chunk] = (np.einsum("tjk,jk->tj", r, f) / d ** 3).sum(1) / (4 * math.pi)
    return out


def brute_stresslet(kind, A, C, center, quat, p, x, q_h, nv=160, nphi=320, chunk=64):
    """Stokes double layer, D[q](x)_i = 3/(4 pi) int (r.q)(r.nu) r_i / |r|^5 dS,
    r = x - y, nu the outward normal (the sign that makes D[const] = -q
    inside, like the Laplace double layer); q by its plain coefficients q_h[k]
    per Cartesian component."""
    V, PHI, W, y, ny, sw = fine_surface(kind, A, C, center, quat, nv, nphi)
    Y = L.real_Y(V, PHI, p)
    q = np.stack([Y @ q_h[k] for k in range(3)], axis=-1) * W[:, None]
    x = np.atleast_2d(x)
    out = np.zeros((len(x), 3))
    for c0 in range(0, len(x), chunk):
        r = x[c0:c0 + chunk, None, :] - y[None, :, :]
        d = np.linalg.norm(r, axis=-1)
        s = np.einsum("tjk,jk->tj", r, q) * np.einsum("tjk,jk->tj", r, ny) / d ** 5
        out[c0:c0 + chunk] = 3.0 / (4 * math.pi) * np.einsum("tjk,tj->tk", r, s)
    return out
